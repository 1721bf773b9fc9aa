// Explicit inverses P_e^{-1} of the float32 block forms by Gauss-Jordan elimination with
// partial pivoting (SIMT forms), their variants and the per-device tuner.  The tensor-core
// form is in gj_tc.cu.
#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "blocks.cuh"
#include "common.cuh"
#include "gj.cuh"

namespace emg {

emg_status launch_gj_tc(emg_ctx* c, int B, float* blk, bool* built);

// Blocked form of the same Gauss-Jordan inversion (right-looking, panels of NB = 8 pivot
// columns), SIMT.  Layout of k_gj_cols: lane tx owns rows tx + 32 i, warp w owns columns
// w + W j; after every panel each thread rotates its column slots by NB / W, so the next
// panel's columns always sit in slots 0 .. NB/W - 1 (no runtime-indexed register access).
// The NB steps of a panel act on every column c outside it as A[:, c] <- T A[:, c],
// T = T_{k0+NB-1} ... T_{k0} (T_k: the elementary Gauss-Jordan transform of step k, identity
// but for column p_k).  T differs from I only in the pivot-row columns P, and the in-place
// rule leaves exactly F = T[:, P] in the panel's columns once the panel is factored, so
//   rows r outside P:  A[r, c] <- A[r, c] + sum_s F[r, s] A[p_s, c]
//   rows r = p_t in P: A[r, c] <-           sum_s F[r, s] A[p_s, c]
// (writing the second case without "A[r, c] +" avoids forming T[p_t, p_t] - 1 in float).
// Per panel: (A) the panel's owners copy its columns to shared memory; (B) warp 0 alone
// factors the panel in registers (the in-place steps of k_gj_rot on B x NB values: pivot
// search by warp reductions, the pivot row by shuffles: no block barrier inside) and
// publishes F and the pivot rows; (C) every warp gathers the pivot rows' entries of its own
// columns in a warp-private buffer (no block barrier) and applies the rank-NB update,
// s = 0 .. NB-1 in order, one FMA per term.  Pivot choice and tie rule are those of the
// unblocked forms in gj_tile.cu and gj_cols.cu (largest |a_rk| among the unused rows, lowest
// row on ties, the lowest unused row if no candidate is a number).  The summation order
// differs from the unblocked forms (results agree to float rounding, not bitwise); the
// variants with different W compute identically.  The inverse is written column-major, as
// by the other forms.
// ---- pieces shared by the blocked forms (k_gj_blk, k_gj_la) --------------------------------
// Pivot key of row r: the magnitude bits of |a| without their lowest 8 (pivots within 2^-15
// relative of each other tie), then 255 - r, so that the largest key is a row of (nearly) the
// largest |a| and, among those, the lowest row; a NaN has magnitude part 0, so any number
// beats it and a column without a number yields its lowest unused row.  Rows r < 128.
__device__ __forceinline__ unsigned piv_pack(float x, int r) {
    const unsigned k = (unsigned)(piv_key(x) + 1);   // 0 for NaN
    return ((k >> 8) << 8) | (unsigned)(255 - r);
}

// The in-place Gauss-Jordan steps of a panel of NB columns held by one warp (lane tx: rows
// tx + 32 i, x[i][c] for panel column c), one warp reduction per pivot: pivot rows are
// recorded in perm[k0 + s] and their steps in invk[p] = k0 + s; `used` marks this lane's rows
// already taken.
template <int B, int RS, int NB>
__device__ __forceinline__ void gj_panel_steps(float (&x)[RS][NB], unsigned& used, int nb, int k0, int tx, int* perm,
                                               int* invk) {
#pragma unroll
    for (int s = 0; s < NB; ++s) {
        if (s >= nb) break;   // uniform
        unsigned km = 0u;
#pragma unroll
        for (int i = 0; i < RS; ++i) {
            const int r = tx + 32 * i;
            const unsigned kk = (r < B && !((used >> i) & 1u)) ? piv_pack(x[i][s], r) : 0u;
            km = kk > km ? kk : km;
        }
        km = __reduce_max_sync(0xffffffffu, km);
        const int p = 255 - (int)(km & 255u);
        const int pl = p & 31, pi = p >> 5;
        float rk[NB];
#pragma unroll
        for (int ii = 0; ii < RS; ++ii)
            if (pi == ii) {   // warp-uniform branch
#pragma unroll
                for (int c = 0; c < NB; ++c) rk[c] = __shfl_sync(0xffffffffu, x[ii][c], pl);
            }
        const float inv = __frcp_rn(rk[s]);   // correctly rounded, as 1.0f / rk[s]
#pragma unroll
        for (int c = 0; c < NB; ++c) rk[c] = (c == s) ? inv : rk[c] * inv;
        float f[RS];
#pragma unroll
        for (int i = 0; i < RS; ++i) {
            f[i] = (tx + 32 * i == p) ? 0.0f : x[i][s];
            x[i][s] = 0.0f;
        }
#pragma unroll
        for (int i = 0; i < RS; ++i) {
#pragma unroll
            for (int c = 0; c + 1 < NB; c += 2) fma2f(-f[i], rk[c], rk[c + 1], x[i][c], x[i][c + 1]);
            if (NB % 2) x[i][NB - 1] = fmaf(-f[i], rk[NB - 1], x[i][NB - 1]);
        }
        if (tx == pl) {
            used |= 1u << pi;
#pragma unroll
            for (int ii = 0; ii < RS; ++ii)
                if (pi == ii) {
#pragma unroll
                    for (int c = 0; c < NB; ++c) x[ii][c] = rk[c];
                }
        }
        if (tx == 0) {
            perm[k0 + s] = p;
            invk[p] = k0 + s;
        }
    }
}

// The panel's pivot rows on this warp's non-panel slots j = SPW .. CS-1 into its buffer yw
// (the row of step k0 + s at yw + s YL, 16 bytes at a time), and the factor m[i] that clears
// this lane's pivot rows (they are rebuilt from F alone): 0 for a pivot row, else 1.  Every
// lane writes its own rows at once: invk[r] is the step at which row r was chosen (-1 while
// it has not been; rows >= B never are), so the panel's pivot rows are those with
// k0 <= invk[r] < k0 + nb.
template <int RS, int CS, int SPW, int YL>
__device__ __forceinline__ void gj_gather_pivot_rows(const float (&a)[RS][CS], const int* invk, int k0, int nb,
                                                     int tx, float* yw, float (&m)[RS]) {
#pragma unroll
    for (int i = 0; i < RS; ++i) {
        const int s = invk[tx + 32 * i] - k0;
        const bool piv = (unsigned)s < (unsigned)nb;
        m[i] = piv ? 0.0f : 1.0f;
        if (piv) {
#pragma unroll
            for (int j0 = 0; j0 < CS - SPW; j0 += 4) {
                float4 v;
                v.x = a[i][SPW + j0];
                v.y = (j0 + 1 < CS - SPW) ? a[i][SPW + j0 + 1] : 0.0f;
                v.z = (j0 + 2 < CS - SPW) ? a[i][SPW + j0 + 2] : 0.0f;
                v.w = (j0 + 3 < CS - SPW) ? a[i][SPW + j0 + 3] : 0.0f;
                *reinterpret_cast<float4*>(yw + s * YL + j0) = v;
            }
        }
    }
}

// a[i][j] *= m[i] on the non-panel slots j = SPW .. CS-1, two products per instruction.
template <int RS, int CS, int SPW>
__device__ __forceinline__ void gj_clear_pivot_rows(float (&a)[RS][CS], const float (&m)[RS]) {
#pragma unroll
    for (int i = 0; i < RS; ++i) {
#pragma unroll
        for (int j = SPW; j + 1 < CS; j += 2) {
            const float2 r = __fmul2_rn(make_float2(a[i][j], a[i][j + 1]), make_float2(m[i], m[i]));
            a[i][j] = r.x;
            a[i][j + 1] = r.y;
        }
        if ((CS - SPW) % 2) a[i][CS - 1] *= m[i];
    }
}

// One step of the rank-NB update on the column slots j and j + 1 of a thread,
// a[i][j] += f[i] y0 and a[i][j + 1] += f[i] y1, for the slots in [JLO, CS) only; both slots
// in range take one paired multiply-add per row (bitwise two fmaf).
template <int RS, int CS, int JLO>
__device__ __forceinline__ void gj_update_pair(float (&a)[RS][CS], const float (&f)[RS], int j, float y0, float y1) {
    const bool in0 = j >= JLO && j < CS, in1 = j + 1 >= JLO && j + 1 < CS;
    if (in0 && in1) {
#pragma unroll
        for (int i = 0; i < RS; ++i) fma2f(f[i], y0, y1, a[i][j], a[i][j + 1]);
    } else if (in0) {
#pragma unroll
        for (int i = 0; i < RS; ++i) a[i][j] = fmaf(f[i], y0, a[i][j]);
    } else if (in1) {
#pragma unroll
        for (int i = 0; i < RS; ++i) a[i][j + 1] = fmaf(f[i], y1, a[i][j + 1]);
    }
}

template <int B, int W>
struct GjBlk {
    static constexpr int NB = 8;                        // panel width
    static constexpr int SPW = NB / W;                  // panel columns per warp and panel
    static constexpr int RS = (B + 31) / 32;            // row slots per lane
    static constexpr int R32 = 32 * RS;
    static constexpr int NP = (B + NB - 1) / NB;        // panels
    static constexpr int CS = NP * SPW;                 // column slots per thread
    static constexpr int PLD = NB + 1;                  // row stride of the panel buffers
    static constexpr int YN = CS - SPW;                 // non-panel slots per thread
    static constexpr int YL = YN > 0 ? ((YN + 3) / 4) * 4 : 4;
    static constexpr int LD = (B % 2) ? B + 2 : B + 1;  // row stride of the staging tile
    static constexpr size_t TILE = (size_t)B * LD * sizeof(float);
    static constexpr size_t WORK = (size_t)(2 * R32 * PLD + W * NB * YL) * sizeof(float);
    static constexpr size_t SMEM = ((TILE > WORK ? TILE : WORK) + 15) / 16 * 16;
    static constexpr bool VALID = (NB % W == 0) && RS * CS <= 64 && B <= 128;   // piv_pack: rows < 128
};

template <int B, int W>
__global__ void __launch_bounds__(32 * W, 16 / W) k_gj_blk(int E, float* __restrict__ blk) {
    using G = GjBlk<B, W>;
    constexpr int NB = G::NB, SPW = G::SPW, RS = G::RS, R32 = G::R32, NP = G::NP, CS = G::CS;
    constexpr int PLD = G::PLD, YL = G::YL, LD = G::LD, T = 32 * W;
    extern __shared__ __align__(16) unsigned char smraw[];
    float* tile = reinterpret_cast<float*>(smraw);      // staging (load and store only)
    float* Pn = tile;                                   // panel columns [R32][PLD]
    float* Fs = tile + R32 * PLD;                       // factored panel F [R32][PLD]
    float* Yw = tile + 2 * R32 * PLD;                   // pivot rows, per warp [W][NB][YL]
    __shared__ int perm[B], invk[R32];
    const int e = blockIdx.x;
    const int tx = threadIdx.x & 31, w = threadIdx.x >> 5;
    float* g = blk + (size_t)e * B * B;
    for (int t = threadIdx.x; t < R32; t += T) invk[t] = -1;
    for (int t = threadIdx.x; t < B * B; t += T) tile[(t / B) * LD + (t % B)] = g[t];
    __syncthreads();
    float a[RS][CS];
#pragma unroll
    for (int i = 0; i < RS; ++i)
#pragma unroll
        for (int j = 0; j < CS; ++j) {
            const int r = tx + 32 * i, c = w + W * j;
            a[i][j] = (r < B && c < B) ? tile[r * LD + c] : 0.0f;
        }
    unsigned used = 0u;   // warp 0: bit i set once row tx + 32 i has been a pivot row
    float* yw = Yw + (size_t)w * NB * YL;
#pragma unroll 1
    for (int t = 0; t < NP; ++t) {
        const int k0 = t * NB;
        const int nb = (B - k0) < NB ? (B - k0) : NB;
        __syncthreads();   // the previous panel's F and the staging tile are no longer read
        // (A) the panel's columns k0 + w + W s (slots s < SPW) to the panel buffer
#pragma unroll
        for (int s = 0; s < SPW; ++s)
#pragma unroll
            for (int i = 0; i < RS; ++i) Pn[(tx + 32 * i) * PLD + w + W * s] = a[i][s];
        __syncthreads();
        // (B) warp 0 factors the panel
        if (w == 0) {
            float x[RS][NB];
#pragma unroll
            for (int i = 0; i < RS; ++i)
#pragma unroll
                for (int c = 0; c < NB; ++c) x[i][c] = Pn[(tx + 32 * i) * PLD + c];
            gj_panel_steps<B, RS, NB>(x, used, nb, k0, tx, perm, invk);
#pragma unroll
            for (int i = 0; i < RS; ++i)
#pragma unroll
                for (int c = 0; c < NB; ++c) Fs[(tx + 32 * i) * PLD + c] = x[i][c];
        }
        __syncthreads();
        // (C) pivot rows of this warp's non-panel columns into the warp's buffer; the pivot
        // rows' own entries are then cleared (they are rebuilt from F alone)
        __syncwarp();
        float mrow[RS];
        gj_gather_pivot_rows<RS, CS, SPW, YL>(a, invk, k0, nb, tx, yw, mrow);
        __syncwarp();
        gj_clear_pivot_rows<RS, CS, SPW>(a, mrow);
#pragma unroll
        for (int s = 0; s < NB; ++s) {
            if (s >= nb) break;   // uniform
            float f[RS];
#pragma unroll
            for (int i = 0; i < RS; ++i) f[i] = Fs[(tx + 32 * i) * PLD + s];
            const float* yr = yw + s * YL;
#pragma unroll
            for (int j0 = 0; j0 < CS - SPW; j0 += 4) {
                const float4 y4 = *reinterpret_cast<const float4*>(yr + j0);
                const float yv[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
                for (int q = 0; q < 4; q += 2) gj_update_pair<RS, CS, SPW>(a, f, SPW + j0 + q, yv[q], yv[q + 1]);
            }
        }
        // the panel's own columns become F
#pragma unroll
        for (int s = 0; s < SPW; ++s)
#pragma unroll
            for (int i = 0; i < RS; ++i) a[i][s] = Fs[(tx + 32 * i) * PLD + w + W * s];
        // rotate the column slots by SPW: the next panel's columns move to slots 0 .. SPW-1
#pragma unroll
        for (int i = 0; i < RS; ++i) {
            float t0[SPW];
#pragma unroll
            for (int s = 0; s < SPW; ++s) t0[s] = a[i][s];
#pragma unroll
            for (int j = 0; j < CS - SPW; ++j) a[i][j] = a[i][j + SPW];
#pragma unroll
            for (int s = 0; s < SPW; ++s) a[i][CS - SPW + s] = t0[s];
        }
    }
    // NP rotations by SPW = CS slots: every column is back in its own slot
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RS; ++i)
#pragma unroll
        for (int j = 0; j < CS; ++j) {
            const int r = tx + 32 * i, c = w + W * j;
            if (r < B && c < B) tile[perm[c] * LD + invk[r]] = a[i][j];
        }
    __syncthreads();
    for (int t = threadIdx.x; t < B * B; t += T) g[t] = tile[(t / B) * LD + (t % B)];
}

// Look-ahead form of k_gj_blk: warp 0 only factors panels and warps 1..W own the columns
// (column c: warp 1 + c mod W, slot c / W).  At panel t the update warps first bring panel
// t+1's columns up to date and hand them to warp 0, then update the remaining columns, so the
// factorisation of panel t+1 runs while the trailing update of panel t is still going on.
// Two named barriers carry the hand-offs (panel ready: the update warps arrive, warp 0 waits;
// factor ready: warp 0 arrives, the update warps wait); panel and factor buffers are double
// buffered.  Every entry receives the multiply-adds of k_gj_blk in the same order, and the
// panel steps are those of k_gj_blk: bitwise the same inverse.
template <int B, int W>
struct GjLa {
    static constexpr int NB = 8;
    static constexpr int SPW = NB / W;
    static constexpr int RS = (B + 31) / 32;
    static constexpr int R32 = 32 * RS;
    static constexpr int NP = (B + NB - 1) / NB;
    static constexpr int CS = NP * SPW;
    static constexpr int PLD = NB + 1;
    static constexpr int YN = CS - SPW;
    static constexpr int YL = YN > 0 ? ((YN + 3) / 4) * 4 : 4;
    static constexpr int LD = (B % 2) ? B + 2 : B + 1;
    static constexpr int THREADS = 32 * (W + 1);
    static constexpr size_t TILE = (size_t)B * LD * sizeof(float);
    static constexpr size_t WORK = (size_t)(4 * R32 * PLD + W * NB * YL) * sizeof(float);
    static constexpr size_t SMEM = ((TILE > WORK ? TILE : WORK) + 15) / 16 * 16;
    static constexpr bool VALID = (NB % W == 0) && RS * CS <= 64 && NP >= 2 && B <= 128;
};

__device__ __forceinline__ void named_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int count) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

template <int B, int W>
__global__ void __launch_bounds__(32 * (W + 1)) k_gj_la(int E, float* __restrict__ blk) {
    using G = GjLa<B, W>;
    constexpr int NB = G::NB, SPW = G::SPW, RS = G::RS, R32 = G::R32, NP = G::NP, CS = G::CS;
    constexpr int PLD = G::PLD, YL = G::YL, LD = G::LD, T = G::THREADS;
    constexpr int BAR_PANEL = 1, BAR_F = 2;
    extern __shared__ __align__(16) unsigned char smraw[];
    float* tile = reinterpret_cast<float*>(smraw);      // staging (load and store only)
    float* Pn = tile;                                   // 2 x [R32][PLD] panel columns
    float* Fs = tile + 2 * R32 * PLD;                   // 2 x [R32][PLD] factored panels
    float* Yw = tile + 4 * R32 * PLD;                   // [W][NB][YL] pivot rows per update warp
    __shared__ int perm[B], invk[R32];
    const int e = blockIdx.x;
    const int tx = threadIdx.x & 31, wq = threadIdx.x >> 5, w = wq - 1;
    float* g = blk + (size_t)e * B * B;
    for (int t = threadIdx.x; t < R32; t += T) invk[t] = -1;
    for (int t = threadIdx.x; t < B * B; t += T) tile[(t / B) * LD + (t % B)] = g[t];
    __syncthreads();
    float a[RS][CS];
    if (wq > 0) {
#pragma unroll
        for (int i = 0; i < RS; ++i)
#pragma unroll
            for (int j = 0; j < CS; ++j) {
                const int r = tx + 32 * i, c = w + W * j;
                a[i][j] = (r < B && c < B) ? tile[r * LD + c] : 0.0f;
            }
    }
    __syncthreads();   // the staging tile becomes the work buffers
    if (wq == 0) {
        // ---- factor warp -----------------------------------------------------------------
        unsigned used = 0u;
#pragma unroll 1
        for (int t = 0; t < NP; ++t) {
            const int k0 = t * NB;
            const int nb = (B - k0) < NB ? (B - k0) : NB;
            const float* pn = Pn + (t & 1) * R32 * PLD;
            float* fs = Fs + (t & 1) * R32 * PLD;
            named_sync(BAR_PANEL, T);
            float x[RS][NB];
#pragma unroll
            for (int i = 0; i < RS; ++i)
#pragma unroll
                for (int c = 0; c < NB; ++c) x[i][c] = pn[(tx + 32 * i) * PLD + c];
            gj_panel_steps<B, RS, NB>(x, used, nb, k0, tx, perm, invk);
#pragma unroll
            for (int i = 0; i < RS; ++i)
#pragma unroll
                for (int c = 0; c < NB; ++c) fs[(tx + 32 * i) * PLD + c] = x[i][c];
            __threadfence_block();
            named_arrive(BAR_F, T);
        }
    } else {
        // ---- update warps ----------------------------------------------------------------
        float* yw = Yw + (size_t)w * NB * YL;
#pragma unroll
        for (int s = 0; s < SPW; ++s)
#pragma unroll
            for (int i = 0; i < RS; ++i) Pn[(tx + 32 * i) * PLD + w + W * s] = a[i][s];
        __threadfence_block();
        named_arrive(BAR_PANEL, T);
#pragma unroll 1
        for (int t = 0; t < NP; ++t) {
            const int k0 = t * NB;
            const int nb = (B - k0) < NB ? (B - k0) : NB;
            const float* fs = Fs + (t & 1) * R32 * PLD;
            named_sync(BAR_F, T);
            // pivot rows of this warp's non-panel columns; their own entries are rebuilt from F.
            // Warp 0 may meanwhile be recording panel t+1's pivots in invk: a row it records
            // reads as -1 or as a step >= k0 + NB, outside this panel's range either way.
            __syncwarp();
            float mrow[RS];
            gj_gather_pivot_rows<RS, CS, SPW, YL>(a, invk, k0, nb, tx, yw, mrow);
            __syncwarp();
            gj_clear_pivot_rows<RS, CS, SPW>(a, mrow);
            // (1) slots SPW .. 2 SPW - 1 first: the next panel's columns, handed to warp 0 at once
            // (at the last panel they hold earlier columns, updated like the rest)
#pragma unroll
            for (int s = 0; s < NB; ++s) {
                if (s >= nb) break;   // uniform
                float f[RS];
#pragma unroll
                for (int i = 0; i < RS; ++i) f[i] = fs[(tx + 32 * i) * PLD + s];
                const float* yr = yw + s * YL;
#pragma unroll
                for (int q = 0; q < SPW; ++q) {
                    const float yv = yr[q];
#pragma unroll
                    for (int i = 0; i < RS; ++i) a[i][SPW + q] = fmaf(f[i], yv, a[i][SPW + q]);
                }
            }
            if (t + 1 < NP) {
                float* pn = Pn + ((t + 1) & 1) * R32 * PLD;
#pragma unroll
                for (int q = 0; q < SPW; ++q)
#pragma unroll
                    for (int i = 0; i < RS; ++i) pn[(tx + 32 * i) * PLD + w + W * q] = a[i][SPW + q];
                __threadfence_block();
                named_arrive(BAR_PANEL, T);
            }
            // (2) the remaining columns (slots 2 SPW .. CS - 1)
#pragma unroll
            for (int s = 0; s < NB; ++s) {
                if (s >= nb) break;   // uniform
                float f[RS];
#pragma unroll
                for (int i = 0; i < RS; ++i) f[i] = fs[(tx + 32 * i) * PLD + s];
                const float* yr = yw + s * YL;
#pragma unroll
                for (int j0 = 0; j0 < CS - SPW; j0 += 4) {
                    const float4 y4 = *reinterpret_cast<const float4*>(yr + j0);
                    const float yv[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
                    for (int q = 0; q < 4; q += 2)
                        gj_update_pair<RS, CS, 2 * SPW>(a, f, SPW + j0 + q, yv[q], yv[q + 1]);
                }
            }
            // (3) the panel's own columns become F
#pragma unroll
            for (int s = 0; s < SPW; ++s)
#pragma unroll
                for (int i = 0; i < RS; ++i) a[i][s] = fs[(tx + 32 * i) * PLD + w + W * s];
#pragma unroll
            for (int i = 0; i < RS; ++i) {
                float t0[SPW];
#pragma unroll
                for (int s = 0; s < SPW; ++s) t0[s] = a[i][s];
#pragma unroll
                for (int j = 0; j < CS - SPW; ++j) a[i][j] = a[i][j + SPW];
#pragma unroll
                for (int s = 0; s < SPW; ++s) a[i][CS - SPW + s] = t0[s];
            }
        }
    }
    __syncthreads();
    if (wq > 0) {
#pragma unroll
        for (int i = 0; i < RS; ++i)
#pragma unroll
            for (int j = 0; j < CS; ++j) {
                const int r = tx + 32 * i, c = w + W * j;
                if (r < B && c < B) tile[perm[c] * LD + invk[r]] = a[i][j];
            }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < B * B; t += T) g[t] = tile[(t / B) * LD + (t % B)];
}

// ---- variants of the FP32 Gauss-Jordan kernel and their tuning --------------------------------
// Two families.  Unblocked (variants 0..13): variant v < 4 unrolls the pivot loop kGjUnroll[v]
// times (0 = fully, only for B <= 100); 4..8 are the column-owner form with kGjWarps[v - 4]
// warps per element (valid while a thread's share of the block stays at most 128 values);
// 9..13 the rotating column-owner form with kGjWarps[v - 9] warps.  Blocked (14..21):
// k_gj_blk with kGjBlkWarps[v - 14] warps and the look-ahead k_gj_la with 1 + kGjBlkWarps[v - 18]
// warps (valid while a thread holds at most 64 values).
// Within a family the variants do the same arithmetic in the same order, so the tuner's choice
// never changes a result; the tuner times one family only (the blocked one where it is valid,
// unless emg_params.block_kernels asks for the unblocked forms).
constexpr int kGjUnroll[] = {1, 4, 16, 0};
constexpr int kGjWarps[] = {1, 2, 4, 8, 16};
constexpr int kGjBlkWarps[] = {1, 2, 4, 8};
constexpr int kGjBlkFirst = 14;
constexpr int kGjLaFirst = 18;   // look-ahead form, kGjBlkWarps[v - 18] update warps
constexpr int kGjVariants = 22;

template <int B, int W>
constexpr bool gj_blk_valid() {
    return GjBlk<B, W>::VALID;
}

template <int B>
static bool gj_variant_valid(int v) {
    if (v < 0 || v >= kGjVariants) return false;
    if (v < 4) return kGjUnroll[v] != 0 || B <= 100;
    if (v >= kGjLaFirst) {
        switch (kGjBlkWarps[v - kGjLaFirst]) {
            case 1: return GjLa<B, 1>::VALID;
            case 2: return GjLa<B, 2>::VALID;
            case 4: return GjLa<B, 4>::VALID;
            default: return GjLa<B, 8>::VALID;
        }
    }
    if (v >= kGjBlkFirst) {
        switch (kGjBlkWarps[v - kGjBlkFirst]) {
            case 1: return gj_blk_valid<B, 1>();
            case 2: return gj_blk_valid<B, 2>();
            case 4: return gj_blk_valid<B, 4>();
            default: return gj_blk_valid<B, 8>();
        }
    }
    const int W = kGjWarps[(v - 4) % 5];
    return ((B + 31) / 32) * ((B + W - 1) / W) <= 128;
}

static std::string gj_variant_name(int v) {
    if (v < 4) return "tile unroll " + std::to_string(kGjUnroll[v]);
    if (v >= kGjLaFirst) return "look-ahead 1+" + std::to_string(kGjBlkWarps[v - kGjLaFirst]) + " warps";
    if (v >= kGjBlkFirst) return "blocked " + std::to_string(kGjBlkWarps[v - kGjBlkFirst]) + " warps";
    return std::string(v < 9 ? "cols " : "rotating cols ") + std::to_string(kGjWarps[(v - 4) % 5]) + " warps";
}

template <int B, int W>
static cudaError_t gj_blk_go(unsigned E, float* blk, cudaStream_t st) {
    if constexpr (GjBlk<B, W>::VALID) {
        const size_t sm = GjBlk<B, W>::SMEM;
        cudaError_t e = cudaFuncSetAttribute(k_gj_blk<B, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_gj_blk<B, W><<<E, 32 * W, sm, st>>>((int)E, blk);
        return cudaGetLastError();
    } else {
        return cudaErrorInvalidValue;   // not reached: gj_dispatch checks the variant first
    }
}

template <int B, int W>
static cudaError_t gj_la_go(unsigned E, float* blk, cudaStream_t st) {
    if constexpr (GjLa<B, W>::VALID) {
        const size_t sm = GjLa<B, W>::SMEM;
        cudaError_t e = cudaFuncSetAttribute(k_gj_la<B, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_gj_la<B, W><<<E, GjLa<B, W>::THREADS, sm, st>>>((int)E, blk);
        return cudaGetLastError();
    } else {
        return cudaErrorInvalidValue;   // not reached: gj_dispatch checks the variant first
    }
}

template <int B>
static cudaError_t gj_launch(int v, unsigned E, float* blk, cudaStream_t st) {
    switch (v) {
        case 18: return gj_la_go<B, 1>(E, blk, st);
        case 19: return gj_la_go<B, 2>(E, blk, st);
        case 20: return gj_la_go<B, 4>(E, blk, st);
        case 21: return gj_la_go<B, 8>(E, blk, st);
        case 14: return gj_blk_go<B, 1>(E, blk, st);
        case 15: return gj_blk_go<B, 2>(E, blk, st);
        case 16: return gj_blk_go<B, 4>(E, blk, st);
        case 17: return gj_blk_go<B, 8>(E, blk, st);
        case 9: return gj_rot_go<B, 1>(E, blk, st);
        case 10: return gj_rot_go<B, 2>(E, blk, st);
        case 11: return gj_rot_go<B, 4>(E, blk, st);
        case 12: return gj_rot_go<B, 8>(E, blk, st);
        case 13: return gj_rot_go<B, 16>(E, blk, st);
        case 4: return gj_cols_go<B, 1>(E, blk, st);
        case 5: return gj_cols_go<B, 2>(E, blk, st);
        case 6: return gj_cols_go<B, 4>(E, blk, st);
        case 7: return gj_cols_go<B, 8>(E, blk, st);
        case 8: return gj_cols_go<B, 16>(E, blk, st);
        case 1: return gj_go<B, 4>(E, blk, st);
        case 2: return gj_go<B, 16>(E, blk, st);
        case 3: return gj_go<B, (B <= 100 ? B : 1)>(E, blk, st);
        default: return gj_go<B, 1>(E, blk, st);
    }
}

static cudaError_t gj_dispatch(int B, int v, unsigned E, float* blk, cudaStream_t st, bool* ok) {
    *ok = true;
    switch (B) {
#define EMG_GJ_CASE(BB) \
    case BB:            \
        return gj_variant_valid<BB>(v) ? gj_launch<BB>(v, E, blk, st) : gj_launch<BB>(0, E, blk, st);
        EMG_BSIZES(EMG_GJ_CASE)
#undef EMG_GJ_CASE
        default:
            *ok = false;
            return cudaSuccess;
    }
}

static bool gj_valid(int B, int v) {
    switch (B) {
#define EMG_GJ_CASE(BB) \
    case BB:            \
        return gj_variant_valid<BB>(v);
        EMG_BSIZES(EMG_GJ_CASE)
#undef EMG_GJ_CASE
        default:
            return false;
    }
}

// Deterministic, diagonally dominant stand-in blocks for timing the variants.
__global__ void k_fill_tuning_blocks(int64_t n, int B, float* __restrict__ blk) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * B * B) return;
    const int c = (int)(t % B), r = (int)((t / B) % B);
    const uint32_t h = (uint32_t)(t * 2654435761ull) ^ (uint32_t)(t >> 13);
    blk[t] = (r == c ? (float)B : 0.0f) + ((float)(h & 0xffffu) / 65536.0f - 0.5f);
}

namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, bool>, int> g_gj_best;   // (device, B, unblocked asked) -> variant
}  // namespace

// Times every valid variant on min(E, 2048) stand-in blocks per block size of the FP32 levels
// and keeps the fastest, once per (device, B) for the process.
emg_status tune_gj(emg_ctx* c) {
    if (!blocks_f32(c->prm.prec)) return EMG_OK;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (int p = 1; p <= c->p_max; ++p) {
        LevelDev& L = c->lv[p];
        const auto key = std::make_tuple(c->device, L.B, c->prm.block_kernels == 3);
        // the family: blocked where a blocked variant is valid (unless the unblocked forms are
        // asked for), else unblocked
        bool blocked = false;
        if (c->prm.block_kernels != 3)
            for (int v = kGjBlkFirst; v < kGjVariants; ++v) blocked = blocked || gj_valid(L.B, v);
        const int v_lo = blocked ? kGjBlkFirst : 0, v_hi = blocked ? kGjVariants : kGjBlkFirst;   // 14..21 / 0..13
        if (!c->prm.autotune) {
            L.gj_variant = 0;
            for (int v = v_lo; v < v_hi; ++v)
                if (gj_valid(L.B, v)) {
                    L.gj_variant = v;
                    break;
                }
            continue;
        }
        if (L.tc_gj) {
            c->tuning += "gj B=" + std::to_string(L.B) + ": blocked tensor-core form (not tuned); ";
            continue;
        }
        auto it = g_gj_best.find(key);
        if (it != g_gj_best.end()) {
            L.gj_variant = it->second;
            c->tuning += "gj B=" + std::to_string(L.B) + ": " + gj_variant_name(it->second) +
                         " (tuned earlier in this process); ";
            continue;
        }
        const int64_t n = std::min<int64_t>(c->E, 2048);
        float* scratch = nullptr;
        EMG_CUDA_TRY(c, cudaMallocAsync((void**)&scratch, (size_t)n * L.B * L.B * sizeof(float), c->stream));
        k_fill_tuning_blocks<<<(unsigned)((n * L.B * L.B + 255) / 256), 256, 0, c->stream>>>(n, L.B, scratch);
        cudaEvent_t e0, e1;
        EMG_CUDA_TRY(c, cudaEventCreate(&e0));
        EMG_CUDA_TRY(c, cudaEventCreate(&e1));
        int best = v_lo;
        float best_ms = 1e30f;
        std::string note = "gj B=" + std::to_string(L.B) + ":";
        for (int v = v_lo; v < v_hi; ++v) {
            if (!gj_valid(L.B, v)) continue;
            bool ok = true;
            float ms = 1e30f;
            for (int rep = 0; rep < 3 && ok; ++rep) {
                EMG_CUDA_TRY(c, cudaEventRecord(e0, c->stream));
                EMG_CUDA_TRY(c, gj_dispatch(L.B, v, (unsigned)n, scratch, c->stream, &ok));
                EMG_CUDA_TRY(c, cudaEventRecord(e1, c->stream));
                EMG_CUDA_TRY(c, cudaEventSynchronize(e1));
                float t = 0.0f;
                EMG_CUDA_TRY(c, cudaEventElapsedTime(&t, e0, e1));
                if (rep > 0) ms = std::min(ms, t);   // the first run warms up
            }
            char buf[64];
            std::snprintf(buf, sizeof(buf), " %.3f ms, ", ms);
            note += " " + gj_variant_name(v) + buf;
            if (ms < best_ms) {
                best_ms = ms;
                best = v;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        EMG_CUDA_TRY(c, cudaFreeAsync(scratch, c->stream));
        g_gj_best[key] = best;
        L.gj_variant = best;
        c->tuning += note + "-> " + gj_variant_name(best) + "; ";
    }
    return EMG_OK;
}

emg_status launch_lu32(emg_ctx* c, int p) {
    LevelDev& L = c->lv[p];
    if (L.tc_gj) {
        bool built = false;
        const emg_status st = launch_gj_tc(c, L.B, L.blk32, &built);
        if (built) return st;
    }
    bool ok = true;
    {
        ProfScope _ps(c, PC_LU);
        EMG_CUDA_TRY(c, gj_dispatch(L.B, L.gj_variant, (unsigned)c->E, L.blk32, c->stream, &ok));
    }
    if (!ok) {
        c->err = "unsupported block size";
        return EMG_ERR_ARG;
    }
    return EMG_OK;
}

}  // namespace emg
