// Batched element-block solves of the PRK smoother (Eq. prk_scalar):
//  * k_lu: LU factorisation with partial pivoting of every P_e = I/dtau_e - D_e, one CTA
//    per element with the block in shared memory; factors stored column-major so that the
//    substitutions read contiguous columns.
//  * k_stage: one warp per element: y = P_e^{-1} r_e (row swaps, unit-lower forward and
//    upper backward substitution), u^(k) = u^n + beta_k y.
// T is the block precision (double for the FP64 form, float for the FP32 block form);
// the residual r, u^n and u^(k) are always double.
#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>

#include "common.cuh"
#include "tc.cuh"

namespace emg {

// Pivot magnitude as an ordered integer key: the IEEE bits of |x| order like its value for
// every finite or infinite x; a NaN gets -1, so it never wins against a number.  Comparing
// keys as integers keeps the pivot search deterministic and independent of how the compiler
// treats float comparisons with NaN (where every thread of a warp computes the pivot on its
// own, a disagreement would break the permutation).
__device__ __forceinline__ int piv_key(float x) {
    const unsigned b = __float_as_uint(x) & 0x7fffffffu;
    return b <= 0x7f800000u ? (int)b : -1;
}
__device__ __forceinline__ long long piv_key(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
    return b <= 0x7ff0000000000000ull ? (long long)b : -1ll;
}

template <int B, class T>
struct LuCfg {
    static constexpr int LD = B + 1;                 // padded row stride in shared memory
    static constexpr size_t SMEM = (size_t)B * LD * sizeof(T);
};

template <int B, class T>
__global__ void __launch_bounds__(256) k_lu(int E, T* __restrict__ blk, int* __restrict__ piv) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T* a = reinterpret_cast<T*>(smraw);
    constexpr int LD = LuCfg<B, T>::LD;
    __shared__ int s_piv;
    const int e = blockIdx.x;
    const int tid = threadIdx.x, nth = blockDim.x;
    T* g = blk + (size_t)e * B * B;
    for (int t = tid; t < B * B; t += nth) a[(t / B) * LD + (t % B)] = g[t];
    __syncthreads();
    for (int k = 0; k < B; ++k) {
        if (tid < 32) {
            auto best = piv_key((T)0) - 1;   // every key is >= -1: a NaN row is taken only if no row is a number
            int bi = k;
            for (int r = k + tid; r < B; r += 32) {
                const auto v = piv_key(a[r * LD + k]);
                if (v > best) {
                    best = v;
                    bi = r;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const auto ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
            }
            if (tid == 0) {
                s_piv = bi;
                piv[(size_t)e * B + k] = bi;
            }
        }
        __syncthreads();
        const int pr = s_piv;
        if (pr != k)
            for (int cc = tid; cc < B; cc += nth) {
                const T t0 = a[k * LD + cc];
                a[k * LD + cc] = a[pr * LD + cc];
                a[pr * LD + cc] = t0;
            }
        __syncthreads();
        if (k + 1 + tid < B) {   // only the threads that scale a row pay for the division
            const T inv = (T)1 / a[k * LD + k];
            for (int r = k + 1 + tid; r < B; r += nth) a[r * LD + k] *= inv;
        }
        __syncthreads();
        // trailing update on a 32-wide column x 8-row thread grid (no index division)
        const int tx = tid & 31, ty = tid >> 5;
        for (int r = k + 1 + ty; r < B; r += 8) {
            const T l = a[r * LD + k];
            for (int cc = k + 1 + tx; cc < B; cc += 32) a[r * LD + cc] -= l * a[k * LD + cc];
        }
        __syncthreads();
    }
    // column-major out: g[col * B + row]
    for (int t = tid; t < B * B; t += nth) {
        const int cc = t / B, r = t % B;
        g[t] = a[r * LD + cc];
    }
}

// The same factorisation for blocks that do not fit in shared memory (B = 175 in float64):
// the block is factored in place in global memory (it stays in L2 while its CTA works on it),
// row-major during the elimination, then transposed in place to the column-major layout the
// substitutions read.  Pivot choice and tie rule as in k_lu.
template <int B, class T>
__global__ void __launch_bounds__(256) k_lu_gmem(int E, T* __restrict__ blk, int* __restrict__ piv) {
    __shared__ int s_piv;
    const int e = blockIdx.x;
    const int tid = threadIdx.x, nth = blockDim.x;
    T* a = blk + (size_t)e * B * B;
    for (int k = 0; k < B; ++k) {
        if (tid < 32) {
            auto best = piv_key((T)0) - 1;
            int bi = k;
            for (int r = k + tid; r < B; r += 32) {
                const auto v = piv_key(a[(size_t)r * B + k]);
                if (v > best) {
                    best = v;
                    bi = r;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const auto ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
            }
            if (tid == 0) {
                s_piv = bi;
                piv[(size_t)e * B + k] = bi;
            }
        }
        __syncthreads();
        const int pr = s_piv;
        if (pr != k)
            for (int cc = tid; cc < B; cc += nth) {
                const T t0 = a[(size_t)k * B + cc];
                a[(size_t)k * B + cc] = a[(size_t)pr * B + cc];
                a[(size_t)pr * B + cc] = t0;
            }
        __syncthreads();
        if (k + 1 + tid < B) {
            const T inv = (T)1 / a[(size_t)k * B + k];
            for (int r = k + 1 + tid; r < B; r += nth) a[(size_t)r * B + k] *= inv;
        }
        __syncthreads();
        const int tx = tid & 31, ty = tid >> 5;
        for (int r = k + 1 + ty; r < B; r += 8) {
            const T l = a[(size_t)r * B + k];
            for (int cc = k + 1 + tx; cc < B; cc += 32) a[(size_t)r * B + cc] -= l * a[(size_t)k * B + cc];
        }
        __syncthreads();
    }
    // row-major -> column-major, in place
    for (int t = tid; t < B * B; t += nth) {
        const int r = t / B, cc = t % B;
        if (r < cc) {
            const T t0 = a[(size_t)r * B + cc];
            a[(size_t)r * B + cc] = a[(size_t)cc * B + r];
            a[(size_t)cc * B + r] = t0;
        }
    }
}

template <int B, class T>
__global__ void __launch_bounds__(128) k_stage(int E, const T* __restrict__ lu, const int* __restrict__ piv,
                                               const double* __restrict__ r, const double* __restrict__ un,
                                               double beta, double* __restrict__ out) {
    __shared__ T ys[4][B];
    __shared__ T rd[4][B];   // reciprocals of U's diagonal
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int e = blockIdx.x * 4 + warp;
    if (e >= E) return;
    T* y = ys[warp];
    const T* M = lu + (size_t)e * B * B;
    // the B divisions of the back substitution, done once and in parallel across the lanes
    // (a division costs a warp-wide multi-instruction sequence on the FP64 pipe)
    for (int t = lane; t < B; t += 32) {
        y[t] = (T)r[(size_t)e * B + t];
        rd[warp][t] = (T)1 / M[(size_t)t * B + t];
    }
    __syncwarp();
    if (lane == 0) {
        const int* pv = piv + (size_t)e * B;
        for (int k = 0; k < B; ++k) {
            const int p = pv[k];
            if (p != k) {
                const T t0 = y[k];
                y[k] = y[p];
                y[p] = t0;
            }
        }
    }
    __syncwarp();
    for (int j = 0; j < B; ++j) {
        const T yj = y[j];
        const T* col = M + (size_t)j * B;
        for (int rr = j + 1 + lane; rr < B; rr += 32) y[rr] -= col[rr] * yj;
        __syncwarp();
    }
    for (int j = B - 1; j >= 0; --j) {
        const T* col = M + (size_t)j * B;
        const T xj = y[j] * rd[warp][j];
        __syncwarp();
        for (int rr = lane; rr < j; rr += 32) y[rr] -= col[rr] * xj;
        if (lane == 0) y[j] = xj;
        __syncwarp();
    }
    for (int t = lane; t < B; t += 32) out[(size_t)e * B + t] = un[(size_t)e * B + t] + beta * (double)y[t];
}

// Register-tiled Gauss-Jordan inversion with partial pivoting (FP32 block form).
// 256 threads = 32 (tx) x 8 (ty); thread (tx, ty) keeps rows ty + 8i and columns
// tx + 32j of the block in registers for the whole elimination.  Pivoting is implicit:
// rows never move; step k takes the unused row p with the largest |a_pk| (lowest index on
// ties) as its pivot row, and the permutation is applied when the inverse is stored.  Per
// step only the pivot column and the scaled pivot row pass through shared memory, double
// buffered, so a step needs two barriers.  Every warp finds the pivot itself from the
// shared column (the same data in the same order, hence the same row).  The inverse is
// written column-major through a transposing shared tile so that the stores coalesce.
template <int B>
struct GjTile {
    static constexpr int RS = (B + 7) / 8;    // row slots per thread
    static constexpr int CS = (B + 31) / 32;  // column slots per thread
    static constexpr int LD = (B % 2) ? B + 2 : B + 1;   // odd stride of the output tile
    static constexpr size_t SMEM = (size_t)B * LD * sizeof(float);
};

template <int B, int UNR>
__global__ void __launch_bounds__(256) k_gj_tile(int E, float* __restrict__ blk) {
    constexpr int RS = GjTile<B>::RS, CS = GjTile<B>::CS, LD = GjTile<B>::LD;
    constexpr int RP = 8 * RS, CP = 32 * CS;   // zero-padded extents: no bounds checks inside
    constexpr int MW = (B + 31) / 32;          // words of the used-row mask
    extern __shared__ __align__(16) unsigned char smraw[];
    float* tile = reinterpret_cast<float*>(smraw);
    __shared__ float colk[2][RP], rowk[2][CP];
    __shared__ int perm[B], invp[B];
    const int e = blockIdx.x;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    float* g = blk + (size_t)e * B * B;
    float a[RS][CS];
#pragma unroll
    for (int i = 0; i < RS; ++i)
#pragma unroll
        for (int j = 0; j < CS; ++j) {
            const int r = ty + 8 * i, c = tx + 32 * j;
            a[i][j] = (r < B && c < B) ? g[r * B + c] : 0.0f;
        }
    unsigned used[MW];
#pragma unroll
    for (int m = 0; m < MW; ++m) used[m] = 0u;
    // UNR steps per unrolled body: a variant parameter (the arithmetic is the same for every
    // UNR; full unrolling makes k compile-time but the code can outgrow the instruction cache)
#pragma unroll UNR
    for (int k = 0; k < B; ++k) {
        const int kb = k & 1, kj = k >> 5;
        float* ck = colk[kb];
        float* rk_s = rowk[kb];
        // (1) the pivot column, from the lane that owns column k (column k is then rebuilt
        //     by the update: in-place scheme)
        if (tx == (k & 31)) {
#pragma unroll
            for (int i = 0; i < RS; ++i) {
                float v = 0.0f;
#pragma unroll
                for (int j = 0; j < CS; ++j)
                    if (j == kj) {
                        v = a[i][j];
                        a[i][j] = 0.0f;
                    }
                ck[ty + 8 * i] = v;
            }
        }
        __syncthreads();
        // (2) every warp: the pivot row p among the unused rows
        int best = -1;
        int bi = B;
#pragma unroll
        for (int m = 0; m < MW; ++m) {
            const int r = tx + 32 * m;
            if (r < B && !((used[m] >> tx) & 1u)) {
                const int v = piv_key(ck[r]);
                if (v > best) {
                    best = v;
                    bi = r;
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if (bi >= B) {
            // no comparable candidate (a non-finite column): the lowest unused row, so that
            // every index stays inside the block; the non-finite values propagate
#pragma unroll
            for (int m = MW - 1; m >= 0; --m) {
                const int nv = B - 32 * m < 32 ? B - 32 * m : 32;
                const unsigned fr = ~used[m] & (nv == 32 ? 0xffffffffu : ((1u << nv) - 1u));
                if (fr) bi = 32 * m + __ffs((int)fr) - 1;
            }
        }
        const int p = bi;
#pragma unroll
        for (int m = 0; m < MW; ++m)
            if (m == (p >> 5)) used[m] |= 1u << (p & 31);
        const float inv = 1.0f / ck[p];
        // (3) the warp that holds row p publishes it scaled (column k of it becomes 1/a_pk)
        if (ty == (p & 7)) {
            const int pi = p >> 3;
#pragma unroll
            for (int j = 0; j < CS; ++j) {
                float v = 0.0f;
#pragma unroll
                for (int i = 0; i < RS; ++i)
                    if (i == pi) v = a[i][j];
                const int c = tx + 32 * j;
                rk_s[c] = (c == k ? 1.0f : v) * inv;
            }
        }
        if (threadIdx.x == 0) perm[k] = p;
        __syncthreads();
        // (4) eliminate column k from every other row (padded rows have a zero column entry)
        float rk[CS];
#pragma unroll
        for (int j = 0; j < CS; ++j) rk[j] = rk_s[tx + 32 * j];
#pragma unroll
        for (int i = 0; i < RS; ++i) {
            if (ty + 8 * i == p) {
#pragma unroll
                for (int j = 0; j < CS; ++j) a[i][j] = rk[j];
            } else {
                const float f = ck[ty + 8 * i];
#pragma unroll
                for (int j = 0; j < CS; ++j) a[i][j] -= f * rk[j];
            }
        }
    }
    // Row r of the working matrix holds row invp[r] of the inverse, and its column k holds
    // column perm[k] (perm[k] = pivot row of step k, invp its inverse permutation).
    __syncthreads();
    for (int k = threadIdx.x; k < B; k += 256) invp[perm[k]] = k;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RS; ++i)
#pragma unroll
        for (int j = 0; j < CS; ++j) {
            const int r = ty + 8 * i, c = tx + 32 * j;
            if (r < B && c < B) tile[perm[c] * LD + invp[r]] = a[i][j];
        }
    __syncthreads();
    for (int t = threadIdx.x; t < B * B; t += 256) g[t] = tile[(t / B) * LD + (t % B)];
}

// u^(k) = u^n + beta P_e^{-1} r_e with P_e^{-1} column-major: one warp per element, each
// lane owns rows lane, lane+32, ...; every column is a coalesced read.
template <int B, class T>
__global__ void __launch_bounds__(128) k_stage_gemv(int E, const T* __restrict__ inv, const double* __restrict__ r,
                                                    const double* __restrict__ un, double beta,
                                                    double* __restrict__ out) {
    constexpr int RPL = (B + 31) / 32;
    __shared__ T rs[4][B];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int e = blockIdx.x * 4 + warp;
    if (e >= E) return;
    for (int t = lane; t < B; t += 32) rs[warp][t] = (T)r[(size_t)e * B + t];
    __syncwarp();
    T acc[RPL];
#pragma unroll
    for (int t = 0; t < RPL; ++t) acc[t] = (T)0;
    const T* M = inv + (size_t)e * B * B;
#pragma unroll 4
    for (int j = 0; j < B; ++j) {
        const T rj = rs[warp][j];
        const T* col = M + (size_t)j * B;
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
            const int i = lane + 32 * t;
            if (i < B) acc[t] += __ldg(col + i) * rj;
        }
    }
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
        const int i = lane + 32 * t;
        if (i < B) out[(size_t)e * B + i] = un[(size_t)e * B + i] + beta * (double)acc[t];
    }
}

#define EMG_BSIZES(X) X(15) X(30) X(50) X(75) X(20) X(100) X(175)

template <class T>
static emg_status lu_dispatch(emg_ctx* c, int B, T* blk, int* piv) {
    const unsigned E = (unsigned)c->E;
    switch (B) {
#define EMG_LU_CASE(BB)                                                                                      \
    case BB: {                                                                                               \
        const size_t sm = LuCfg<BB, T>::SMEM;                                                                \
        if (sm > 227 * 1024) {                                                                               \
            ProfScope _ps(c, PC_LU);                                                                         \
            k_lu_gmem<BB, T><<<E, 256, 0, c->stream>>>((int)E, blk, piv);                                   \
            EMG_CHECK_LAUNCH(c);                                                                             \
            return EMG_OK;                                                                                   \
        }                                                                                                    \
        EMG_CUDA_TRY(c, cudaFuncSetAttribute(k_lu<BB, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)); \
        {                                                                                                    \
            ProfScope _ps(c, PC_LU);                                                                         \
            k_lu<BB, T><<<E, 256, sm, c->stream>>>((int)E, blk, piv);                                        \
        }                                                                                                    \
        EMG_CHECK_LAUNCH(c);                                                                                 \
        return EMG_OK;                                                                                       \
    }
        EMG_BSIZES(EMG_LU_CASE)
#undef EMG_LU_CASE
        default:
            c->err = "unsupported block size";
            return EMG_ERR_ARG;
    }
}

template <class T>
static emg_status stage_dispatch(emg_ctx* c, int B, const T* lu, const int* piv, const double* r, const double* un,
                                 double beta, double* out) {
    const unsigned E = (unsigned)c->E;
    switch (B) {
#define EMG_ST_CASE(BB)                                                                          \
    case BB: {                                                                                   \
        ProfScope _ps(c, PC_STAGE);                                                              \
        k_stage<BB, T><<<(E + 3) / 4, 128, 0, c->stream>>>((int)E, lu, piv, r, un, beta, out);   \
    }                                                                                            \
        EMG_CHECK_LAUNCH(c);                                                                     \
        return EMG_OK;
        EMG_BSIZES(EMG_ST_CASE)
#undef EMG_ST_CASE
        default:
            c->err = "unsupported block size";
            return EMG_ERR_ARG;
    }
}

emg_status launch_lu(emg_ctx* c, int p) { return lu_dispatch<double>(c, c->lv[p].B, c->lv[p].blk, c->lv[p].piv); }

// Column-owner form of the same Gauss-Jordan inversion: W warps per element; lane tx owns
// rows tx + 32i, warp w owns columns w + W j.  At step k only the warp owning column k
// searches for the pivot (its lanes hold the whole column) and publishes the column and
// the pivot row index; every warp then takes the pivot row's entries for its own columns
// from lane (p mod 32) by shuffles.  One barrier per step (the published column is double
// buffered).  Pivot choice, tie rule and every multiply-add are those of k_gj_tile, so
// both forms give bitwise the same inverse.
template <int B, int W>
struct GjCols {
    static constexpr int RS = (B + 31) / 32;   // row slots per thread
    static constexpr int CS = (B + W - 1) / W; // column slots per thread
    static constexpr int LD = (B % 2) ? B + 2 : B + 1;
    static constexpr size_t SMEM = (size_t)B * LD * sizeof(float);
};

template <int B, int W>
__global__ void __launch_bounds__(32 * W) k_gj_cols(int E, float* __restrict__ blk) {
    using G = GjCols<B, W>;
    constexpr int RS = G::RS, CS = G::CS, LD = G::LD, T = 32 * W;
    extern __shared__ __align__(16) unsigned char smraw[];
    float* tile = reinterpret_cast<float*>(smraw);
    __shared__ float colk[2][32 * RS];
    __shared__ int s_p[2];
    __shared__ int perm[B], invp[B];
    const int e = blockIdx.x;
    const int tx = threadIdx.x & 31, w = threadIdx.x >> 5;
    float* g = blk + (size_t)e * B * B;
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
    unsigned used = 0u;   // bit i: row tx + 32 i has been a pivot row
#pragma unroll 1
    for (int k = 0; k < B; ++k) {
        const int kb = k & 1, wk = k % W, jk = k / W;
        if (w == wk) {
            // (1) column k (then zeroed: in-place scheme), pivot among the unused rows
            float v[RS];
            int best = -1;
            int bi = B, lo = B;
#pragma unroll
            for (int i = 0; i < RS; ++i) {
                float x = 0.0f;
#pragma unroll
                for (int j = 0; j < CS; ++j)
                    if (j == jk) {
                        x = a[i][j];
                        a[i][j] = 0.0f;
                    }
                v[i] = x;
                const int r = tx + 32 * i;
                if (r < B && !((used >> i) & 1u)) {
                    const int m = piv_key(x);
                    if (m > best) {
                        best = m;
                        bi = r;
                    }
                    if (r < lo) lo = r;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const int ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                const int ol = __shfl_xor_sync(0xffffffffu, lo, o);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
                lo = ol < lo ? ol : lo;
            }
            // no comparable candidate (a non-finite column): the lowest unused row
            const int p = bi < B ? bi : lo;
#pragma unroll
            for (int i = 0; i < RS; ++i) colk[kb][tx + 32 * i] = v[i];
            if (tx == 0) {
                s_p[kb] = p;
                perm[k] = p;
            }
        }
        __syncthreads();
        // (2) every warp: the scaled pivot row on its own columns, then the elimination
        const int p = s_p[kb];
        const float inv = 1.0f / colk[kb][p];
        const int pl = p & 31, pi = p >> 5;
        if (tx == pl) used |= 1u << pi;
        float f[RS];
#pragma unroll
        for (int i = 0; i < RS; ++i) f[i] = colk[kb][tx + 32 * i];
#pragma unroll
        for (int j = 0; j < CS; ++j) {
            float x = 0.0f;
#pragma unroll
            for (int i = 0; i < RS; ++i)
                if (i == pi) x = a[i][j];
            x = __shfl_sync(0xffffffffu, x, pl);
            const float rk = (w + W * j == k ? 1.0f : x) * inv;
#pragma unroll
            for (int i = 0; i < RS; ++i) {
                if (tx + 32 * i == p)
                    a[i][j] = rk;
                else
                    a[i][j] -= f[i] * rk;
            }
        }
    }
    // Row r of the working matrix holds row invp[r] of the inverse, and its column k holds
    // column perm[k]; written column-major through the shared tile.
    __syncthreads();
    for (int t = threadIdx.x; t < B; t += T) invp[perm[t]] = t;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RS; ++i)
#pragma unroll
        for (int j = 0; j < CS; ++j) {
            const int r = tx + 32 * i, c = w + W * j;
            if (r < B && c < B) tile[perm[c] * LD + invp[r]] = a[i][j];
        }
    __syncthreads();
    for (int t = threadIdx.x; t < B * B; t += T) g[t] = tile[(t / B) * LD + (t % B)];
}

// Rotating column-owner form: the layout of k_gj_cols, but after every W pivot steps each
// thread rotates its column slots by one, so that the pivot column of a step is always in
// register slot 0 of its owner warp (no runtime-indexed register access).  The pivot row
// slot (p / 32) is warp-uniform: it is taken by branching, not by select chains.  The
// multiply-adds and the pivot choice are those of k_gj_tile (bitwise the same inverse).
template <int B, int W>
__global__ void __launch_bounds__(32 * W) k_gj_rot(int E, float* __restrict__ blk) {
    using G = GjCols<B, W>;
    constexpr int RS = G::RS, CS = G::CS, LD = G::LD, T = 32 * W;
    extern __shared__ __align__(16) unsigned char smraw[];
    float* tile = reinterpret_cast<float*>(smraw);
    __shared__ float colk[2][32 * RS];
    __shared__ int s_p[2];
    __shared__ int perm[B], invp[B];
    const int e = blockIdx.x;
    const int tx = threadIdx.x & 31, w = threadIdx.x >> 5;
    float* g = blk + (size_t)e * B * B;
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
    unsigned used = 0u;
#pragma unroll 1
    for (int kb = 0; kb < CS; ++kb) {
#pragma unroll 1
        for (int wk = 0; wk < W; ++wk) {
            const int k = kb * W + wk;
            if (k >= B) break;   // uniform
            const int buf = k & 1;
            if (w == wk) {
                // (1) column k is slot 0 of this warp; zero it (in-place scheme) and pivot
                float v[RS];
                int best = -1;
                int bi = B, lo = B;
#pragma unroll
                for (int i = 0; i < RS; ++i) {
                    v[i] = a[i][0];
                    a[i][0] = 0.0f;
                    const int r = tx + 32 * i;
                    if (r < B && !((used >> i) & 1u)) {
                        const int m = piv_key(v[i]);
                        if (m > best) {
                            best = m;
                            bi = r;
                        }
                        if (r < lo) lo = r;
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const int ob = __shfl_xor_sync(0xffffffffu, best, o);
                    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                    const int ol = __shfl_xor_sync(0xffffffffu, lo, o);
                    if (ob > best || (ob == best && oi < bi)) {
                        best = ob;
                        bi = oi;
                    }
                    lo = ol < lo ? ol : lo;
                }
                const int p = bi < B ? bi : lo;   // lowest unused row if the column is not finite
#pragma unroll
                for (int i = 0; i < RS; ++i) colk[buf][tx + 32 * i] = v[i];
                if (tx == 0) {
                    s_p[buf] = p;
                    perm[k] = p;
                }
            }
            __syncthreads();
            // (2) the scaled pivot row on this warp's columns, by shuffles from lane p mod 32
            const int p = s_p[buf];
            const float inv = 1.0f / colk[buf][p];
            const int pl = p & 31, pi = p >> 5;
            if (tx == pl) used |= 1u << pi;
            float rk[CS];
#pragma unroll
            for (int c = 0; c < RS; ++c)
                if (pi == c) {   // warp-uniform branch
#pragma unroll
                    for (int j = 0; j < CS; ++j) rk[j] = __shfl_sync(0xffffffffu, a[c][j], pl) * inv;
                }
            if (w == wk) rk[0] = inv;   // column k: 1 / a_pk
            // (3) eliminate column k from every other row; row p becomes the scaled row
            float f[RS];
#pragma unroll
            for (int i = 0; i < RS; ++i) f[i] = (tx + 32 * i == p) ? 0.0f : colk[buf][tx + 32 * i];
#pragma unroll
            for (int i = 0; i < RS; ++i)
#pragma unroll
                for (int j = 0; j < CS; ++j) a[i][j] -= f[i] * rk[j];
            if (tx == pl) {
#pragma unroll
                for (int c = 0; c < RS; ++c)
                    if (pi == c) {
#pragma unroll
                        for (int j = 0; j < CS; ++j) a[c][j] = rk[j];
                    }
            }
        }
        // rotate the column slots: the next group's pivot columns move to slot 0
#pragma unroll
        for (int i = 0; i < RS; ++i) {
            const float t0 = a[i][0];
#pragma unroll
            for (int j = 0; j < CS - 1; ++j) a[i][j] = a[i][j + 1];
            a[i][CS - 1] = t0;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < B; t += T) invp[perm[t]] = t;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RS; ++i)
#pragma unroll
        for (int j = 0; j < CS; ++j) {
            const int r = tx + 32 * i, c = w + W * j;
            if (r < B && c < B) tile[perm[c] * LD + invp[r]] = a[i][j];
        }
    __syncthreads();
    for (int t = threadIdx.x; t < B * B; t += T) g[t] = tile[(t / B) * LD + (t % B)];
}

// ---- blocked Gauss-Jordan inversion with tensor-core trailing updates (tcgen05) ---------------
// The in-place Gauss-Jordan steps of the kernels above, grouped in panels of KB = 16 pivot
// columns.  Step k with pivot row p acts on every column c != k as A[:, c] <- M_k A[:, c],
// M_k = I + x_k e_p^T, so the KB steps of a panel act on the columns outside it as
// T = I + X S_P^T (S_P selects the panel's pivot rows); X[:, j] is the panel's column j after
// all KB steps minus e_{p_j} (the in-place rule leaves M_j e_{p_j} in column j at step j).
// The matrix lives in TMEM (row r in lane r mod 128 of row tile r / 128).  Per panel: every
// warp copies its rows' panel columns to shared memory; warp 0 alone factors the panel in
// registers (lane l holds rows l, l + 32, ...: the pivot search and the pivot row's broadcast
// are warp shuffles, so the steps need no block barrier); then every other column takes the
// rank-KB update A += X A[P, :] as one tcgen05.mma per row tile and 32-byte K step (3xTF32:
// x = hi + lo, X_hi R_hi + X_hi R_lo + X_lo R_hi, float32 accumulation).  Pivot choice and tie
// rule are those of the kernels above (largest |a_rk| among the unused rows, lowest row on
// ties, the lowest unused row for a non-finite column); the inverse is written column-major
// with the same permutation.
template <int B>
struct GjTc {
    static constexpr int RT = (B + 127) / 128;           // 128-row tiles
    static constexpr int RI = (B + 31) / 32;             // rows per lane of the factoring warp
    static constexpr int NC = ((B + 15) / 16) * 16;      // columns held per row tile
    static constexpr int KB = 16;
    static constexpr int NPANEL = (B + KB - 1) / KB;
    static constexpr int COLS = RT * NC;
    static constexpr uint32_t TMEM_COLS = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128 : COLS <= 256 ? 256 : 512;
    static constexpr int T = 128;
    static constexpr uint32_t X_LBO = RT * 2048, R_LBO = (NC / 8) * 128, SBO = 128;
    static constexpr int X_BYTES = RT * 128 * KB * 4;     // one of the hi / lo copies
    static constexpr int R_BYTES = NC * KB * 4;
    static constexpr int PANEL = RT * 128 * KB;            // floats of the shared panel copy
    static constexpr int OPS = 2 * X_BYTES + 2 * R_BYTES + PANEL * 4;
    static constexpr int STAGE = B * B * 4;
    static constexpr int SMEM = OPS > STAGE ? OPS : STAGE;
    static_assert(COLS <= 512, "the block does not fit in the SM's tensor memory");
    static_assert(RI * 32 <= RT * 128, "the factoring warp's rows lie in the panel copy");
};

template <int B>
__global__ void __launch_bounds__(128) k_gj_tc(int E, float* __restrict__ blk, int* __restrict__ timeout_flag) {
    using G = GjTc<B>;
    constexpr int RT = G::RT, RI = G::RI, NC = G::NC, KB = G::KB, T = G::T;
    extern __shared__ __align__(1024) unsigned char gsm[];
    float* stage = reinterpret_cast<float*>(gsm);           // the block at the start and the end
    unsigned char* Xh = gsm;                                // operands during the panels
    unsigned char* Xl = Xh + G::X_BYTES;
    unsigned char* Rh = Xl + G::X_BYTES;
    unsigned char* Rl = Rh + G::R_BYTES;
    float* panel = reinterpret_cast<float*>(Rl + G::R_BYTES);   // [RT * 128][KB]
    __shared__ int pjs[RT * 128];    // pivot step of each row within the current panel, or -1
    __shared__ int perm[B], invp[B];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tbase_s;
    const int e = blockIdx.x;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float* g = blk + (size_t)e * B * B;
    const long long budget = 2000000000LL;   // about a second of SM clock
    if (tid == 0) {
        tc::mbar_init(&mbar, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(&tbase_s, G::TMEM_COLS);
        tc::tmem_relinquish();
    }
    for (int t = tid; t < B * B; t += T) stage[t] = g[t];   // row-major block, coalesced
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = tbase_s;
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
#pragma unroll
    for (int rt = 0; rt < RT; ++rt) {
        const int r = tid + 128 * rt;
#pragma unroll 1
        for (int c0 = 0; c0 < NC; c0 += 16) {
            float v[16];
#pragma unroll
            for (int cc = 0; cc < 16; ++cc) {
                const int c = c0 + cc;
                v[cc] = (r < B && c < B) ? stage[r * B + c] : 0.f;
            }
            tc::st16(tbase + lane_base + (uint32_t)(rt * NC + c0), v);
        }
    }
    unsigned used = 0u;   // factoring warp: bit i set once row lane + 32 i has been a pivot row
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t idesc = tc::idesc(tc::AB_TF32, 128, NC);
    bool failed = false;
    uint32_t phase = 0;
#pragma unroll 1
    for (int pn = 0; pn < G::NPANEL; ++pn) {
        const int k0 = pn * KB;
        const int kw = (B - k0) < KB ? (B - k0) : KB;
        // (1) every warp: its rows' panel columns into the shared copy
#pragma unroll
        for (int rt = 0; rt < RT; ++rt) {
            float v[16];
            tc::ld16(tbase + lane_base + (uint32_t)(rt * NC + k0), v);
            const int r = tid + 128 * rt;
            float4* dst = reinterpret_cast<float4*>(panel + r * KB);
#pragma unroll
            for (int q = 0; q < 4; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            pjs[r] = -1;
        }
        __syncthreads();
        // (2) warp 0 factors the panel
        if (warp == 0) {
            float pr[RI][16];
#pragma unroll
            for (int i = 0; i < RI; ++i) {
                const float4* src = reinterpret_cast<const float4*>(panel + (lane + 32 * i) * KB);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 x = src[q];
                    pr[i][4 * q] = x.x, pr[i][4 * q + 1] = x.y, pr[i][4 * q + 2] = x.z, pr[i][4 * q + 3] = x.w;
                }
            }
#pragma unroll
            for (int j = 0; j < KB; ++j) {
                if (j >= kw) break;
                int best = -1;
                int bi = B, lo = B;
#pragma unroll
                for (int i = 0; i < RI; ++i) {
                    const int r = lane + 32 * i;
                    if (r < B && !((used >> i) & 1u)) {
                        const int m = piv_key(pr[i][j]);
                        if (m > best) {
                            best = m;
                            bi = r;
                        }
                        lo = r < lo ? r : lo;
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const int ob = __shfl_xor_sync(0xffffffffu, best, o);
                    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                    const int ol = __shfl_xor_sync(0xffffffffu, lo, o);
                    if (ob > best || (ob == best && oi < bi)) {
                        best = ob;
                        bi = oi;
                    }
                    lo = ol < lo ? ol : lo;
                }
                // lowest unused row if the column is not finite; lane 0's choice for the whole warp
                const int p = __shfl_sync(0xffffffffu, bi < B ? bi : lo, 0);
                const int pl = p & 31, pi = p >> 5;
                float prow[16];
#pragma unroll
                for (int i = 0; i < RI; ++i)
                    if (i == pi) {   // warp-uniform
#pragma unroll
                        for (int c = 0; c < 16; ++c) prow[c] = __shfl_sync(0xffffffffu, pr[i][c], pl);
                    }
                const float inv = 1.f / prow[j];
                float rk[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) rk[c] = (c == j ? 1.f : prow[c]) * inv;
#pragma unroll
                for (int i = 0; i < RI; ++i) {
                    const int r = lane + 32 * i;
                    if (r == p) {
#pragma unroll
                        for (int c = 0; c < 16; ++c) pr[i][c] = rk[c];
                        used |= 1u << i;
                        pjs[r] = j;
                    } else {
                        const float f = pr[i][j];
                        pr[i][j] = 0.f;
#pragma unroll
                        for (int c = 0; c < 16; ++c) pr[i][c] -= f * rk[c];
                    }
                }
                if (lane == 0) perm[k0 + j] = p;
            }
#pragma unroll
            for (int i = 0; i < RI; ++i) {
                float4* dst = reinterpret_cast<float4*>(panel + (lane + 32 * i) * KB);
#pragma unroll
                for (int q = 0; q < 4; ++q) dst[q] = make_float4(pr[i][4 * q], pr[i][4 * q + 1], pr[i][4 * q + 2], pr[i][4 * q + 3]);
            }
        }
        __syncthreads();
        // (3) every thread: its rows' panel columns after the steps, and X = those - e_{p_j}
        float pv[RT][16];
        int pj[RT];
#pragma unroll
        for (int rt = 0; rt < RT; ++rt) {
            const int r = tid + 128 * rt;
            const float4* src = reinterpret_cast<const float4*>(panel + r * KB);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 x = src[q];
                pv[rt][4 * q] = x.x, pv[rt][4 * q + 1] = x.y, pv[rt][4 * q + 2] = x.z, pv[rt][4 * q + 3] = x.w;
            }
            pj[rt] = pjs[r];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float x[4];
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    const int j = 4 * q + cc;
                    x[cc] = j < kw ? pv[rt][j] - (pj[rt] == j ? 1.f : 0.f) : 0.f;
                }
                float4 hi, lo;
                hi.x = tc::tf32_round(x[0]), lo.x = tc::tf32_round(x[0] - hi.x);
                hi.y = tc::tf32_round(x[1]), lo.y = tc::tf32_round(x[1] - hi.y);
                hi.z = tc::tf32_round(x[2]), lo.z = tc::tf32_round(x[2] - hi.z);
                hi.w = tc::tf32_round(x[3]), lo.w = tc::tf32_round(x[3] - hi.w);
                const size_t off = (size_t)q * G::X_LBO + (size_t)(r >> 3) * G::SBO + (size_t)(r & 7) * 16;
                *reinterpret_cast<float4*>(Xh + off) = hi;
                *reinterpret_cast<float4*>(Xl + off) = lo;
            }
        }
        // (4) R = the pivot rows before the panel, zero on the panel's columns: the B operand
        for (int t = tid; t < 2 * G::R_BYTES / 16; t += T) reinterpret_cast<float4*>(Rh)[t] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
#pragma unroll
        for (int rt = 0; rt < RT; ++rt) {
#pragma unroll 1
            for (int c0 = 0; c0 < NC; c0 += 16) {
                float v[16];
                tc::ld16(tbase + lane_base + (uint32_t)(rt * NC + c0), v);
                const int jj = pj[rt];
                if (jj >= 0 && c0 != k0) {
#pragma unroll
                    for (int cc = 0; cc < 16; ++cc) {
                        const int c = c0 + cc;
                        const float hi = tc::tf32_round(v[cc]), lo = tc::tf32_round(v[cc] - hi);
                        const size_t off = (size_t)(jj >> 2) * G::R_LBO + (size_t)(c >> 3) * G::SBO + (size_t)(c & 7) * 16 +
                                           (size_t)(jj & 3) * 4;
                        *reinterpret_cast<float*>(Rh + off) = hi;
                        *reinterpret_cast<float*>(Rl + off) = lo;
                    }
                }
            }
        }
        tc::fence_proxy_async();
        tc::fence_before();
        __syncthreads();
        // (5) the rank-KB update of every row tile
        if (tid == 0) {
            tc::fence_after();
            const uint32_t xh = tc::smem_u32(Xh), xl = tc::smem_u32(Xl), rh = tc::smem_u32(Rh), rl = tc::smem_u32(Rl);
#pragma unroll
            for (int rt = 0; rt < RT; ++rt)
#pragma unroll
                for (int s2 = 0; s2 < KB / 8; ++s2) {
                    const uint32_t ka = (uint32_t)(2 * s2) * G::X_LBO + (uint32_t)rt * 16u * G::SBO;
                    const uint32_t kr = (uint32_t)(2 * s2) * G::R_LBO;
                    const uint64_t dxh = tc::sdesc(xh + ka, G::X_LBO, G::SBO);
                    const uint64_t drh = tc::sdesc(rh + kr, G::R_LBO, G::SBO);
                    const uint32_t d = tbase + (uint32_t)(rt * NC);
                    tc::mma_tf32(d, dxh, drh, idesc, 1u);
                    tc::mma_tf32(d, dxh, tc::sdesc(rl + kr, G::R_LBO, G::SBO), idesc, 1u);
                    tc::mma_tf32(d, tc::sdesc(xl + ka, G::X_LBO, G::SBO), drh, idesc, 1u);
                }
            tc::commit(&mbar);
        }
        if (!tc::mbar_wait(&mbar, phase, budget)) failed = true;
        phase ^= 1u;
        tc::fence_after();
        // (6) the panel's columns take their values after the steps (the MMA added zero there)
#pragma unroll
        for (int rt = 0; rt < RT; ++rt) tc::st16(tbase + lane_base + (uint32_t)(rt * NC + k0), pv[rt]);
        tc::fence_before();
        failed = __syncthreads_or(failed) != 0;   // the same decision in every thread
        if (failed) break;
        tc::fence_after();
    }
    if (failed) {
        if (tid == 0) atomicExch(timeout_flag, 1);
        tc::fence_before();
        __syncthreads();
        if (warp == 0) tc::tmem_dealloc(tbase, G::TMEM_COLS);
        return;
    }
    // row r of the working matrix holds row invp[r] of the inverse and its column c holds
    // column perm[c]: written column-major through the shared tile
    for (int t = tid; t < B; t += T) invp[perm[t]] = t;
    __syncthreads();
#pragma unroll
    for (int rt = 0; rt < RT; ++rt) {
        const int r = tid + 128 * rt;
#pragma unroll 1
        for (int c0 = 0; c0 < NC; c0 += 16) {
            float v[16];
            tc::ld16(tbase + lane_base + (uint32_t)(rt * NC + c0), v);
            if (r < B) {
#pragma unroll
                for (int cc = 0; cc < 16; ++cc) {
                    const int c = c0 + cc;
                    if (c < B) stage[perm[c] * B + invp[r]] = v[cc];
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, G::TMEM_COLS);
    for (int t = tid; t < B * B; t += T) g[t] = stage[t];
}

// ---- variants of the FP32 Gauss-Jordan kernel and their tuning --------------------------------
// Variant v unrolls the pivot loop kGjUnroll[v] times (0 = fully, only for B <= 100).  The
// variants do the same arithmetic in the same order, so the choice never changes a result.
// Variants 4..8 are the column-owner form with kGjWarps[v - 4] warps per element (valid
// while a thread's share of the block stays at most 128 values).
// Variants 9..13 the rotating column-owner form with kGjWarps[v - 9] warps.
constexpr int kGjUnroll[] = {1, 4, 16, 0};
constexpr int kGjWarps[] = {1, 2, 4, 8, 16};
constexpr int kGjVariants = 14;

template <int B>
static bool gj_variant_valid(int v) {
    if (v < 0 || v >= kGjVariants) return false;
    if (v < 4) return kGjUnroll[v] != 0 || B <= 100;
    const int W = kGjWarps[(v - 4) % 5];
    return ((B + 31) / 32) * ((B + W - 1) / W) <= 128;
}

static std::string gj_variant_name(int v) {
    if (v < 4) return "tile unroll " + std::to_string(kGjUnroll[v]);
    return std::string(v < 9 ? "cols " : "rotating cols ") + std::to_string(kGjWarps[(v - 4) % 5]) + " warps";
}

template <int B, int U>
static cudaError_t gj_go(unsigned E, float* blk, cudaStream_t st) {
    const size_t sm = GjTile<B>::SMEM;
    cudaError_t e = cudaFuncSetAttribute(k_gj_tile<B, U>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_gj_tile<B, U><<<E, 256, sm, st>>>((int)E, blk);
    return cudaGetLastError();
}

template <int B, int W>
static cudaError_t gj_cols_go(unsigned E, float* blk, cudaStream_t st) {
    const size_t sm = GjCols<B, W>::SMEM;
    cudaError_t e = cudaFuncSetAttribute(k_gj_cols<B, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_gj_cols<B, W><<<E, 32 * W, sm, st>>>((int)E, blk);
    return cudaGetLastError();
}

template <int B, int W>
static cudaError_t gj_rot_go(unsigned E, float* blk, cudaStream_t st) {
    const size_t sm = GjCols<B, W>::SMEM;
    cudaError_t e = cudaFuncSetAttribute(k_gj_rot<B, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_gj_rot<B, W><<<E, 32 * W, sm, st>>>((int)E, blk);
    return cudaGetLastError();
}

template <int B>
static cudaError_t gj_launch(int v, unsigned E, float* blk, cudaStream_t st) {
    switch (v) {
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
std::map<std::pair<int, int>, int> g_gj_best;   // (device, B) -> variant
}  // namespace

// Times every valid variant on min(E, 2048) stand-in blocks per block size of the FP32 levels
// and keeps the fastest, once per (device, B) for the process.
emg_status tune_gj(emg_ctx* c) {
    if (!blocks_f32(c->prm.prec)) return EMG_OK;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (int p = 1; p <= c->p_max; ++p) {
        LevelDev& L = c->lv[p];
        const auto key = std::make_pair(c->device, L.B);
        if (!c->prm.autotune) {
            L.gj_variant = 0;
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
        int best = 0;
        float best_ms = 1e30f;
        std::string note = "gj B=" + std::to_string(L.B) + ":";
        for (int v = 0; v < kGjVariants; ++v) {
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

// FP32 block form: explicit inverse (Gauss-Jordan), applied by k_stage_gemv.
template <int B>
static emg_status gj_tc_go(emg_ctx* c, float* blk) {
    using G = GjTc<B>;
    EMG_CUDA_TRY(c, cudaFuncSetAttribute(k_gj_tc<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM));
    {
        ProfScope _ps(c, PC_LU);
        k_gj_tc<B><<<(unsigned)c->E, G::T, G::SMEM, c->stream>>>((int)c->E, blk, &c->sc->timeout);
    }
    EMG_CHECK_LAUNCH(c);
    return EMG_OK;
}

emg_status launch_lu32(emg_ctx* c, int p) {
    LevelDev& L = c->lv[p];
    if (L.tc_gj) switch (L.B) {
            case 75: return gj_tc_go<75>(c, L.blk32);
            case 100: return gj_tc_go<100>(c, L.blk32);
            case 175: return gj_tc_go<175>(c, L.blk32);
            default: break;
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

emg_status launch_stage(emg_ctx* c, int p, const double* r, const double* un, double beta, double* out) {
    LevelDev& L = c->lv[p];
    return stage_dispatch<double>(c, L.B, L.blk, L.piv, r, un, beta, out);
}

emg_status launch_stage32(emg_ctx* c, int p, const double* r, const double* un, double beta, double* out) {
    LevelDev& L = c->lv[p];
    const unsigned E = (unsigned)c->E;
    switch (L.B) {
#define EMG_GV_CASE(BB)                                                                                  \
    case BB: {                                                                                           \
        ProfScope _ps(c, PC_STAGE);                                                                      \
        k_stage_gemv<BB, float><<<(E + 3) / 4, 128, 0, c->stream>>>((int)E, L.blk32, r, un, beta, out);  \
    }                                                                                                    \
        EMG_CHECK_LAUNCH(c);                                                                             \
        return EMG_OK;
        EMG_BSIZES(EMG_GV_CASE)
#undef EMG_GV_CASE
        default:
            c->err = "unsupported block size";
            return EMG_ERR_ARG;
    }
}

}  // namespace emg
