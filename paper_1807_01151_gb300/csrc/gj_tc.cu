// Explicit inverses P_e^{-1} of the float32 block forms with the trailing updates of the
// blocked Gauss-Jordan elimination on the fifth-generation tensor cores (tcgen05).
#include "blocks.cuh"
#include "common.cuh"
#include "tc.cuh"

namespace emg {
// ---- blocked Gauss-Jordan inversion with tensor-core trailing updates (tcgen05) ---------------
// The in-place Gauss-Jordan steps of the SIMT forms (gj.cu, gj_tile.cu, gj_cols.cu), grouped
// in panels of KB = 16 pivot columns.  Step k with pivot row p acts on every column c != k as
// A[:, c] <- M_k A[:, c],
// M_k = I + x_k e_p^T, so the KB steps of a panel act on the columns outside it as
// T = I + X S_P^T (S_P selects the panel's pivot rows); X[:, j] is the panel's column j after
// all KB steps minus e_{p_j} (the in-place rule leaves M_j e_{p_j} in column j at step j).
// The matrix lives in TMEM (row r in lane r mod 128 of row tile r / 128).  Per panel: every
// warp copies its rows' panel columns to shared memory; warp 0 alone factors the panel in
// registers (lane l holds rows l, l + 32, ...: the pivot search and the pivot row's broadcast
// are warp shuffles, so the steps need no block barrier); then every other column takes the
// rank-KB update A += X A[P, :] as one tcgen05.mma per row tile and 32-byte K step (3xTF32:
// x = hi + lo, X_hi R_hi + X_hi R_lo + X_lo R_hi, float32 accumulation).  Pivot choice and tie
// rule are those of the SIMT forms (largest |a_rk| among the unused rows, lowest row on
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

// The tensor-core inverse of the level's blocks; *built = false for block sizes it has no
// instance for.
emg_status launch_gj_tc(emg_ctx* c, int B, float* blk, bool* built) {
    *built = true;
    switch (B) {
        case 75: return gj_tc_go<75>(c, blk);
        case 100: return gj_tc_go<100>(c, blk);
        case 175: return gj_tc_go<175>(c, blk);
        default: *built = false; return EMG_OK;
    }
}

}  // namespace emg
