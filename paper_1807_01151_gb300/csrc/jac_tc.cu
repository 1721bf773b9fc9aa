// Tensor-core assembly of the float32 block forms (Eq. jac1 per element on tcgen05).
#include <cuda_bf16.h>

#include "common.cuh"
#include "euler.cuh"
#include "jacobian.cuh"
#include "tc.cuh"

namespace emg {

// ---- tensor-core assembly of the float32 block forms (tcgen05) ------------------------------
// Eq. jac1 per element as one matrix product C = G Psi with
//   rows    m = (a b, i)      (25 N rows, in 128-row tiles),
//   columns j                  (N, padded to a multiple of 16),
//   depth   k = quadrature point: the Q volume points, then the QF points of every face,
//   G[m][k] = sum_d W_k d_d psi_i(x_k) A_d[a][b](U(x_k))      (volume point)
//           = -/+ psi_i(x_k) w|n dS| dF~/dU_{L/R}[a][b]          (face point, L/R side)
//   Psi[k][j] = psi_j(x_k),
// so D[(a,i),(b,j)] = C[(a b, i)][j] and P_e = I/dtau_e - D.  The depth is processed in chunks
// of KC points: all threads build the chunk's G and Psi in shared memory in the K-major
// core-matrix layout (each thread one 16-byte core row), one thread issues the MMAs into the
// TMEM accumulators (one 128 x NPAD accumulator per row tile), and the chunk buffers are
// double buffered against the MMAs through one mbarrier each.
//  * EMG_PREC_FP32_BLOCKS: kind::tf32 with each operand split as x = hi + lo (hi = tf32(x)) and
//    C += G_hi Psi_hi + G_hi Psi_lo + G_lo Psi_hi, which keeps float32 accuracy;
//  * EMG_PREC_BF16_BLOCKS: kind::f16 with bfloat16 operands, one product.
// Accumulation is in float32 throughout.  The epilogue reads the accumulators back with
// tcgen05.ld (warp w owns TMEM lanes 32 (w mod 4) ...), applies the I/dtau shift and writes
// the block row-major, through shared memory when it fits.
template <int D, int P, bool BF16>
struct TcAsm {
    using L = Lv<D, P>;
    static constexpr int N = L::N, Q = L::Q, QF = L::QF, NF = L::NF, B = L::B;
    static constexpr int MROWS = 25 * N;
    static constexpr int MT = (MROWS + 127) / 128;
    static constexpr int MPAD = 128 * MT;
    static constexpr int NPAD = ((N + 15) / 16) * 16;
    static constexpr int KTOT = Q + NF * QF;
    static constexpr int KSTEP = BF16 ? 16 : 8;          // depth of one MMA (32 bytes of K)
    static constexpr int KC = BF16 ? 16 : 8;               // points per chunk (small: more CTAs per SM)
    static constexpr int NCHUNK = (KTOT + KC - 1) / KC;
    static constexpr int ESZ = BF16 ? 2 : 4;
    static constexpr int PER_CORE = 16 / ESZ;            // depth elements per core-matrix row
    static constexpr int NSPLIT = BF16 ? 1 : 2;
    static constexpr uint32_t A_LBO = (MPAD / 8) * 128, B_LBO = (NPAD / 8) * 128, SBO = 128;
    static constexpr int A_BYTES = MPAD * KC * ESZ;
    static constexpr int B_BYTES = NPAD * KC * ESZ;
    static constexpr int BUF = NSPLIT * (A_BYTES + B_BYTES);
    static constexpr int COLS = MT * NPAD;
    static constexpr uint32_t TMEM_COLS = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128 : COLS <= 256 ? 256 : 512;
    static constexpr int THREADS = 256;
    static constexpr int OUT_BYTES = B * B * 4;
    static constexpr bool STAGE_OUT = OUT_BYTES <= 2 * BUF;
    static constexpr int SMEM = 2 * BUF;
    static_assert(KC % KSTEP == 0 && KC % PER_CORE == 0, "chunk must hold whole MMAs");
    static_assert(COLS <= 512, "accumulators exceed the SM's tensor memory");
};

template <int D, int P, bool BF16>
__global__ void __launch_bounds__(256) k_diag_blocks_tc(
    int E, int nmax, const double* __restrict__ u, const float* __restrict__ vpsi, const float* __restrict__ vgw,
    const int* __restrict__ elem_face, const float* __restrict__ fpsiL, const float* __restrict__ fpsiR,
    const float* __restrict__ fjl, const float* __restrict__ fjr, const double* __restrict__ psic,
    const double* __restrict__ hlen, const double* __restrict__ cfl_dev, double g, int shifted,
    const double* __restrict__ vvr, float* __restrict__ out, int* __restrict__ timeout_flag) {
    using C = TcAsm<D, P, BF16>;
    constexpr int N = C::N, Q = C::Q, QF = C::QF, NF = C::NF, B = C::B, KC = C::KC, KTOT = C::KTOT;
    constexpr int NPAD = C::NPAD, MPAD = C::MPAD, MROWS = C::MROWS, T = C::THREADS;
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ double ud[B];
    __shared__ float us[B];
    __shared__ float Uq[KC][5];
    __shared__ float psi_s[KC][NPAD];
    __shared__ float basis_s[KC][D][N];
    __shared__ float coef_s[KC][D][25];
    __shared__ int fcode[NF];
    __shared__ double s_dtau;
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tbase_s;
    __shared__ int s_fail;
    const int e = blockIdx.x;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long budget = 2000000000LL;   // about a second of SM clock per wait
    for (int t = tid; t < B; t += T) {
        const double v = u[(size_t)e * B + t];
        ud[t] = v;
        us[t] = (float)v;
    }
    if (tid < NF) fcode[tid] = elem_face[(size_t)e * NF + tid];
    if (tid == 0) {
        s_fail = 0;
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(&tbase_s, C::TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = tbase_s;
    if (tid == 0 && shifted) {
        double Uc[5];
        for (int a = 0; a < 5; ++a) {
            double s = 0.0;
            for (int i = 0; i < N; ++i) s += ud[a * N + i] * psic[(size_t)e * nmax + i];
            Uc[a] = s;
        }
        const double ir = 1.0 / Uc[0];
        const double vx = Uc[1] * ir, vy = Uc[2] * ir, vz = Uc[3] * ir;
        const double q2 = vx * vx + vy * vy + vz * vz;
        const double pr = (g - 1.0) * (Uc[4] - 0.5 * Uc[0] * q2);
        const double cs = sqrt(g * pr * ir);
        s_dtau = cfl_dev[0] * hlen[e] / ((2 * P + 1) * (sqrt(q2) + cs));
    }
    const uint32_t idesc = tc::idesc(BF16 ? tc::AB_BF16 : tc::AB_TF32, 128, NPAD);
    bool failed = false;
#pragma unroll 1
    for (int c = 0; c < C::NCHUNK; ++c) {
        const int buf = c & 1;
        const int k0 = c * KC;
        __syncthreads();   // the previous chunk's staging arrays are consumed
        // (1) staging: U at the chunk's volume points; psi at every chunk point; the basis
        //     factors and the Jacobian coefficients of G
        for (int t = tid; t < KC; t += T) {
            const int k = k0 + t;
            if (k < Q) {
                const float* ps = vpsi + ((size_t)e * Q + k) * N;
                float U[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
                for (int i = 0; i < N; ++i) {
                    const float w = ps[i];
#pragma unroll
                    for (int a = 0; a < 5; ++a) U[a] += us[a * N + i] * w;
                }
#pragma unroll
                for (int a = 0; a < 5; ++a) Uq[t][a] = U[a];
            }
        }
        for (int t = tid; t < KC * NPAD; t += T) {
            const int kl = t / NPAD, j = t % NPAD, k = k0 + kl;
            float v = 0.f;
            if (j < N && k < KTOT) {
                if (k < Q) {
                    v = vpsi[((size_t)e * Q + k) * N + j];
                } else {
                    const int lf = (k - Q) / QF, tt = (k - Q) % QF, code = fcode[lf];
                    v = ((code & 1) ? fpsiR : fpsiL)[((size_t)(code >> 1) * QF + tt) * N + j];
                }
            }
            psi_s[kl][j] = v;
        }
        for (int t = tid; t < KC * D * N; t += T) {
            const int kl = t / (D * N), kk = (t / N) % D, i = t % N, k = k0 + kl;
            float v = 0.f;
            if (k < Q) {
                v = vgw[(((size_t)e * D + kk) * Q + k) * N + i];
            } else if (k < KTOT && kk == 0) {
                const int lf = (k - Q) / QF, tt = (k - Q) % QF, code = fcode[lf];
                v = ((code & 1) ? fpsiR : fpsiL)[((size_t)(code >> 1) * QF + tt) * N + i];
            }
            basis_s[kl][kk][i] = v;
        }
        __syncthreads();
        for (int t = tid; t < KC * D; t += T) {
            const int kl = t / D, kk = t % D, k = k0 + kl;
            float A[25];
            if (k < Q) {
                flux_jac_k(Uq[kl], (float)g, kk, A);
                if (vvr) {   // rotating frame: A_k - (v_r)_k I
                    const float vr = (float)vvr[((size_t)e * Q + k) * 3 + kk];
#pragma unroll
                    for (int a = 0; a < 5; ++a) A[a * 6] -= vr;
                }
            } else if (k < KTOT && kk == 0) {
                const int lf = (k - Q) / QF, tt = (k - Q) % QF, code = fcode[lf];
                const float* fj = ((code & 1) ? fjr : fjl) + ((size_t)(code >> 1) * QF + tt) * 25;
                const float sg = (code & 1) ? 1.f : -1.f;
#pragma unroll
                for (int ab = 0; ab < 25; ++ab) A[ab] = sg * fj[ab];
            } else {
#pragma unroll
                for (int ab = 0; ab < 25; ++ab) A[ab] = 0.f;
            }
#pragma unroll
            for (int ab = 0; ab < 25; ++ab) coef_s[kl][kk][ab] = A[ab];
        }
        // (2) the buffer is free once the MMAs of chunk c - 2 have completed
        if (c >= 2) {
            const bool ok = tc::mbar_wait(&mbar[buf], ((c - 2) >> 1) & 1, budget);
            if (!ok) s_fail = 1;
        }
        __syncthreads();
        if (s_fail) {
            failed = true;
            break;
        }
        unsigned char* bufp = tsm + buf * C::BUF;
        unsigned char* Ahi = bufp;
        unsigned char* Alo = bufp + (C::NSPLIT - 1) * C::A_BYTES;
        unsigned char* Bhi = bufp + C::NSPLIT * C::A_BYTES;
        unsigned char* Blo = Bhi + (C::NSPLIT - 1) * C::B_BYTES;
        constexpr int PC = C::PER_CORE;
        constexpr int KG = KC / PC;   // 16-byte core rows per matrix row in the chunk
        for (int it = tid; it < MPAD * KG; it += T) {
            const int m = it % MPAD, gq = it / MPAD;
            float v[PC];
            if (m < MROWS) {
                const int ab = m / N, i = m % N;
#pragma unroll
                for (int r = 0; r < PC; ++r) {
                    const int kl = gq * PC + r;
                    float s = 0.f;
#pragma unroll
                    for (int kk = 0; kk < D; ++kk) s += basis_s[kl][kk][i] * coef_s[kl][kk][ab];
                    v[r] = s;
                }
            } else {
#pragma unroll
                for (int r = 0; r < PC; ++r) v[r] = 0.f;
            }
            const size_t off = (size_t)gq * C::A_LBO + (size_t)(m >> 3) * C::SBO + (size_t)(m & 7) * 16;
            if constexpr (BF16) {
                __nv_bfloat162 h[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) h[r] = __floats2bfloat162_rn(v[2 * r], v[2 * r + 1]);
                *reinterpret_cast<uint4*>(Ahi + off) = *reinterpret_cast<uint4*>(h);
            } else {
                float4 hi, lo;
                hi.x = tc::tf32_round(v[0]), lo.x = tc::tf32_round(v[0] - hi.x);
                hi.y = tc::tf32_round(v[1]), lo.y = tc::tf32_round(v[1] - hi.y);
                hi.z = tc::tf32_round(v[2]), lo.z = tc::tf32_round(v[2] - hi.z);
                hi.w = tc::tf32_round(v[3]), lo.w = tc::tf32_round(v[3] - hi.w);
                *reinterpret_cast<float4*>(Ahi + off) = hi;
                *reinterpret_cast<float4*>(Alo + off) = lo;
            }
        }
        for (int it = tid; it < NPAD * KG; it += T) {
            const int n = it % NPAD, gq = it / NPAD;
            float v[PC];
#pragma unroll
            for (int r = 0; r < PC; ++r) v[r] = psi_s[gq * PC + r][n];
            const size_t off = (size_t)gq * C::B_LBO + (size_t)(n >> 3) * C::SBO + (size_t)(n & 7) * 16;
            if constexpr (BF16) {
                __nv_bfloat162 h[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) h[r] = __floats2bfloat162_rn(v[2 * r], v[2 * r + 1]);
                *reinterpret_cast<uint4*>(Bhi + off) = *reinterpret_cast<uint4*>(h);
            } else {
                float4 hi, lo;
                hi.x = tc::tf32_round(v[0]), lo.x = tc::tf32_round(v[0] - hi.x);
                hi.y = tc::tf32_round(v[1]), lo.y = tc::tf32_round(v[1] - hi.y);
                hi.z = tc::tf32_round(v[2]), lo.z = tc::tf32_round(v[2] - hi.z);
                hi.w = tc::tf32_round(v[3]), lo.w = tc::tf32_round(v[3] - hi.w);
                *reinterpret_cast<float4*>(Bhi + off) = hi;
                *reinterpret_cast<float4*>(Blo + off) = lo;
            }
        }
        tc::fence_proxy_async();
        __syncthreads();
        // (3) one thread issues the chunk's MMAs into every row tile's accumulator
        if (tid == 0) {
            tc::fence_after();
            const uint32_t ah = tc::smem_u32(Ahi), al = tc::smem_u32(Alo);
            const uint32_t bh = tc::smem_u32(Bhi), bl = tc::smem_u32(Blo);
#pragma unroll 1
            for (int t = 0; t < C::MT; ++t) {
                const uint32_t dcol = tbase + (uint32_t)(t * NPAD);
#pragma unroll
                for (int s = 0; s < KC / C::KSTEP; ++s) {
                    const uint32_t acc = (c == 0 && s == 0) ? 0u : 1u;
                    const uint32_t ka = (uint32_t)(2 * s) * C::A_LBO + (uint32_t)t * 16u * C::SBO;
                    const uint32_t kb = (uint32_t)(2 * s) * C::B_LBO;
                    const uint64_t dah = tc::sdesc(ah + ka, C::A_LBO, C::SBO);
                    const uint64_t dbh = tc::sdesc(bh + kb, C::B_LBO, C::SBO);
                    if constexpr (BF16) {
                        tc::mma_bf16(dcol, dah, dbh, idesc, acc);
                    } else {
                        tc::mma_tf32(dcol, dah, dbh, idesc, acc);
                        tc::mma_tf32(dcol, dah, tc::sdesc(bl + kb, C::B_LBO, C::SBO), idesc, 1u);
                        tc::mma_tf32(dcol, tc::sdesc(al + ka, C::A_LBO, C::SBO), dbh, idesc, 1u);
                    }
                }
            }
            tc::commit(&mbar[buf]);
        }
    }
    // every MMA has completed once the last chunk's commit has arrived
    {
        const int cl = C::NCHUNK - 1;
        const bool ok = tc::mbar_wait(&mbar[cl & 1], (cl >> 1) & 1, budget);
        if (!ok) failed = true;
    }
    if (__syncthreads_or(failed)) {
        if (tid == 0) atomicExch(timeout_flag, 1);
        tc::fence_before();
        __syncthreads();
        if (warp == 0) tc::tmem_dealloc(tbase, C::TMEM_COLS);
        return;
    }
    tc::fence_after();
    // (4) epilogue: P = I/dtau - D (or D), row (a, i) column (b, j)
    const float idt = shifted ? (float)(1.0 / s_dtau) : 0.f;
    float* ob = reinterpret_cast<float*>(tsm);
    float* og = out + (size_t)e * B * B;
    const int qd = warp & 3, grp = warp >> 2;
#pragma unroll 1
    for (int t = grp; t < C::MT; t += 2) {
        const int m = 128 * t + 32 * qd + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < NPAD; c0 += 16) {
            float r[16];
            tc::ld16(tbase + ((uint32_t)(32 * qd) << 16) + (uint32_t)(t * NPAD + c0), r);
            if (m < MROWS) {
                const int ab = m / N, i = m % N, a = ab / 5, b = ab % 5;
                float* row = (C::STAGE_OUT ? ob : og) + (size_t)(a * N + i) * B + b * N;
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    const int j = c0 + jj;
                    if (j < N) row[j] = ((a == b && i == j) ? idt : 0.f) - r[jj] * (shifted ? 1.f : -1.f);
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, C::TMEM_COLS);
    if constexpr (C::STAGE_OUT) {
        for (int t = tid; t < B * B; t += T) og[t] = ob[t];
    }
}

template <int D, int P, bool BF16>
static emg_status diag_tc_go(emg_ctx* c, const double* u, const double* cfl_dev, int shifted, float* out) {
    using C = TcAsm<D, P, BF16>;
    LevelDev& L = c->lv[P];
    const int nmax = n_modes(c->dim, c->p_max);
    EMG_CUDA_TRY(c, cudaFuncSetAttribute(k_diag_blocks_tc<D, P, BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         C::SMEM));
    {
        ProfScope _ps(c, PC_DIAG);
        k_diag_blocks_tc<D, P, BF16><<<(unsigned)c->E, C::THREADS, C::SMEM, c->stream>>>(
            (int)c->E, nmax, u, L.vpsi32, L.vgw32, c->elem_face, L.fpsiL32, L.fpsiR32, L.fjl32, L.fjr32, c->psic,
            c->h, cfl_dev, c->prm.gamma, shifted, L.vvr, out, &c->sc->timeout);
    }
    EMG_CHECK_LAUNCH(c);
    return EMG_OK;
}

emg_status launch_diag_blocks_tc(emg_ctx* c, int p, const double* u, const double* cfl_dev, int shifted,
                                 float* out) {
    const bool bf = c->prm.prec == EMG_PREC_BF16_BLOCKS;
#define EMG_TC(DD, PP) return bf ? diag_tc_go<DD, PP, true>(c, u, cfl_dev, shifted, out) \
                             : diag_tc_go<DD, PP, false>(c, u, cfl_dev, shifted, out)
    switch (c->dim * 8 + p) {
        case 17: EMG_TC(2, 1);
        case 18: EMG_TC(2, 2);
        case 19: EMG_TC(2, 3);
        case 20: EMG_TC(2, 4);
        case 25: EMG_TC(3, 1);
        case 26: EMG_TC(3, 2);
        case 27: EMG_TC(3, 3);
        case 28: EMG_TC(3, 4);
        default:
            c->err = "unsupported (dim, p) for the float32 block assembly";
            return EMG_ERR_ARG;
    }
#undef EMG_TC
}

}  // namespace emg
