// Exact Jacobian blocks (Sec. 3.3).  The face Jacobians dF~/dU_L, dF~/dU_R (forward-mode AD
// of the Roe flux) are in jac_face.cu, the tensor-core form of the float32 assembly in
// jac_tc.cu; here:
//  * k_diag_blocks: element-diagonal block of Eq. jac1,
//      D[(a,i),(b,j)] = sum_q psi_j(x_q) sum_k W_q d_k psi_i(x_q) A_k[a][b](U_q)
//                       - sum_{L faces} sum_t psi_i psi_j w|n dS| dF~/dU_L[a][b]
//                       + sum_{R faces} sum_t psi_i psi_j w|n dS| dF~/dU_R[a][b]
//    with A_k = dF_k/dU in closed form (Appendix, Eq. dfdu, omega = 0), written either as
//    D or as the PRK operator P = I/dtau - D with dtau of Eq. x3d.
//  * k_bsr0: the p = 0 Jacobian (Eqs. jac1, jac2) as one diagonal and 2d off-diagonal
//    5x5 blocks per element.
#include <algorithm>

#include <cuda_bf16.h>

#include "blocks.cuh"
#include "common.cuh"
#include "dispatch.cuh"
#include "euler.cuh"
#include "jacobian.cuh"

namespace emg {

template <int D, int P>
struct DiagCfg {
    static constexpr int QC = D == 2 ? 32 : 16;  // volume points per shared-memory chunk
    static constexpr int THREADS = ((25 * Lv<D, P>::N + 31) / 32) * 32;
};

// Resident blocks asked of the register allocator: about 56 registers per thread for the
// FP32 blocks, 80 for FP64 (its 2N-register accumulator row).
template <int D, int P, class T>
struct DiagMinB {
    static constexpr int R = sizeof(T) == 4 ? 56 : 80;
    static constexpr int T_ = DiagCfg<D, P>::THREADS;
    static constexpr int V = (65536 / (T_ * R)) < 1 ? 1 : 65536 / (T_ * R);
};

// 16-byte vector of T (float4 or double2) for the broadcast reads of the staged basis rows.
template <class T>
struct Vec16;
template <>
struct Vec16<float> {
    using V = float4;
    static constexpr int L = 4;
    __device__ static void get(const float* p, float o[4]) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        o[0] = v.x, o[1] = v.y, o[2] = v.z, o[3] = v.w;
    }
};
template <>
struct Vec16<double> {
    using V = double2;
    static constexpr int L = 2;
    __device__ static void get(const double* p, double o[2]) {
        const double2 v = *reinterpret_cast<const double2*>(p);
        o[0] = v.x, o[1] = v.y;
    }
};

// acc[j] += s * row[j], j < N, with the row read 16 bytes at a time (row padded to NP).
template <int N, int NP, class T>
__device__ __forceinline__ void axpy_row(T (&acc)[N], T s, const T* row) {
    constexpr int VL = Vec16<T>::L;
#pragma unroll
    for (int j0 = 0; j0 < NP; j0 += VL) {
        T v[VL];
        Vec16<T>::get(row + j0, v);
#pragma unroll
        for (int c = 0; c < VL; ++c)
            if (j0 + c < N) acc[j0 + c] += s * v[c];
    }
}

// One CTA per element; thread (a, b, i) accumulates row (a,i), columns (b, 0..N-1).
// T is the block precision: double (FP64 form) or float (FP32 block form, with float
// copies of the basis tables; state and face Jacobians are rounded to float on load).
template <int D, int P, class T>
__global__ void __launch_bounds__(DiagCfg<D, P>::THREADS, (DiagMinB<D, P, T>::V)) k_diag_blocks(
    int E, int nmax, const double* __restrict__ u, const T* __restrict__ vpsi, const T* __restrict__ vgw,
    const int* __restrict__ elem_face, const T* __restrict__ fpsiL, const T* __restrict__ fpsiR,
    const T* __restrict__ fjl, const T* __restrict__ fjr, const double* __restrict__ psic,
    const double* __restrict__ hlen, const double* __restrict__ cfl_dev, double g, int shifted,
    const double* __restrict__ vvr, T* __restrict__ out) {
    using L = Lv<D, P>;
    constexpr int N = L::N, Q = L::Q, QF = L::QF, B = L::B, NF = L::NF;
    constexpr int QC = DiagCfg<D, P>::QC;
    constexpr int VL = Vec16<T>::L, NP = ((N + VL - 1) / VL) * VL;   // padded basis rows
    // the finished block goes out through shared memory (coalesced) when it fits
    constexpr bool STAGE = (size_t)B * B * sizeof(T) <= 24576;
    __shared__ double ud[B];
    __shared__ T us[B];
    __shared__ T As[QC][D][25];
    __shared__ __align__(16) T ps[QC][NP];
    __shared__ T gs[QC][D][N];
    __shared__ T Us[QC][5];
    __shared__ __align__(16) T fps[QF][NP];
    __shared__ T fjs[QF][25];
    __shared__ __align__(16) T ob[STAGE ? B * B : 1];
    __shared__ double s_dtau;
    const int e = blockIdx.x;
    const int tid = threadIdx.x;
    for (int t = tid; t < B; t += blockDim.x) {
        const double v = u[(size_t)e * B + t];
        ud[t] = v;
        us[t] = (T)v;
    }
    __syncthreads();
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
    const bool active = tid < 25 * N;
    const int ab = tid / N, i = tid % N;
    const int a = ab / 5, b = ab % 5;
    T acc[N];
#pragma unroll
    for (int j = 0; j < N; ++j) acc[j] = (T)0;
    if (P > 0) {
        for (int q0 = 0; q0 < Q; q0 += QC) {
            const int nq = (Q - q0) < QC ? (Q - q0) : QC;
            __syncthreads();
            // stage the chunk's psi and W grad psi, and build U at its points (all threads)
            const T* pg = vpsi + ((size_t)e * Q + q0) * N;
            for (int t = tid; t < nq * NP; t += blockDim.x) {
                const int q = t / NP, j = t % NP;
                ps[q][j] = j < N ? pg[q * N + j] : (T)0;
            }
            for (int t = tid; t < D * nq * N; t += blockDim.x) {
                const int k = t / (nq * N), r = t % (nq * N);
                gs[r / N][k][r % N] = vgw[(((size_t)e * D + k) * Q + q0) * N + r];
            }
            for (int t = tid; t < nq * 5; t += blockDim.x) {
                const int q = t / 5, c = t % 5;
                const T* pq = pg + (size_t)q * N;
                T s = (T)0;
                for (int m = 0; m < N; ++m) s += us[c * N + m] * pq[m];
                Us[q][c] = s;
            }
            __syncthreads();
            for (int t = tid; t < nq * D; t += blockDim.x) {
                flux_jac_k(Us[t / D], (T)g, t % D, As[t / D][t % D]);
                if (vvr) {   // rotating frame: A_k - (v_r)_k I
                    const T vr = (T)vvr[((size_t)e * Q + q0 + t / D) * 3 + t % D];
#pragma unroll
                    for (int a = 0; a < 5; ++a) As[t / D][t % D][a * 6] -= vr;
                }
            }
            __syncthreads();
            if (active) {
                for (int t = 0; t < nq; ++t) {
                    T s = (T)0;
#pragma unroll
                    for (int k = 0; k < D; ++k) s += gs[t][k][i] * As[t][k][ab];
                    axpy_row<N, NP, T>(acc, s, ps[t]);
                }
            }
        }
    }
    // faces, one at a time: stage psi at its points and the face Jacobians of this
    // element's side (sign -1 on the L side, +1 on the R side)
#pragma unroll 1
    for (int lf = 0; lf < NF; ++lf) {
        const int code = elem_face[(size_t)e * NF + lf];
        const T* pt = ((code & 1) ? fpsiR : fpsiL) + ((size_t)(code >> 1) * QF) * N;
        const T* fj = ((code & 1) ? fjr : fjl) + ((size_t)(code >> 1) * QF) * 25;
        __syncthreads();
        for (int t = tid; t < QF * NP; t += blockDim.x) {
            const int q = t / NP, j = t % NP;
            fps[q][j] = j < N ? pt[q * N + j] : (T)0;
        }
        for (int t = tid; t < QF * 25; t += blockDim.x) fjs[t / 25][t % 25] = (code & 1) ? fj[t] : -fj[t];
        __syncthreads();
        if (active) {
            for (int t = 0; t < QF; ++t) {
                const T s = fps[t][i] * fjs[t][ab];
                axpy_row<N, NP, T>(acc, s, fps[t]);
            }
        }
    }
    __syncthreads();
    if (active) {
        T* row = STAGE ? ob + (size_t)(a * N + i) * B + b * N : out + (size_t)e * B * B + (size_t)(a * N + i) * B + b * N;
        if (shifted) {
            const T idt = (T)(1.0 / s_dtau);
#pragma unroll
            for (int j = 0; j < N; ++j) row[j] = ((a == b && i == j) ? idt : (T)0) - acc[j];
        } else {
#pragma unroll
            for (int j = 0; j < N; ++j) row[j] = acc[j];
        }
    }
    if (STAGE) {
        __syncthreads();
        T* g = out + (size_t)e * B * B;
        for (int t = tid; t < B * B; t += blockDim.x) g[t] = ob[t];
    }
}

// Register-blocked SIMT form of the float32 assembly (the default float32 form): thread
// (a, i, jg) accumulates row (a,i) of the block for all five b and the JW columns j of group jg,
// acc[b][j] += s_b psi_j with s_b = sum_k W d_k psi_i A_k[a][b] formed once per point and
// reused across the JW columns; every staged basis row is read 16 bytes at a time and
// broadcast.  Per entry the terms are summed in the order of k_diag_blocks (points in order,
// then the faces, each product as one FMA), so both forms give bitwise the same blocks.
template <int D, int P>
struct DiagRb {
    static constexpr int N = Lv<D, P>::N;
    static constexpr int JW = N <= 16 ? ((N + 3) / 4) * 4 : 20;    // columns j per thread
    static constexpr int JG = (N + JW - 1) / JW;                     // column groups
    static constexpr int NPAD = JG * JW;                             // padded basis row
    static constexpr int ROWS = 5 * N;                               // (a, i)
    static constexpr int THREADS = ((ROWS * JG + 31) / 32) * 32;
    static constexpr int QC = D == 2 ? 36 : 24;                      // volume points per chunk
    static constexpr int B = Lv<D, P>::B;
    // the finished block leaves through shared memory: whole when it fits, else one b at a time
    static constexpr bool WHOLE = (size_t)B * B * sizeof(float) <= 24576;
    static constexpr int OLD = N + 1;                                // row stride of a b-slab
    static constexpr int OB = WHOLE ? B * B : ROWS * OLD;
    // shared memory (floats): the chunk and face buffers, with the output buffer over them
    static constexpr int Q = Lv<D, P>::Q, QF = Lv<D, P>::QF;
    static constexpr int O_PS = 0;                                   // [QC][NPAD]
    static constexpr int O_FPS = O_PS + QC * NPAD;                   // [QF][NPAD]
    static constexpr int O_GS = O_FPS + QF * NPAD;                   // [QC][D][N]
    static constexpr int O_AS = O_GS + QC * D * N;                   // [QC][D][25]
    static constexpr int O_US = O_AS + QC * D * 25;                  // [QC][5]
    static constexpr int O_FJ = O_US + QC * 5;                       // [QF][25]
    static constexpr int PHASE = O_FJ + QF * 25;
    static constexpr int SM = PHASE > OB ? PHASE : OB;
    static constexpr int REGS = 5 * JW > 80 ? 168 : 128;             // register budget per thread
    static constexpr int MINB = (65536 / (THREADS * REGS)) < 1 ? 1 : 65536 / (THREADS * REGS);
};

template <int D, int P>
__global__ void __launch_bounds__(DiagRb<D, P>::THREADS, DiagRb<D, P>::MINB) k_diag_blocks_rb(
    int E, int nmax, const double* __restrict__ u, const float* __restrict__ vpsi, const float* __restrict__ vgw,
    const int* __restrict__ elem_face, const float* __restrict__ fpsiL, const float* __restrict__ fpsiR,
    const float* __restrict__ fjl, const float* __restrict__ fjr, const double* __restrict__ psic,
    const double* __restrict__ hlen, const double* __restrict__ cfl_dev, double g, int shifted,
    const double* __restrict__ vvr, float* __restrict__ out) {
    using L = Lv<D, P>;
    using R = DiagRb<D, P>;
    constexpr int N = L::N, Q = L::Q, QF = L::QF, B = L::B, NF = L::NF;
    constexpr int JW = R::JW, JG = R::JG, NPAD = R::NPAD, QC = R::QC;
    __shared__ double ud[B];
    __shared__ float us[B];
    __shared__ __align__(16) float smf[R::SM];
    __shared__ double s_dtau;
    float(*ps)[NPAD] = reinterpret_cast<float(*)[NPAD]>(smf + R::O_PS);
    float(*fps)[NPAD] = reinterpret_cast<float(*)[NPAD]>(smf + R::O_FPS);
    float(*gs)[D][N] = reinterpret_cast<float(*)[D][N]>(smf + R::O_GS);
    float(*As)[D][25] = reinterpret_cast<float(*)[D][25]>(smf + R::O_AS);
    float(*Us)[5] = reinterpret_cast<float(*)[5]>(smf + R::O_US);
    float(*fjs)[25] = reinterpret_cast<float(*)[25]>(smf + R::O_FJ);
    float* ob = smf;   // over the chunk buffers, once the accumulation is done
    const int e = blockIdx.x;
    const int tid = threadIdx.x;
    for (int t = tid; t < B; t += blockDim.x) {
        const double v = u[(size_t)e * B + t];
        ud[t] = v;
        us[t] = (float)v;
    }
    __syncthreads();
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
    // thread (a, i, jg): consecutive threads take consecutive i, so a warp shares a and jg
    const bool active = tid < R::ROWS * JG;
    const int a = tid / (N * JG), rem = tid % (N * JG);
    const int jg = rem / N, i = rem % N;
    const int j0 = jg * JW;
    float acc[5][JW];
#pragma unroll
    for (int b = 0; b < 5; ++b)
#pragma unroll
        for (int j = 0; j < JW; ++j) acc[b][j] = 0.0f;
    // face data (basis traces and the signed face Jacobians) of the next face, loaded into
    // registers one face ahead so that the loads overlap the previous face's (or, for the
    // first face, the volume's) accumulation; stored to shared memory between two barriers
    constexpr int T = R::THREADS;
    constexpr int NPF = (QF * NPAD + T - 1) / T, NJF = (QF * 25 + T - 1) / T;
    float pf[NPF], pj[NJF];
    auto fetch_face = [&](int lf) {
        const int code = elem_face[(size_t)e * NF + lf];
        const float* pt = ((code & 1) ? fpsiR : fpsiL) + ((size_t)(code >> 1) * QF) * N;
        const float* fj = ((code & 1) ? fjr : fjl) + ((size_t)(code >> 1) * QF) * 25;
#pragma unroll
        for (int k = 0; k < NPF; ++k) {
            const int t = tid + k * T, q = t / NPAD, j = t % NPAD;
            pf[k] = (t < QF * NPAD && j < N) ? pt[q * N + j] : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < NJF; ++k) {
            const int t = tid + k * T;
            pj[k] = t < QF * 25 ? ((code & 1) ? fj[t] : -fj[t]) : 0.0f;
        }
    };
    fetch_face(0);
    if (P > 0) {
        for (int q0 = 0; q0 < Q; q0 += QC) {
            const int nq = (Q - q0) < QC ? (Q - q0) : QC;
            __syncthreads();
            const float* pg = vpsi + ((size_t)e * Q + q0) * N;
            for (int t = tid; t < nq * NPAD; t += blockDim.x) {
                const int q = t / NPAD, j = t % NPAD;
                ps[q][j] = j < N ? pg[q * N + j] : 0.0f;
            }
            for (int t = tid; t < D * nq * N; t += blockDim.x) {
                const int k = t / (nq * N), r = t % (nq * N);
                gs[r / N][k][r % N] = vgw[(((size_t)e * D + k) * Q + q0) * N + r];
            }
            for (int t = tid; t < nq * 5; t += blockDim.x) {
                const int q = t / 5, c = t % 5;
                const float* pq = pg + (size_t)q * N;
                float s = 0.0f;
                for (int m = 0; m < N; ++m) s += us[c * N + m] * pq[m];
                Us[q][c] = s;
            }
            __syncthreads();
            for (int t = tid; t < nq * D; t += blockDim.x) {
                flux_jac_k(Us[t / D], (float)g, t % D, As[t / D][t % D]);
                if (vvr) {   // rotating frame: A_k - (v_r)_k I
                    const float vr = (float)vvr[((size_t)e * Q + q0 + t / D) * 3 + t % D];
#pragma unroll
                    for (int a = 0; a < 5; ++a) As[t / D][t % D][a * 6] -= vr;
                }
            }
            __syncthreads();
            if (active) {
#pragma unroll 1
                for (int t = 0; t < nq; ++t) {
                    float gk[D];
#pragma unroll
                    for (int k = 0; k < D; ++k) gk[k] = gs[t][k][i];
                    float s[5];
#pragma unroll
                    for (int b = 0; b < 5; ++b) {
                        float x = 0.0f;
#pragma unroll
                        for (int k = 0; k < D; ++k) x += gk[k] * As[t][k][a * 5 + b];
                        s[b] = x;
                    }
#pragma unroll
                    for (int jj = 0; jj < JW; jj += 4) {
                        const float4 v = *reinterpret_cast<const float4*>(&ps[t][j0 + jj]);
                        const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int c = 0; c < 4; c += 2)
#pragma unroll
                            for (int b = 0; b < 5; ++b) fma2f(s[b], vv[c], vv[c + 1], acc[b][jj + c], acc[b][jj + c + 1]);
                    }
                }
            }
        }
    }
#pragma unroll 1
    for (int lf = 0; lf < NF; ++lf) {
        __syncthreads();
#pragma unroll
        for (int k = 0; k < NPF; ++k) {
            const int t = tid + k * T;
            if (t < QF * NPAD) fps[t / NPAD][t % NPAD] = pf[k];
        }
#pragma unroll
        for (int k = 0; k < NJF; ++k) {
            const int t = tid + k * T;
            if (t < QF * 25) fjs[t / 25][t % 25] = pj[k];
        }
        __syncthreads();
        if (lf + 1 < NF) fetch_face(lf + 1);
        if (active) {
#pragma unroll 1
            for (int t = 0; t < QF; ++t) {
                const float pi = fps[t][i];
                float s[5];
#pragma unroll
                for (int b = 0; b < 5; ++b) s[b] = pi * fjs[t][a * 5 + b];
#pragma unroll
                for (int jj = 0; jj < JW; jj += 4) {
                    const float4 v = *reinterpret_cast<const float4*>(&fps[t][j0 + jj]);
                    const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int c = 0; c < 4; c += 2)
#pragma unroll
                        for (int b = 0; b < 5; ++b) fma2f(s[b], vv[c], vv[c + 1], acc[b][jj + c], acc[b][jj + c + 1]);
                }
            }
        }
    }
    const float idt = shifted ? (float)(1.0 / s_dtau) : 0.0f;
    float* g_out = out + (size_t)e * B * B;
    if (R::WHOLE) {
        __syncthreads();
        if (active) {
#pragma unroll
            for (int b = 0; b < 5; ++b)
#pragma unroll
                for (int j = 0; j < JW; ++j) {
                    const int jj = j0 + j;
                    if (jj < N) {
                        const float v = acc[b][j];
                        ob[(a * N + i) * B + b * N + jj] = shifted ? ((a == b && i == jj) ? idt : 0.0f) - v : v;
                    }
                }
        }
        __syncthreads();
        for (int t = tid; t < B * B; t += blockDim.x) g_out[t] = ob[t];
    } else {
        constexpr int OLD = R::OLD;
#pragma unroll
        for (int b = 0; b < 5; ++b) {   // unrolled: acc[b] stays in registers
            __syncthreads();
            if (active) {
#pragma unroll
                for (int j = 0; j < JW; ++j) {
                    const int jj = j0 + j;
                    if (jj < N) {
                        const float v = acc[b][j];
                        ob[(a * N + i) * OLD + jj] = shifted ? ((a == b && i == jj) ? idt : 0.0f) - v : v;
                    }
                }
            }
            __syncthreads();
            for (int t = tid; t < R::ROWS * N; t += blockDim.x) {
                const int r = t / N, j = t % N;
                g_out[(size_t)r * B + b * N + j] = ob[r * OLD + j];
            }
        }
    }
}

// Float copies of the level tables used by the FP32 block path.
__global__ void k_to_float(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = (float)x[i];
}

// p = 0 block-sparse Jacobian: bsr[e][0] = diagonal block, bsr[e][1+lf] = dR_e/du_nb(lf).
__global__ void k_bsr0(int E, int NF, int QF, const int* __restrict__ elem_face, const double* __restrict__ fpsiL,
                       const double* __restrict__ fpsiR, const double* __restrict__ fjl,
                       const double* __restrict__ fjr, int F_int, double* __restrict__ bsr) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)E * 25) return;
    const int e = (int)(idx / 25), ab = (int)(idx % 25);
    double diag = 0.0;
    double* row = bsr + (size_t)e * (1 + NF) * 25;
    for (int lf = 0; lf < NF; ++lf) {
        const int code = elem_face[(size_t)e * NF + lf];
        const int f = code >> 1;
        const bool rside = code & 1;
        double sd = 0.0, so = 0.0;
        for (int t = 0; t < QF; ++t) {
            const size_t pidx = (size_t)f * QF + t;
            if (!rside) {
                const double pl = fpsiL[pidx];
                sd -= pl * pl * fjl[pidx * 25 + ab];
                if (f < F_int) so -= pl * fpsiR[pidx] * fjr[pidx * 25 + ab];
            } else {
                const double pr = fpsiR[pidx];
                sd += pr * pr * fjr[pidx * 25 + ab];
                so += pr * fpsiL[pidx] * fjl[pidx * 25 + ab];
            }
        }
        diag += sd;
        row[(1 + lf) * 25 + ab] = so;
    }
    row[ab] = diag;
}

// Jacobian of the rotating frame's source (Eq. euler: S = (0, -omega x (rho v), 0), linear in U):
// dS_m/d(rho v)_n = -eps_{m k n} omega_k, so with the orthonormal basis every element's block
// gains dS/dU on the momentum rows and columns of each mode i (the same i).  The Appendix's
// printed dS/dU (Eq. dsdu) has the opposite sign; the sign here is that of S as written.
// Added to D = dR/du (shifted = 0) or subtracted from P = I/dtau - D (shifted = 1); block rows
// (a, i) of stride ld per element, element stride es.
template <class T>
__global__ void k_add_source(int64_t E, int N, int64_t es, int ld, int shifted, U5 om, T* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const double dS[3][3] = {{0.0, om.v[2], -om.v[1]}, {-om.v[2], 0.0, om.v[0]}, {om.v[1], -om.v[0], 0.0}};
    const double sg = shifted ? -1.0 : 1.0;
    T* b = out + e * es;
    for (int i = 0; i < N; ++i)
        for (int m = 0; m < 3; ++m)
            for (int n = 0; n < 3; ++n)
                if (m != n) b[(size_t)((1 + m) * N + i) * ld + (1 + n) * N + i] += (T)(sg * dS[m][n]);
}

template <class T>
static emg_status add_source_jacobian(emg_ctx* c, int p, int shifted, T* out) {
    if (!c->rot) return EMG_OK;
    const LevelDev& L = c->lv[p];
    U5 om{};
    for (int k = 0; k < 3; ++k) om.v[k] = c->prm.omega[k];
    { ProfScope _ps(c, PC_DIAG); k_add_source<T><<<(unsigned)((c->E + 127) / 128), 128, 0, c->stream>>>(
        c->E, L.N, (int64_t)L.B * L.B, L.B, shifted, om, out); }
    EMG_CHECK_LAUNCH(c);
    return EMG_OK;
}

emg_status launch_diag_blocks(emg_ctx* c, int p, const double* u, const double* cfl_dev, int shifted, double* out) {
    emg_status st = launch_face_jacobian(c, p, u);
    if (st != EMG_OK) return st;
    LevelDev& L = c->lv[p];
    const int nmax = n_modes(c->dim, c->p_max);
#define EMG_DB(DD, PP)                                                                                      \
    {                                                                                                       \
        ProfScope _ps(c, PC_DIAG);                                                                          \
        k_diag_blocks<DD, PP, double><<<(unsigned)c->E, DiagCfg<DD, PP>::THREADS, 0, c->stream>>>(          \
            (int)c->E, nmax, u, L.vpsi, L.vgw, c->elem_face, L.fpsiL, L.fpsiR, L.fjl, L.fjr, c->psic, c->h, \
            cfl_dev, c->prm.gamma, shifted, L.vvr, out);                                                    \
    }
    EMG_DISPATCH_DP(c->dim, p, EMG_DB)
#undef EMG_DB
    EMG_CHECK_LAUNCH(c);
    return add_source_jacobian(c, p, shifted, out);
}

// Block assembly of the float32 block forms (levels p >= 1): on the tensor cores or, where the
// level's choice says so, the SIMT form.
emg_status launch_diag_blocks32(emg_ctx* c, int p, const double* u, const double* cfl_dev, int shifted,
                                float* out) {
    emg_status st = launch_face_jacobian32(c, p, u);
    if (st != EMG_OK) return st;
    LevelDev& L = c->lv[p];
    if (!L.vpsi32) {
        c->err = "FP32 tables not built";
        return EMG_ERR_ARG;
    }
    if (!L.tc_asm) {
        // the SIMT (FMA) form of the same contraction
        const int nmax = n_modes(c->dim, c->p_max);
#define EMG_DB32(DD, PP)                                                                                    \
    {                                                                                                       \
        ProfScope _ps(c, PC_DIAG);                                                                          \
        if (c->prm.block_kernels == 3)                                                                      \
            k_diag_blocks<DD, PP, float><<<(unsigned)c->E, DiagCfg<DD, PP>::THREADS, 0, c->stream>>>(       \
                (int)c->E, nmax, u, L.vpsi32, L.vgw32, c->elem_face, L.fpsiL32, L.fpsiR32, L.fjl32, L.fjr32,  \
                c->psic, c->h, cfl_dev, c->prm.gamma, shifted, L.vvr, out);                                 \
        else                                                                                                \
            k_diag_blocks_rb<DD, PP><<<(unsigned)c->E, DiagRb<DD, PP>::THREADS, 0, c->stream>>>(            \
                (int)c->E, nmax, u, L.vpsi32, L.vgw32, c->elem_face, L.fpsiL32, L.fpsiR32, L.fjl32, L.fjr32,  \
                c->psic, c->h, cfl_dev, c->prm.gamma, shifted, L.vvr, out);                                 \
    }
        EMG_DISPATCH_DP(c->dim, p, EMG_DB32)
#undef EMG_DB32
        EMG_CHECK_LAUNCH(c);
        return add_source_jacobian(c, p, shifted, out);
    }
    st = launch_diag_blocks_tc(c, p, u, cfl_dev, shifted, out);
    if (st != EMG_OK) return st;
    return add_source_jacobian(c, p, shifted, out);
}

emg_status build_float_tables(emg_ctx* c) {
    for (int p = 1; p <= c->p_max; ++p) {
        LevelDev& L = c->lv[p];
        const int64_t n1 = c->E * L.Q * L.N, n2 = c->E * c->dim * L.Q * L.N;
        const int64_t n3 = c->F * L.QF * L.N, n4 = std::max<int64_t>(c->F_int, 1) * L.QF * L.N;
        const double* src[4] = {L.vpsi, L.vgw, L.fpsiL, L.fpsiR};
        float* dst[4] = {L.vpsi32, L.vgw32, L.fpsiL32, L.fpsiR32};
        const int64_t cnt[4] = {n1, n2, n3, n4};
        for (int k = 0; k < 4; ++k) {
            ProfScope _ps(c, PC_SETUP);
            k_to_float<<<(unsigned)((cnt[k] + 255) / 256), 256, 0, c->stream>>>(cnt[k], src[k], dst[k]);
        }
        EMG_CHECK_LAUNCH(c);
    }
    return EMG_OK;
}

emg_status launch_bsr0(emg_ctx* c) {
    LevelDev& L = c->lv[0];
    const int64_t n = c->E * 25;
    { ProfScope _ps(c, PC_BSR0); k_bsr0<<<(unsigned)((n + 127) / 128), 128, 0, c->stream>>>((int)c->E, 2 * c->dim, L.QF, c->elem_face, L.fpsiL,
                                                               L.fpsiR, L.fjl, L.fjr, (int)c->F_int, c->bsr); }
    EMG_CHECK_LAUNCH(c);
    if (c->rot) {   // p = 0: the diagonal 5x5 block (first of each element's row) gains dS/dU
        U5 om{};
        for (int k = 0; k < 3; ++k) om.v[k] = c->prm.omega[k];
        { ProfScope _ps(c, PC_BSR0); k_add_source<double><<<(unsigned)((c->E + 127) / 128), 128, 0, c->stream>>>(
            c->E, 1, (1 + 2 * c->dim) * 25, 5, 0, om, c->bsr); }
        EMG_CHECK_LAUNCH(c);
    }
    return EMG_OK;
}

}  // namespace emg
