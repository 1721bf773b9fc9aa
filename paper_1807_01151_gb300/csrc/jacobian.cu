// Exact Jacobian blocks (Sec. 3.3).
//  * k_face_jac: per face point, dF~/dU_L and dF~/dU_R of the Roe flux by forward-mode
//    AD (Dual<5>); on boundary faces the total derivative through the ghost state,
//    dF~/dU_L + dF~/dU_ghost dU_ghost/dU_L.
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
#include "tc.cuh"

namespace emg {

// The Roe flux of a face point and the ghost state of a boundary point for dual-number
// states; ROT: the face moves with the rotating frame (v_r at the point from fvr).
template <bool ROT, class T>
__device__ __forceinline__ void face_flux_d(const T UL[5], const T UR[5], const double n[3], double g,
                                            const double* __restrict__ fvr, int64_t idx, T F[5]) {
    if constexpr (ROT) {
        const double vrn = fvr[idx * 3] * n[0] + fvr[idx * 3 + 1] * n[1] + fvr[idx * 3 + 2] * n[2];
        roe_flux<T, true>(UL, UR, n, g, F, vrn);
    } else {
        roe_flux(UL, UR, n, g, F);
    }
}
template <bool ROT, class T>
__device__ __forceinline__ void ghost_d(const T UL[5], const double n[3], int bc, const double* __restrict__ wn,
                                        const U5& uinf, double g, const double* __restrict__ fvr, int64_t idx,
                                        T G[5]) {
    if (bc == EMG_BC_WALL || bc == EMG_BC_SYMMETRY) {
        const double nw[3] = {wn[0], wn[1], wn[2]};
        if constexpr (ROT) {
            const double vr[3] = {fvr[idx * 3], fvr[idx * 3 + 1], fvr[idx * 3 + 2]};
            wall_ghost_rel(UL, nw, vr, g, G);
        } else {
            wall_ghost(UL, nw, G);
        }
    } else {
        if constexpr (ROT) {
            const double vr[3] = {fvr[idx * 3], fvr[idx * 3 + 1], fvr[idx * 3 + 2]};
            farfield_ghost_rel(UL, n, uinf.v, g, vr, G);
        } else {
            farfield_ghost(UL, n, uinf.v, g, G);
        }
    }
}

template <int D, int P, class S, bool ROT>
__global__ void __launch_bounds__(128) k_face_jac(int F, int F_int, const int* __restrict__ fL,
                                                  const int* __restrict__ fR, const int* __restrict__ fbc,
                                                  const double* __restrict__ fnrm,
                                                  const double* __restrict__ famag,
                                                  const S* __restrict__ fpsiL,
                                                  const S* __restrict__ fpsiR,
                                                  const double* __restrict__ fwn,
                                                  const double* __restrict__ u, double g, U5 uinf,
                                                  const double* __restrict__ fvr,
                                                  S* __restrict__ fjl, S* __restrict__ fjr) {
    using L = Lv<D, P>;
    constexpr int N = L::N, QF = L::QF;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)F * QF) return;
    const int f = (int)(idx / QF);
    const double n[3] = {fnrm[idx * 3], fnrm[idx * 3 + 1], fnrm[idx * 3 + 2]};
    const S am = (S)famag[idx];
    S UL[5];
    {
        const double* ue = u + (size_t)fL[f] * 5 * N;
        const S* ps = fpsiL + idx * N;
        for (int a = 0; a < 5; ++a) {
            S s = (S)0;
            for (int i = 0; i < N; ++i) s += (S)ue[a * N + i] * ps[i];
            UL[a] = s;
        }
    }
    Dual<5, S> dL[5], dR[5], Fd[5];
    for (int a = 0; a < 5; ++a) {
        dL[a] = dconst<5, S>(UL[a]);
        dL[a].d[a] = (S)1;
    }
    if (f < F_int) {
        const double* ur = u + (size_t)fR[f] * 5 * N;
        const S* pr = fpsiR + idx * N;
        S UR[5];
        for (int a = 0; a < 5; ++a) {
            S s = (S)0;
            for (int i = 0; i < N; ++i) s += (S)ur[a * N + i] * pr[i];
            UR[a] = s;
            dR[a] = dconst<5, S>(s);
        }
        face_flux_d<ROT>(dL, dR, n, g, fvr, idx, Fd);
        for (int a = 0; a < 5; ++a)
            for (int b = 0; b < 5; ++b) fjl[idx * 25 + a * 5 + b] = am * Fd[a].d[b];
        Dual<5, S> cL[5];
        for (int a = 0; a < 5; ++a) {
            cL[a] = dconst<5, S>(UL[a]);
            dR[a].d[a] = (S)1;
        }
        face_flux_d<ROT>(cL, dR, n, g, fvr, idx, Fd);
        for (int a = 0; a < 5; ++a)
            for (int b = 0; b < 5; ++b) fjr[idx * 25 + a * 5 + b] = am * Fd[a].d[b];
    } else {
        ghost_d<ROT>(dL, n, fbc[f], fwn + (idx - (int64_t)F_int * QF) * 3, uinf, g, fvr, idx, dR);
        face_flux_d<ROT>(dL, dR, n, g, fvr, idx, Fd);
        for (int a = 0; a < 5; ++a)
            for (int b = 0; b < 5; ++b) fjl[idx * 25 + a * 5 + b] = am * Fd[a].d[b];
    }
}

// The same face Jacobians with one thread per (face point, side, direction b): the traces of a
// block's PPB face points are formed once in shared memory (one thread per point, side and
// component, the sums of k_face_jac in its order), then each thread differentiates the Roe flux
// (on a boundary face: the flux through the ghost state) along U_side[b] alone, with a
// one-direction dual number: column b of dF~/dU_side.  Forward mode computes every direction
// with the same operations, so the columns are bitwise those of the five-direction kernel; the
// flux value is recomputed per direction, for a tenth of the registers and ten threads per point.
template <int D, int P, class S>
struct FaceJacCol {
    static constexpr int PPB = 12;   // face points per block (10 threads each)
    static constexpr int THREADS = 128;
};

template <int D, int P, class S, bool ROT>
__global__ void __launch_bounds__(128) k_face_jac_col(int F, int F_int, const int* __restrict__ fL,
                                                      const int* __restrict__ fR, const int* __restrict__ fbc,
                                                      const double* __restrict__ fnrm,
                                                      const double* __restrict__ famag,
                                                      const S* __restrict__ fpsiL,
                                                      const S* __restrict__ fpsiR,
                                                      const double* __restrict__ fwn,
                                                      const double* __restrict__ u, double g, U5 uinf,
                                                      const double* __restrict__ fvr,
                                                      S* __restrict__ fjl, S* __restrict__ fjr) {
    using L = Lv<D, P>;
    constexpr int N = L::N, QF = L::QF, PPB = FaceJacCol<D, P, S>::PPB;
    __shared__ S Ut[PPB][2][5];
    const int64_t npts = (int64_t)F * QF;
    const int64_t p0 = (int64_t)blockIdx.x * PPB;
    const int tid = threadIdx.x;
    const int pt = tid / 10, r = tid % 10, side = r / 5, c = r % 5;
    const int64_t idx = p0 + pt;
    const bool live = tid < PPB * 10 && idx < npts;
    const int f = live ? (int)(idx / QF) : 0;
    const bool used = live && (side == 0 || f < F_int);
    if (used) {   // trace: component c on this side
        const double* ue = u + (size_t)(side ? fR[f] : fL[f]) * 5 * N;
        const S* ps = (side ? fpsiR : fpsiL) + idx * N;
        S s = (S)0;
        for (int i = 0; i < N; ++i) s += (S)ue[c * N + i] * ps[i];
        Ut[pt][side][c] = s;
    }
    __syncthreads();
    if (!used) return;
    const int b = c;   // from here on: the derivative direction
    const double n[3] = {fnrm[idx * 3], fnrm[idx * 3 + 1], fnrm[idx * 3 + 2]};
    const S am = (S)famag[idx];
    Dual<1, S> dL[5], dR[5], Fd[5];
    for (int a = 0; a < 5; ++a) dL[a] = dconst<1, S>(Ut[pt][0][a]);
    if (f < F_int) {
        for (int a = 0; a < 5; ++a) dR[a] = dconst<1, S>(Ut[pt][1][a]);
        if (side == 0)
            dL[b].d[0] = (S)1;
        else
            dR[b].d[0] = (S)1;
        face_flux_d<ROT>(dL, dR, n, g, fvr, idx, Fd);
        S* out = side ? fjr : fjl;
        for (int a = 0; a < 5; ++a) out[idx * 25 + a * 5 + b] = am * Fd[a].d[0];
    } else {
        dL[b].d[0] = (S)1;
        ghost_d<ROT>(dL, n, fbc[f], fwn + (idx - (int64_t)F_int * QF) * 3, uinf, g, fvr, idx, dR);
        face_flux_d<ROT>(dL, dR, n, g, fvr, idx, Fd);
        for (int a = 0; a < 5; ++a) fjl[idx * 25 + a * 5 + b] = am * Fd[a].d[0];
    }
}

// A_k = dF_k/dU (closed form, Appendix Eq. dfdu with grad psi -> e_k and omega = 0).
__device__ __forceinline__ void flux_jac_k(const double U[5], double g, int k, double A[25]) {
    const double ir = 1.0 / U[0];
    const double v[3] = {U[1] * ir, U[2] * ir, U[3] * ir};
    const double q2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const double a0 = 0.5 * (g - 1.0) * q2;
    const double p = (g - 1.0) * (U[4] - 0.5 * U[0] * q2);
    const double H = (U[4] + p) * ir;
    const double vk = v[k];
#pragma unroll
    for (int t = 0; t < 25; ++t) A[t] = 0.0;
    A[1 + k] = 1.0;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        double* row = A + 5 * (1 + m);
        row[0] = (m == k ? a0 : 0.0) - v[m] * vk;
#pragma unroll
        for (int l = 0; l < 3; ++l)
            row[1 + l] = (l == k ? v[m] : 0.0) - (m == k ? (g - 1.0) * v[l] : 0.0) + (m == l ? vk : 0.0);
        row[4] = m == k ? (g - 1.0) : 0.0;
    }
    A[20] = (a0 - H) * vk;
#pragma unroll
    for (int l = 0; l < 3; ++l) A[21 + l] = (l == k ? H : 0.0) - (g - 1.0) * v[l] * vk;
    A[24] = g * vk;
}

// The same closed form in float for the FP32 block path.
__device__ __forceinline__ void flux_jac_k(const float U[5], float g, int k, float A[25]) {
    const float ir = 1.0f / U[0];
    const float v[3] = {U[1] * ir, U[2] * ir, U[3] * ir};
    const float q2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const float a0 = 0.5f * (g - 1.0f) * q2;
    const float p = (g - 1.0f) * (U[4] - 0.5f * U[0] * q2);
    const float H = (U[4] + p) * ir;
    const float vk = v[k];
#pragma unroll
    for (int t = 0; t < 25; ++t) A[t] = 0.0f;
    A[1 + k] = 1.0f;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        float* row = A + 5 * (1 + m);
        row[0] = (m == k ? a0 : 0.0f) - v[m] * vk;
#pragma unroll
        for (int l = 0; l < 3; ++l)
            row[1 + l] = (l == k ? v[m] : 0.0f) - (m == k ? (g - 1.0f) * v[l] : 0.0f) + (m == l ? vk : 0.0f);
        row[4] = m == k ? (g - 1.0f) : 0.0f;
    }
    A[20] = (a0 - H) * vk;
#pragma unroll
    for (int l = 0; l < 3; ++l) A[21 + l] = (l == k ? H : 0.0f) - (g - 1.0f) * v[l] * vk;
    A[24] = g * vk;
}

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

emg_status launch_face_jacobian(emg_ctx* c, int p, const double* u) {
    LevelDev& L = c->lv[p];
    const int F = (int)c->F, Fi = (int)c->F_int;
    U5 ui;
    for (int a = 0; a < 5; ++a) ui.v[a] = c->uinf[a];
#define EMG_FJ(DD, PP)                                                                                       \
    {                                                                                                        \
        const int64_t nf = (int64_t)F * Lv<DD, PP>::QF;                                                      \
        ProfScope _ps(c, PC_FACE_JAC);                                                                       \
        if (c->rot)                                                                                          \
            k_face_jac<DD, PP, double, true><<<(unsigned)((nf + 127) / 128), 128, 0, c->stream>>>(           \
                F, Fi, c->face_L, c->face_R, c->face_bc, L.fnrm, L.famag, L.fpsiL, L.fpsiR, L.fwn, u,          \
                c->prm.gamma, ui, L.fvr, L.fjl, L.fjr);                                                      \
        else                                                                                                 \
            k_face_jac<DD, PP, double, false><<<(unsigned)((nf + 127) / 128), 128, 0, c->stream>>>(          \
                F, Fi, c->face_L, c->face_R, c->face_bc, L.fnrm, L.famag, L.fpsiL, L.fpsiR, L.fwn, u,          \
                c->prm.gamma, ui, nullptr, L.fjl, L.fjr);                                                    \
        EMG_CHECK_LAUNCH(c);                                                                                 \
    }
    EMG_DISPATCH_DP(c->dim, p, EMG_FJ)
#undef EMG_FJ
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

emg_status launch_face_jacobian32(emg_ctx* c, int p, const double* u) {
    LevelDev& L = c->lv[p];
    const int F = (int)c->F, Fi = (int)c->F_int;
    U5 ui;
    for (int a = 0; a < 5; ++a) ui.v[a] = c->uinf[a];
#define EMG_FJ32(DD, PP)                                                                                     \
    {                                                                                                        \
        const int64_t nf = (int64_t)F * Lv<DD, PP>::QF;                                                      \
        ProfScope _ps(c, PC_FACE_JAC);                                                                       \
        constexpr int PPB = FaceJacCol<DD, PP, float>::PPB;                                                  \
        const unsigned g1 = (unsigned)((nf + 127) / 128), gc = (unsigned)((nf + PPB - 1) / PPB);             \
        if (c->prm.block_kernels == 3 && c->rot)                                                             \
            k_face_jac<DD, PP, float, true><<<g1, 128, 0, c->stream>>>(                                      \
                F, Fi, c->face_L, c->face_R, c->face_bc, L.fnrm, L.famag, L.fpsiL32, L.fpsiR32, L.fwn, u,      \
                c->prm.gamma, ui, L.fvr, L.fjl32, L.fjr32);                                                  \
        else if (c->prm.block_kernels == 3)                                                                  \
            k_face_jac<DD, PP, float, false><<<g1, 128, 0, c->stream>>>(                                     \
                F, Fi, c->face_L, c->face_R, c->face_bc, L.fnrm, L.famag, L.fpsiL32, L.fpsiR32, L.fwn, u,      \
                c->prm.gamma, ui, nullptr, L.fjl32, L.fjr32);                                                \
        else if (c->rot)                                                                                     \
            k_face_jac_col<DD, PP, float, true><<<gc, 128, 0, c->stream>>>(                                  \
                F, Fi, c->face_L, c->face_R, c->face_bc, L.fnrm, L.famag, L.fpsiL32, L.fpsiR32, L.fwn, u,      \
                c->prm.gamma, ui, L.fvr, L.fjl32, L.fjr32);                                                  \
        else                                                                                                 \
            k_face_jac_col<DD, PP, float, false><<<gc, 128, 0, c->stream>>>(                                 \
                F, Fi, c->face_L, c->face_R, c->face_bc, L.fnrm, L.famag, L.fpsiL32, L.fpsiR32, L.fwn, u,      \
                c->prm.gamma, ui, nullptr, L.fjl32, L.fjr32);                                                \
    }
    EMG_DISPATCH_DP(c->dim, p, EMG_FJ32)
#undef EMG_FJ32
    EMG_CHECK_LAUNCH(c);
    return EMG_OK;
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
    return add_source_jacobian(c, P, shifted, out);
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
    const bool bf = c->prm.prec == EMG_PREC_BF16_BLOCKS;
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
