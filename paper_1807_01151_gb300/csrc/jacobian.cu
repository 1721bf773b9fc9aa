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

#include "common.cuh"
#include "dispatch.cuh"
#include "euler.cuh"

namespace emg {

template <int D, int P, class S>
__global__ void __launch_bounds__(128) k_face_jac(int F, int F_int, const int* __restrict__ fL,
                                                  const int* __restrict__ fR, const int* __restrict__ fbc,
                                                  const double* __restrict__ fnrm,
                                                  const double* __restrict__ famag,
                                                  const S* __restrict__ fpsiL,
                                                  const S* __restrict__ fpsiR,
                                                  const double* __restrict__ fwn,
                                                  const double* __restrict__ u, double g, U5 uinf,
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
        roe_flux(dL, dR, n, g, Fd);
        for (int a = 0; a < 5; ++a)
            for (int b = 0; b < 5; ++b) fjl[idx * 25 + a * 5 + b] = am * Fd[a].d[b];
        Dual<5, S> cL[5];
        for (int a = 0; a < 5; ++a) {
            cL[a] = dconst<5, S>(UL[a]);
            dR[a].d[a] = (S)1;
        }
        roe_flux(cL, dR, n, g, Fd);
        for (int a = 0; a < 5; ++a)
            for (int b = 0; b < 5; ++b) fjr[idx * 25 + a * 5 + b] = am * Fd[a].d[b];
    } else {
        if (fbc[f] == EMG_BC_WALL || fbc[f] == EMG_BC_SYMMETRY) {
            const int64_t bi = idx - (int64_t)F_int * QF;
            const double nw[3] = {fwn[bi * 3], fwn[bi * 3 + 1], fwn[bi * 3 + 2]};
            wall_ghost(dL, nw, dR);
        } else {
            farfield_ghost(dL, n, uinf.v, g, dR);
        }
        roe_flux(dL, dR, n, g, Fd);
        for (int a = 0; a < 5; ++a)
            for (int b = 0; b < 5; ++b) fjl[idx * 25 + a * 5 + b] = am * Fd[a].d[b];
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
    T* __restrict__ out) {
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
            for (int t = tid; t < nq * D; t += blockDim.x) flux_jac_k(Us[t / D], (T)g, t % D, As[t / D][t % D]);
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

emg_status launch_face_jacobian(emg_ctx* c, int p, const double* u) {
    LevelDev& L = c->lv[p];
    const int F = (int)c->F, Fi = (int)c->F_int;
    U5 ui;
    for (int a = 0; a < 5; ++a) ui.v[a] = c->uinf[a];
#define EMG_FJ(DD, PP)                                                                                       \
    {                                                                                                        \
        const int64_t nf = (int64_t)F * Lv<DD, PP>::QF;                                                      \
        { ProfScope _ps(c, PC_FACE_JAC); k_face_jac<DD, PP, double><<<(unsigned)((nf + 127) / 128), 128, 0, c->stream>>>(                             \
            F, Fi, c->face_L, c->face_R, c->face_bc, L.fnrm, L.famag, L.fpsiL, L.fpsiR, L.fwn, u, c->prm.gamma, ui, \
            L.fjl, L.fjr); }                                                                                   \
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
            cfl_dev, c->prm.gamma, shifted, out);                                                           \
    }
    EMG_DISPATCH_DP(c->dim, p, EMG_DB)
#undef EMG_DB
    EMG_CHECK_LAUNCH(c);
    return EMG_OK;
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
        k_face_jac<DD, PP, float><<<(unsigned)((nf + 127) / 128), 128, 0, c->stream>>>(                      \
            F, Fi, c->face_L, c->face_R, c->face_bc, L.fnrm, L.famag, L.fpsiL32, L.fpsiR32, L.fwn, u,          \
            c->prm.gamma, ui, L.fjl32, L.fjr32);                                                             \
    }
    EMG_DISPATCH_DP(c->dim, p, EMG_FJ32)
#undef EMG_FJ32
    EMG_CHECK_LAUNCH(c);
    return EMG_OK;
}

emg_status launch_diag_blocks32(emg_ctx* c, int p, const double* u, const double* cfl_dev, int shifted,
                                float* out) {
    emg_status st = launch_face_jacobian32(c, p, u);
    if (st != EMG_OK) return st;
    LevelDev& L = c->lv[p];
    if (!L.vpsi32) {
        c->err = "FP32 tables not built";
        return EMG_ERR_ARG;
    }
    const int nmax = n_modes(c->dim, c->p_max);
#define EMG_DB32(DD, PP)                                                                                    \
    {                                                                                                       \
        ProfScope _ps(c, PC_DIAG);                                                                          \
        k_diag_blocks<DD, PP, float><<<(unsigned)c->E, DiagCfg<DD, PP>::THREADS, 0, c->stream>>>(           \
            (int)c->E, nmax, u, L.vpsi32, L.vgw32, c->elem_face, L.fpsiL32, L.fpsiR32, L.fjl32, L.fjr32, c->psic, \
            c->h, cfl_dev, c->prm.gamma, shifted, out);                                                     \
    }
    EMG_DISPATCH_DP(c->dim, p, EMG_DB32)
#undef EMG_DB32
    EMG_CHECK_LAUNCH(c);
    return EMG_OK;
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
    return EMG_OK;
}

}  // namespace emg
