// Face Jacobians of the exact Jacobian blocks (Sec. 3.3): k_face_jac, per face point,
// dF~/dU_L and dF~/dU_R of the Roe flux by forward-mode AD (Dual<5>); on boundary faces the
// total derivative through the ghost state, dF~/dU_L + dF~/dU_ghost dU_ghost/dU_L;
// k_face_jac_col the same, one derivative direction per thread.  Instantiated for FP64 in
// jac_face.cu and for float32 in jac_face32.cu (2-D) and jac_face32_3d.cu (3-D).
#pragma once

#include "common.cuh"
#include "dispatch.cuh"
#include "euler.cuh"

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

// Launch of the float32 face Jacobians of level P in dimension D (the kernel form chosen by
// block_kernels and the rotating frame); the caller checks the launch.
template <int D, int P>
void face_jacobian32_go(emg_ctx* c, const double* u) {
    LevelDev& L = c->lv[P];
    const int F = (int)c->F, Fi = (int)c->F_int;
    U5 ui;
    for (int a = 0; a < 5; ++a) ui.v[a] = c->uinf[a];
    const int64_t nf = (int64_t)F * Lv<D, P>::QF;
    ProfScope _ps(c, PC_FACE_JAC);
    constexpr int PPB = FaceJacCol<D, P, float>::PPB;
    const unsigned g1 = (unsigned)((nf + 127) / 128), gc = (unsigned)((nf + PPB - 1) / PPB);
    if (c->prm.block_kernels == 3 && c->rot)
        k_face_jac<D, P, float, true><<<g1, 128, 0, c->stream>>>(
            F, Fi, c->face_L, c->face_R, c->face_bc, L.fnrm, L.famag, L.fpsiL32, L.fpsiR32, L.fwn, u,
            c->prm.gamma, ui, L.fvr, L.fjl32, L.fjr32);
    else if (c->prm.block_kernels == 3)
        k_face_jac<D, P, float, false><<<g1, 128, 0, c->stream>>>(
            F, Fi, c->face_L, c->face_R, c->face_bc, L.fnrm, L.famag, L.fpsiL32, L.fpsiR32, L.fwn, u,
            c->prm.gamma, ui, nullptr, L.fjl32, L.fjr32);
    else if (c->rot)
        k_face_jac_col<D, P, float, true><<<gc, 128, 0, c->stream>>>(
            F, Fi, c->face_L, c->face_R, c->face_bc, L.fnrm, L.famag, L.fpsiL32, L.fpsiR32, L.fwn, u,
            c->prm.gamma, ui, L.fvr, L.fjl32, L.fjr32);
    else
        k_face_jac_col<D, P, float, false><<<gc, 128, 0, c->stream>>>(
            F, Fi, c->face_L, c->face_R, c->face_bc, L.fnrm, L.famag, L.fpsiL32, L.fpsiR32, L.fwn, u,
            c->prm.gamma, ui, nullptr, L.fjl32, L.fjr32);
}

}  // namespace emg
