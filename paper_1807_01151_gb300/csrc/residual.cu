// DG residual R_p(U) of Eq. euler3 with the orthonormal basis (mass matrix = I):
//   R_{e,a,i} = sum_q sum_k W_q d_k psi_i(x_q) F_{k,a}(U_h(x_q))
//             - sum_faces sum_t w|n dS| psi_i(x_t) F~_a(U_in, U_out, n)
// Two kernels: k_face_flux evaluates the Roe flux once per face point (interior faces
// with both traces, boundary faces with the ghost state of Sec. 3.3) and stores
// w|n dS| F~; k_volume does, per element, the volume quadrature and the projection of
// its faces' fluxes (sign -1 on the L side, +1 on the R side: no atomics, deterministic).
// ROT: a frame rotating with angular velocity omega (Eq. euler): the fluxes carry the velocity
// relative to the frame v_r = omega x x (tabulated at the points), F_k - (v_r)_k U, the face
// fluxes move with v_r . n, the ghosts are taken relative to the frame, and the source
// S = (0, -rho omega x v, 0), linear in U, adds -omega x u_{m,i} to the momentum modes (the
// orthonormal basis makes int psi_i S = -omega x (rho v)_i).
#include "common.cuh"
#include "dispatch.cuh"
#include "euler.cuh"

namespace emg {

template <int D, int P, bool ROT>
__global__ void __launch_bounds__(128) k_face_flux(int F, int F_int, const int* __restrict__ fL,
                                                   const int* __restrict__ fR, const int* __restrict__ fbc,
                                                   const double* __restrict__ fnrm,
                                                   const double* __restrict__ famag,
                                                   const double* __restrict__ fpsiL,
                                                   const double* __restrict__ fpsiR,
                                                   const double* __restrict__ fwn,
                                                   const double* __restrict__ u, double g, U5 uinf,
                                                   const double* __restrict__ fvr, double* __restrict__ fhat) {
    using L = Lv<D, P>;
    constexpr int N = L::N, QF = L::QF;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)F * QF) return;
    const int f = (int)(idx / QF);
    const double n[3] = {fnrm[idx * 3], fnrm[idx * 3 + 1], fnrm[idx * 3 + 2]};
    const double* ue = u + (size_t)fL[f] * 5 * N;
    const double* ps = fpsiL + idx * N;
    double UL[5], UR[5], Fl[5];
#pragma unroll
    for (int a = 0; a < 5; ++a) {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < N; ++i) s += ue[a * N + i] * ps[i];
        UL[a] = s;
    }
    if (f < F_int) {
        const double* ur = u + (size_t)fR[f] * 5 * N;
        const double* pr = fpsiR + idx * N;
#pragma unroll
        for (int a = 0; a < 5; ++a) {
            double s = 0.0;
#pragma unroll
            for (int i = 0; i < N; ++i) s += ur[a * N + i] * pr[i];
            UR[a] = s;
        }
    } else if (fbc[f] == EMG_BC_WALL || fbc[f] == EMG_BC_SYMMETRY) {
        // mirror ghost about the reflection normal (body normal on walls, face normal on
        // symmetry planes)
        const int64_t bi = idx - (int64_t)F_int * QF;
        const double nw[3] = {fwn[bi * 3], fwn[bi * 3 + 1], fwn[bi * 3 + 2]};
        if constexpr (ROT) {
            const double vr[3] = {fvr[idx * 3], fvr[idx * 3 + 1], fvr[idx * 3 + 2]};
            wall_ghost_rel(UL, nw, vr, g, UR);
        } else {
            wall_ghost(UL, nw, UR);
        }
    } else {
        if constexpr (ROT) {
            const double vr[3] = {fvr[idx * 3], fvr[idx * 3 + 1], fvr[idx * 3 + 2]};
            farfield_ghost_rel(UL, n, uinf.v, g, vr, UR);
        } else {
            farfield_ghost(UL, n, uinf.v, g, UR);
        }
    }
    if constexpr (ROT) {
        const double vrn = fvr[idx * 3] * n[0] + fvr[idx * 3 + 1] * n[1] + fvr[idx * 3 + 2] * n[2];
        roe_flux<double, true>(UL, UR, n, g, Fl, vrn);
    } else {
        roe_flux(UL, UR, n, g, Fl);
    }
    const double am = famag[idx];
#pragma unroll
    for (int a = 0; a < 5; ++a) fhat[idx * 5 + a] = am * Fl[a];
}

// k_volume: a block holds ET elements.  Thread (element, mode i) accumulates the five
// variables of R_{e,a,i} in registers, so one table value feeds five FMAs.  The point
// fluxes are staged in shared memory QC points at a time (all Q in 2-D; chunks in 3-D),
// so that 3-D elements still fill the block.
template <int D, int P>
struct VolCfg {
    using L = Lv<D, P>;
    static constexpr int THREADS = L::N >= 20 ? 256 : 128;
    static constexpr int ET = THREADS / L::N;                        // elements per block
    static constexpr int FS = 6;                                       // padded variable stride
    static constexpr int QC0 = 36864 / (ET * D * FS * 8);
    static constexpr int QC = P == 0 ? 1 : (QC0 < L::Q ? (QC0 < 1 ? 1 : QC0) : L::Q);   // points per chunk
};

template <int D, int P, bool ROT>
__global__ void __launch_bounds__(VolCfg<D, P>::THREADS) k_volume(
    int E, const double* __restrict__ u, const double* __restrict__ vpsi, const double* __restrict__ vgw,
    const int* __restrict__ elem_face, const double* __restrict__ fpsiL, const double* __restrict__ fpsiR,
    const double* __restrict__ fhat, const double* __restrict__ tau, double g, const double* __restrict__ vvr,
    U5 om, double* __restrict__ R) {
    using L = Lv<D, P>;
    using CF = VolCfg<D, P>;
    constexpr int N = L::N, Q = L::Q, QF = L::QF, B = L::B, NF = L::NF;
    constexpr int ET = CF::ET, QC = CF::QC, FS = CF::FS, T = CF::THREADS;
    __shared__ double us[ET][B];
    __shared__ __align__(16) double Fs[ET][QC][D][FS];
    const int e0 = blockIdx.x * ET;
    for (int t = threadIdx.x; t < ET * B; t += T) {
        const int el = t / B, r = t % B, e = e0 + el;
        us[el][r] = e < E ? u[(size_t)e * B + r] : 0.0;
    }
    const int el2 = threadIdx.x / N, i2 = threadIdx.x % N;   // this thread's (element, mode)
    const int e2 = e0 + el2;
    const bool own = el2 < ET && e2 < E;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (P > 0) {
        for (int q0 = 0; q0 < Q; q0 += QC) {
            const int nq = (Q - q0) < QC ? (Q - q0) : QC;
            __syncthreads();   // us staged / previous chunk consumed
            // (1) U_h and the Euler flux at the chunk's points
            for (int t = threadIdx.x; t < ET * nq; t += T) {
                const int el = t / nq, qq = t % nq, e = e0 + el;
                if (e >= E) continue;
                const double* ps = vpsi + ((size_t)e * Q + q0 + qq) * N;
                double U[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    const double w = ps[i];
#pragma unroll
                    for (int a = 0; a < 5; ++a) U[a] += us[el][a * N + i] * w;
                }
                double Fk[3][5];
                flux_k(U, g, Fk);
                if constexpr (ROT) {   // F_k - (v_r)_k U
                    const double* vr = vvr + ((size_t)e * Q + q0 + qq) * 3;
#pragma unroll
                    for (int k = 0; k < D; ++k)
#pragma unroll
                        for (int a = 0; a < 5; ++a) Fk[k][a] -= vr[k] * U[a];
                }
#pragma unroll
                for (int k = 0; k < D; ++k)
#pragma unroll
                    for (int a = 0; a < 5; ++a) Fs[el][qq][k][a] = Fk[k][a];
            }
            __syncthreads();
            // (2) projection on the gradients: acc_a += sum_q sum_k W_q d_k psi_i F_k,a
            if (own) {
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const double* gw = vgw + (((size_t)e2 * D + k) * Q + q0) * N + i2;
#pragma unroll 4
                    for (int qq = 0; qq < nq; ++qq) {
                        const double w = gw[(size_t)qq * N];
                        const double* f = Fs[el2][qq][k];
                        const double2 f01 = *reinterpret_cast<const double2*>(f);
                        const double2 f23 = *reinterpret_cast<const double2*>(f + 2);
                        acc[0] += w * f01.x;
                        acc[1] += w * f01.y;
                        acc[2] += w * f23.x;
                        acc[3] += w * f23.y;
                        acc[4] += w * f[4];
                    }
                }
            }
        }
    }
    if (!own) return;
    // (3) faces: -(L side) / +(R side) sum_t psi_i(x_t) w|n dS| F~_a
#pragma unroll
    for (int lf = 0; lf < NF; ++lf) {
        const int code = elem_face[(size_t)e2 * NF + lf];
        const int f = code >> 1;
        const double* ps = ((code & 1) ? fpsiR : fpsiL) + (size_t)f * QF * N + i2;
        const double* fh = fhat + (size_t)f * QF * 5;
        double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll 2
        for (int t2 = 0; t2 < QF; ++t2) {
            const double w = ps[(size_t)t2 * N];
#pragma unroll
            for (int a = 0; a < 5; ++a) s[a] += w * fh[t2 * 5 + a];
        }
        const double sg = (code & 1) ? 1.0 : -1.0;
#pragma unroll
        for (int a = 0; a < 5; ++a) acc[a] += sg * s[a];
    }
    if constexpr (ROT) {   // source: -omega x (rho v)_i
        const double mx = us[el2][1 * N + i2], my = us[el2][2 * N + i2], mz = us[el2][3 * N + i2];
        acc[1] -= om.v[1] * mz - om.v[2] * my;
        acc[2] -= om.v[2] * mx - om.v[0] * mz;
        acc[3] -= om.v[0] * my - om.v[1] * mx;
    }
    double* Re = R + (size_t)e2 * B + i2;
    const double* te = tau ? tau + (size_t)e2 * B + i2 : nullptr;
#pragma unroll
    for (int a = 0; a < 5; ++a) Re[a * N] = te ? acc[a] + te[a * N] : acc[a];
}

emg_status launch_residual(emg_ctx* c, int p, const double* u, const double* tau, double* R) {
    LevelDev& L = c->lv[p];
    const int F = (int)c->F, Fi = (int)c->F_int, E = (int)c->E;
    U5 ui;
    for (int a = 0; a < 5; ++a) ui.v[a] = c->uinf[a];
    const double g = c->prm.gamma;
    U5 om{};
    for (int k = 0; k < 3; ++k) om.v[k] = c->prm.omega[k];
#define EMG_RES_ROT(DD, PP, RR)                                                                                 \
    {                                                                                                          \
        const int64_t nf = (int64_t)F * Lv<DD, PP>::QF;                                                        \
        { ProfScope _ps(c, PC_RES_FACE); k_face_flux<DD, PP, RR><<<(unsigned)((nf + 127) / 128), 128, 0, c->stream>>>( \
            F, Fi, c->face_L, c->face_R, c->face_bc, L.fnrm, L.famag, L.fpsiL, L.fpsiR, L.fwn, u, g, ui, L.fvr,     \
            L.fhat); }                                                                                         \
        EMG_CHECK_LAUNCH(c);                                                                                   \
        constexpr int ET = VolCfg<DD, PP>::ET;                                                                 \
        { ProfScope _ps(c, PC_RES_VOL); k_volume<DD, PP, RR><<<(unsigned)((E + ET - 1) / ET), VolCfg<DD, PP>::THREADS, 0, \
            c->stream>>>(E, u, L.vpsi, L.vgw, c->elem_face, L.fpsiL, L.fpsiR, L.fhat, tau, g, L.vvr, om, R); }      \
        EMG_CHECK_LAUNCH(c);                                                                                   \
    }
#define EMG_RES(DD, PP)                   \
    if (c->rot)                           \
        EMG_RES_ROT(DD, PP, true)         \
    else                                  \
        EMG_RES_ROT(DD, PP, false)
    EMG_DISPATCH_DP(c->dim, p, EMG_RES)
#undef EMG_RES
#undef EMG_RES_ROT
    return EMG_OK;
}

}  // namespace emg
