// DG residual R_p(U) of Eq. euler3 with the orthonormal basis (mass matrix = I):
//   R_{e,a,i} = sum_q sum_k W_q d_k psi_i(x_q) F_{k,a}(U_h(x_q))
//             - sum_faces sum_t w|n dS| psi_i(x_t) F~_a(U_in, U_out, n)
// Two kernels: k_face_flux evaluates the Roe flux once per face point (interior faces
// with both traces, boundary faces with the ghost state of Sec. 3.3) and stores
// w|n dS| F~; k_volume does, per element, the volume quadrature and the projection of
// its faces' fluxes (sign -1 on the L side, +1 on the R side: no atomics, deterministic).
#include "common.cuh"
#include "dispatch.cuh"
#include "euler.cuh"

namespace emg {

template <int D, int P>
__global__ void __launch_bounds__(128) k_face_flux(int F, int F_int, const int* __restrict__ fL,
                                                   const int* __restrict__ fR, const int* __restrict__ fbc,
                                                   const double* __restrict__ fnrm,
                                                   const double* __restrict__ famag,
                                                   const double* __restrict__ fpsiL,
                                                   const double* __restrict__ fpsiR,
                                                   const double* __restrict__ fwn,
                                                   const double* __restrict__ u, double g, U5 uinf,
                                                   double* __restrict__ fhat) {
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
    } else if (fbc[f] == EMG_BC_WALL) {
        {
        const int64_t bi = idx - (int64_t)F_int * QF;
        const double nw[3] = {fwn[bi * 3], fwn[bi * 3 + 1], fwn[bi * 3 + 2]};
        wall_ghost(UL, nw, UR);
    }
    } else {
        farfield_ghost(UL, n, uinf.v, g, UR);
    }
    roe_flux(UL, UR, n, g, Fl);
    const double am = famag[idx];
#pragma unroll
    for (int a = 0; a < 5; ++a) fhat[idx * 5 + a] = am * Fl[a];
}

template <int D, int P>
struct VolCfg {
    using L = Lv<D, P>;
    static constexpr int per = L::Q * D * 5 * 8 + L::B * 8;
    static constexpr int ET = (24576 / per) < 1 ? 1 : ((24576 / per) > 8 ? 8 : (24576 / per));
};

template <int D, int P>
__global__ void __launch_bounds__(128) k_volume(int E, const double* __restrict__ u, const double* __restrict__ vpsi,
                                                const double* __restrict__ vgw, const int* __restrict__ elem_face,
                                                const double* __restrict__ fpsiL, const double* __restrict__ fpsiR,
                                                const double* __restrict__ fhat, const double* __restrict__ tau,
                                                double g, double* __restrict__ R) {
    using L = Lv<D, P>;
    constexpr int N = L::N, Q = L::Q, QF = L::QF, B = L::B, NF = L::NF;
    constexpr int ET = VolCfg<D, P>::ET;
    __shared__ double us[ET][B];
    __shared__ double Fs[ET][Q][D][5];
    const int e0 = blockIdx.x * ET;
    for (int t = threadIdx.x; t < ET * B; t += blockDim.x) {
        const int el = t / B, r = t % B, e = e0 + el;
        us[el][r] = e < E ? u[(size_t)e * B + r] : 0.0;
    }
    __syncthreads();
    if (P > 0) {
        for (int t = threadIdx.x; t < ET * Q; t += blockDim.x) {
            const int el = t / Q, q = t % Q, e = e0 + el;
            if (e >= E) continue;
            const double* ps = vpsi + ((size_t)e * Q + q) * N;
            double U[5];
#pragma unroll
            for (int a = 0; a < 5; ++a) {
                double s = 0.0;
#pragma unroll
                for (int i = 0; i < N; ++i) s += us[el][a * N + i] * ps[i];
                U[a] = s;
            }
            double Fk[3][5];
            flux_k(U, g, Fk);
#pragma unroll
            for (int k = 0; k < D; ++k)
#pragma unroll
                for (int a = 0; a < 5; ++a) Fs[el][q][k][a] = Fk[k][a];
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < ET * B; t += blockDim.x) {
        const int el = t / B, r = t % B, e = e0 + el;
        if (e >= E) continue;
        const int a = r / N, i = r % N;
        double acc = 0.0;
        if (P > 0) {
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const double* gw = vgw + (((size_t)e * D + k) * Q) * N + i;
#pragma unroll 4
                for (int q = 0; q < Q; ++q) acc += gw[(size_t)q * N] * Fs[el][q][k][a];
            }
        }
#pragma unroll
        for (int lf = 0; lf < NF; ++lf) {
            const int code = elem_face[(size_t)e * NF + lf];
            const int f = code >> 1;
            const double* ps = (code & 1) ? fpsiR : fpsiL;
            double s = 0.0;
#pragma unroll
            for (int t2 = 0; t2 < QF; ++t2)
                s += ps[((size_t)f * QF + t2) * N + i] * fhat[((size_t)f * QF + t2) * 5 + a];
            acc += (code & 1) ? s : -s;
        }
        if (tau) acc += tau[(size_t)e * B + r];
        R[(size_t)e * B + r] = acc;
    }
}

emg_status launch_residual(emg_ctx* c, int p, const double* u, const double* tau, double* R) {
    LevelDev& L = c->lv[p];
    const int F = (int)c->F, Fi = (int)c->F_int, E = (int)c->E;
    U5 ui;
    for (int a = 0; a < 5; ++a) ui.v[a] = c->uinf[a];
    const double g = c->prm.gamma;
#define EMG_RES(DD, PP)                                                                                        \
    {                                                                                                          \
        const int64_t nf = (int64_t)F * Lv<DD, PP>::QF;                                                        \
        { ProfScope _ps(c, PC_RES_FACE); k_face_flux<DD, PP><<<(unsigned)((nf + 127) / 128), 128, 0, c->stream>>>(                              \
            F, Fi, c->face_L, c->face_R, c->face_bc, L.fnrm, L.famag, L.fpsiL, L.fpsiR, L.fwn, u, g, ui, L.fhat); }     \
        EMG_CHECK_LAUNCH(c);                                                                                   \
        constexpr int ET = VolCfg<DD, PP>::ET;                                                                 \
        { ProfScope _ps(c, PC_RES_VOL); k_volume<DD, PP><<<(unsigned)((E + ET - 1) / ET), 128, 0, c->stream>>>(                                \
            E, u, L.vpsi, L.vgw, c->elem_face, L.fpsiL, L.fpsiR, L.fhat, tau, g, R); }                           \
        EMG_CHECK_LAUNCH(c);                                                                                   \
    }
    EMG_DISPATCH_DP(c->dim, p, EMG_RES)
#undef EMG_RES
    return EMG_OK;
}

}  // namespace emg
