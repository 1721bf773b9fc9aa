// Level transfer and control kernels of the V-cycle (Sec. 2.3, Sec. 4):
//  * restriction = truncation to the first N_{p-1} modes of the hierarchical orthonormal
//    basis; FAS forcing tau_{p-1} = trunc(R~_p(v_p)) - R_{p-1}(trunc(v_p));
//    prolongation = zero padding, v_p += P(v_{p-1} - v0_{p-1});
//  * ||R(rho)|| of Eq. cfl from the p_max residual coefficients (orthonormal basis:
//    int R^2 = sum of squared coefficients) and CFL_n of Eq. cfl, on the device;
//  * dtau_e of Eq. x3d from the state at the cell centre.
#include "common.cuh"

namespace emg {

__global__ void k_restrict(int64_t E, int Nf, int Nc, const double* __restrict__ f, double* __restrict__ c) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= E * 5 * Nc) return;
    const int64_t ea = idx / Nc;
    const int i = (int)(idx % Nc);
    c[idx] = f[ea * Nf + i];
}

__global__ void k_tau(int64_t E, int Nf, int Nc, const double* __restrict__ rf, const double* __restrict__ rc,
                      double* __restrict__ tau) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= E * 5 * Nc) return;
    const int64_t ea = idx / Nc;
    const int i = (int)(idx % Nc);
    tau[idx] = rf[ea * Nf + i] - rc[idx];
}

__global__ void k_prolong(int64_t E, int Nf, int Nc, double* __restrict__ f, const double* __restrict__ vc,
                          const double* __restrict__ v0c) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= E * 5 * Nc) return;
    const int64_t ea = idx / Nc;
    const int i = (int)(idx % Nc);
    f[ea * Nf + i] += vc[idx] - v0c[idx];
}

__global__ void k_axpby(int64_t n, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                        double* __restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) out[idx] = a * x[idx] + b * y[idx];
}

constexpr int NORM_THREADS = 256;

// Per-block partial sums of squared residual coefficients, per variable.
__global__ void k_norm_partial(int64_t E, int N, const double* __restrict__ R, double* __restrict__ partial) {
    __shared__ double sh[NORM_THREADS / 32][5];
    double acc[5] = {0, 0, 0, 0, 0};
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < E * 5 * N; t += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)((t / N) % 5);
        const double v = R[t];
        acc[a] += v * v;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int a = 0; a < 5; ++a) {
        double v = acc[a];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[warp][a] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double s = 0.0;
        for (int w = 0; w < NORM_THREADS / 32; ++w) s += sh[w][threadIdx.x];
        partial[blockIdx.x * 5 + threadIdx.x] = s;
    }
}

__global__ void k_norm_final(int nb, const double* __restrict__ partial, double inv_vol, int p_max,
                             double cfl_max, int update_cfl, DevScalars* sc) {
    if (threadIdx.x != 0) return;
    double s[5] = {0, 0, 0, 0, 0};
    for (int b = 0; b < nb; ++b)
        for (int a = 0; a < 5; ++a) s[a] += partial[b * 5 + a];
    for (int a = 0; a < 5; ++a) sc->res5[a] = sqrt(s[a]) * inv_vol;
    const double res = sc->res5[0];
    sc->res = res;
    bool bad = false;
    for (int a = 0; a < 5; ++a) bad |= !isfinite(s[a]);
    if (bad) sc->nonfinite = 1;
    if (update_cfl) {
        if (!(sc->res_ref > 0.0)) sc->res_ref = res;
        const double ramp = 1.0 + (double)(sc->cycle - 1) / (2 * p_max + 1);
        const double inv = res > 0.0 ? sc->res_ref / res : INFINITY;
        sc->cfl = fmin(cfl_max, fmax(inv, ramp));
    }
}

// dt_e = factor * CFL h_e / ((2p+1)(|v|+c)) at the cell centre; flags non-positive rho or p.
__global__ void k_dtau(int64_t E, int N, int nmax, const double* __restrict__ u, const double* __restrict__ psic,
                       const double* __restrict__ h, const double* __restrict__ cfl_dev, int p, double factor,
                       double g, double* __restrict__ dt, DevScalars* sc) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    double U[5];
    for (int a = 0; a < 5; ++a) {
        double s = 0.0;
        for (int i = 0; i < N; ++i) s += u[(e * 5 + a) * N + i] * psic[e * nmax + i];
        U[a] = s;
    }
    const double ir = 1.0 / U[0];
    const double vx = U[1] * ir, vy = U[2] * ir, vz = U[3] * ir;
    const double q2 = vx * vx + vy * vy + vz * vz;
    const double pr = (g - 1.0) * (U[4] - 0.5 * U[0] * q2);
    if (!(U[0] > 0.0) || !(pr > 0.0)) sc->pad = 1;
    const double c = sqrt(g * pr * ir);
    dt[e] = factor * cfl_dev[0] * h[e] / ((2 * p + 1) * (sqrt(q2) + c));
}

// dt_e <- min_e dt_e for every element (one block; the minimum does not depend on the
// order of the comparisons).  A NaN step stays NaN.
__global__ void k_dt_global(int64_t E, double* __restrict__ dt) {
    __shared__ double sh[32];
    double m = INFINITY;
    bool nan = false;
    for (int64_t e = threadIdx.x; e < E; e += blockDim.x) {
        const double v = dt[e];
        nan |= isnan(v);
        m = fmin(m, v);
    }
    nan = __syncthreads_or(nan);
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        double x = threadIdx.x < blockDim.x / 32 ? sh[threadIdx.x] : INFINITY;
        for (int o = 16; o > 0; o >>= 1) x = fmin(x, __shfl_xor_sync(0xffffffffu, x, o));
        if (threadIdx.x == 0) sh[0] = nan ? NAN : x;
    }
    __syncthreads();
    const double g = sh[0];
    for (int64_t e = threadIdx.x; e < E; e += blockDim.x) dt[e] = g;
}

__global__ void k_check_finite(int64_t n, const double* __restrict__ u, DevScalars* sc) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n && !isfinite(u[idx])) sc->nonfinite = 1;
}

static unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

emg_status launch_restrict(emg_ctx* c, int p_fine, const double* fine, double* coarse) {
    const int Nf = c->lv[p_fine].N, Nc = c->lv[p_fine - 1].N;
    const int64_t n = c->E * 5 * Nc;
    { ProfScope _ps(c, PC_TRANSFER); k_restrict<<<blocks_for(n, 256), 256, 0, c->stream>>>(c->E, Nf, Nc, fine, coarse); }
    EMG_CHECK_LAUNCH(c);
    return EMG_OK;
}

emg_status launch_tau(emg_ctx* c, int p_coarse, const double* rfine, const double* rcoarse, double* tau) {
    const int Nf = c->lv[p_coarse + 1].N, Nc = c->lv[p_coarse].N;
    const int64_t n = c->E * 5 * Nc;
    { ProfScope _ps(c, PC_TRANSFER); k_tau<<<blocks_for(n, 256), 256, 0, c->stream>>>(c->E, Nf, Nc, rfine, rcoarse, tau); }
    EMG_CHECK_LAUNCH(c);
    return EMG_OK;
}

emg_status launch_prolong(emg_ctx* c, int p_fine, double* fine, const double* vc, const double* v0c) {
    const int Nf = c->lv[p_fine].N, Nc = c->lv[p_fine - 1].N;
    const int64_t n = c->E * 5 * Nc;
    { ProfScope _ps(c, PC_TRANSFER); k_prolong<<<blocks_for(n, 256), 256, 0, c->stream>>>(c->E, Nf, Nc, fine, vc, v0c); }
    EMG_CHECK_LAUNCH(c);
    return EMG_OK;
}

emg_status launch_axpby(emg_ctx* c, int64_t n, double a, const double* x, double b, const double* y, double* out) {
    { ProfScope _ps(c, PC_TRANSFER); k_axpby<<<blocks_for(n, 256), 256, 0, c->stream>>>(n, a, x, b, y, out); }
    EMG_CHECK_LAUNCH(c);
    return EMG_OK;
}

emg_status launch_norm_cfl(emg_ctx* c, const double* R, int update_cfl) {
    const int nb = 152;
    { ProfScope _ps(c, PC_CONTROL); k_norm_partial<<<nb, NORM_THREADS, 0, c->stream>>>(c->E, c->lv[c->p_max].N, R, c->partial); }
    EMG_CHECK_LAUNCH(c);
    { ProfScope _ps(c, PC_CONTROL); k_norm_final<<<1, 32, 0, c->stream>>>(nb, c->partial, 1.0 / c->domain_volume, c->p_max, c->prm.cfl_max,
                                          update_cfl, c->sc); }
    EMG_CHECK_LAUNCH(c);
    return EMG_OK;
}

emg_status launch_dtau(emg_ctx* c, int p, const double* u, const double* cfl_dev, double factor, double* dt) {
    const int nmax = n_modes(c->dim, c->p_max);
    { ProfScope _ps(c, PC_CONTROL); k_dtau<<<blocks_for(c->E, 128), 128, 0, c->stream>>>(c->E, c->lv[p].N, nmax, u, c->psic, c->h, cfl_dev, p, factor,
                                                         c->prm.gamma, dt, c->sc); }
    EMG_CHECK_LAUNCH(c);
    return EMG_OK;
}

emg_status launch_dt_global(emg_ctx* c, double* dt) {
    { ProfScope _ps(c, PC_CONTROL); k_dt_global<<<1, 1024, 0, c->stream>>>(c->E, dt); }
    EMG_CHECK_LAUNCH(c);
    return EMG_OK;
}

emg_status launch_check_state(emg_ctx* c, const double* u, int64_t n) {
    { ProfScope _ps(c, PC_CONTROL); k_check_finite<<<blocks_for(n, 256), 256, 0, c->stream>>>(n, u, c->sc); }
    EMG_CHECK_LAUNCH(c);
    return EMG_OK;
}

}  // namespace emg
