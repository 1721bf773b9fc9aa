// Mesh set-up: face matching (host), then on the device the element geometry
// (|E|, x_c, half bounding box L, |dE|, h = 2d|E|/|dE|; Sec. 3.2 and Eq. x3d), the
// orthonormal Cartesian basis by modified Gram-Schmidt (Eqs. basis2, basis) and the
// quadrature tables of every level.  Quadrature: tensor Gauss-Legendre, q = p + 2
// points per direction, so that psi_i psi_j det J is integrated exactly on bilinear
// and trilinear elements.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "dispatch.cuh"

namespace emg {

// ---- reference element -----------------------------------------------------------------
// Node a of the reference quad/hex: (-1,-1),(1,-1),(1,1),(-1,1) [then the same at zeta=+1].
__host__ __device__ __forceinline__ double ref_coord(int a, int k) {
    const int a4 = a & 3;
    if (k == 0) return (a4 == 1 || a4 == 2) ? 1.0 : -1.0;
    if (k == 1) return (a4 >= 2) ? 1.0 : -1.0;
    return (a >= 4) ? 1.0 : -1.0;
}

// x(xi) and J = dx/dxi of element with node coordinates X[a][D].
template <int D>
__device__ __forceinline__ void map_point(const double* X, const double xi[D], double x[D], double J[D][D]) {
    for (int i = 0; i < D; ++i) {
        x[i] = 0.0;
        for (int k = 0; k < D; ++k) J[i][k] = 0.0;
    }
    for (int a = 0; a < (1 << D); ++a) {
        double fac[D];
        for (int d = 0; d < D; ++d) fac[d] = 0.5 * (1.0 + xi[d] * ref_coord(a, d));
        double Na = 1.0;
        for (int d = 0; d < D; ++d) Na *= fac[d];
        for (int k = 0; k < D; ++k) {
            double dN = 0.5 * ref_coord(a, k);
            for (int d = 0; d < D; ++d)
                if (d != k) dN *= fac[d];
            for (int i = 0; i < D; ++i) J[i][k] += dN * X[a * D + i];
        }
        for (int i = 0; i < D; ++i) x[i] += Na * X[a * D + i];
    }
}

template <int D>
__device__ __forceinline__ double det_of(const double J[D][D]) {
    if (D == 2) return J[0][0] * J[1][1] - J[0][1] * J[1][0];
    return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

// Column k of cof(J) = det(J) J^-T (the area vector of the face xi_k = const per unit
// reference area, before the side sign).
template <int D>
__device__ __forceinline__ void cof_col(const double J[D][D], int k, double a[3]) {
    a[2] = 0.0;
    if (D == 2) {
        if (k == 0) {
            a[0] = J[1][1];
            a[1] = -J[0][1];
        } else {
            a[0] = -J[1][0];
            a[1] = J[0][0];
        }
        return;
    }
    const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
    a[0] = J[1][k1] * J[2][k2] - J[2][k1] * J[1][k2];
    a[1] = J[2][k1] * J[0][k2] - J[0][k1] * J[2][k2];
    a[2] = J[0][k1] * J[1][k2] - J[1][k1] * J[0][k2];
}

// Reference point of volume point index t (axis 0 fastest) and its weight.
template <int D>
__device__ __forceinline__ double vol_point(const double* gl, int q, int t, double xi[D]) {
    const double* x = gl + q * 16;
    const double* w = x + 8;
    double wt = 1.0;
    for (int d = 0; d < D; ++d) {
        const int i = t % q;
        t /= q;
        xi[d] = x[i];
        wt *= w[i];
    }
    return wt;
}

// Reference point of point t on local face f (the lower remaining axis fastest).
template <int D>
__device__ __forceinline__ double face_point(const double* gl, int q, int f, int t, double xi[D]) {
    const double* x = gl + q * 16;
    const double* w = x + 8;
    const int axis = f >> 1;
    xi[axis] = (f & 1) ? 1.0 : -1.0;
    double wt = 1.0;
    for (int d = 0; d < D; ++d) {
        if (d == axis) continue;
        const int i = t % q;
        t /= q;
        xi[d] = x[i];
        wt *= w[i];
    }
    return wt;
}

// ---- geometry: one thread per element ------------------------------------------------------
template <int D>
__global__ void k_geometry(int E, const double* __restrict__ ex, const double* __restrict__ gl, int q,
                           double* vol, double* xc, double* Lh, double* surf, double* h) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const double* X = ex + (size_t)e * (1 << D) * D;
    int Q = 1;
    for (int d = 0; d < D; ++d) Q *= q;
    double V = 0.0, xs[D];
    for (int d = 0; d < D; ++d) xs[d] = 0.0;
    for (int t = 0; t < Q; ++t) {
        double xi[D], x[D], J[D][D];
        const double w = vol_point<D>(gl, q, t, xi);
        map_point<D>(X, xi, x, J);
        const double W = w * det_of<D>(J);
        V += W;
        for (int d = 0; d < D; ++d) xs[d] += W * x[d];
    }
    double S = 0.0;
    const int QF = Q / q;
    for (int f = 0; f < 2 * D; ++f) {
        for (int t = 0; t < QF; ++t) {
            double xi[D], x[D], J[D][D], a[3];
            const double w = face_point<D>(gl, q, f, t, xi);
            map_point<D>(X, xi, x, J);
            cof_col<D>(J, f >> 1, a);
            S += w * sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        }
    }
    vol[e] = V;
    surf[e] = S;
    h[e] = 2.0 * D * V / S;
    for (int d = 0; d < 3; ++d) {
        xc[e * 3 + d] = d < D ? xs[d] / V : 0.0;
        double lo = 1e300, hi = -1e300;
        if (d < D)
            for (int a = 0; a < (1 << D); ++a) {
                lo = fmin(lo, X[a * D + d]);
                hi = fmax(hi, X[a * D + d]);
            }
        Lh[e * 3 + d] = d < D ? 0.5 * (hi - lo) : 1.0;
    }
}

// Scaled monomials chi_k and gradients at x; exps[k][3] in the basis order.
template <int D, int NM>
__device__ __forceinline__ void monomials(const double x[D], const double* xc, const double* L,
                                          const int* __restrict__ exps, int n, double chi[NM],
                                          double grad[NM][D]) {
    double s[D], pw[D][MAX_P + 1];
    for (int d = 0; d < D; ++d) {
        s[d] = (x[d] - xc[d]) / L[d];
        pw[d][0] = 1.0;
        for (int a = 1; a <= MAX_P; ++a) pw[d][a] = pw[d][a - 1] * s[d];
    }
    for (int k = 0; k < n; ++k) {
        double c = 1.0;
        for (int d = 0; d < D; ++d) c *= pw[d][exps[k * 3 + d]];
        chi[k] = c;
        for (int g = 0; g < D; ++g) {
            const int eg = exps[k * 3 + g];
            double v = eg > 0 ? eg * pw[g][eg - 1] / L[g] : 0.0;
            for (int d = 0; d < D; ++d)
                if (d != g) v *= pw[d][exps[k * 3 + d]];
            grad[k][g] = v;
        }
    }
}

// ---- basis: modified Gram-Schmidt, one warp per element --------------------------------
// Inner product <f, g> = sum_q W_q f(x_q) g(x_q) on the p_max volume rule.
template <int D, int NM>
__global__ void k_basis(int E, int n, int q, const double* __restrict__ ex, const double* __restrict__ gl,
                        const double* __restrict__ xc, const double* __restrict__ Lh, const int* __restrict__ exps,
                        double* C, double* psic) {
    extern __shared__ double sm[];
    const int e = blockIdx.x;
    const int lane = threadIdx.x;
    int Q = 1;
    for (int d = 0; d < D; ++d) Q *= q;
    double* ps = sm;               // [n][Q]
    double* W = ps + n * Q;        // [Q]
    double* Cs = W + Q;            // [n][n]
    const double* X = ex + (size_t)e * (1 << D) * D;
    for (int t = lane; t < Q; t += 32) {
        double xi[D], x[D], J[D][D], chi[NM], g[NM][D];
        const double w = vol_point<D>(gl, q, t, xi);
        map_point<D>(X, xi, x, J);
        W[t] = w * det_of<D>(J);
        monomials<D, NM>(x, xc + e * 3, Lh + e * 3, exps, n, chi, g);
        for (int k = 0; k < n; ++k) ps[k * Q + t] = chi[k];
    }
    for (int t = lane; t < n * n; t += 32) Cs[t] = 0.0;
    __syncwarp();
    for (int i = 0; i < n; ++i) {
        if (lane == 0) Cs[i * n + i] = 1.0;
        __syncwarp();
        for (int j = 0; j < i; ++j) {
            double r = 0.0;
            for (int t = lane; t < Q; t += 32) r += W[t] * ps[i * Q + t] * ps[j * Q + t];
            for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
            for (int t = lane; t < Q; t += 32) ps[i * Q + t] -= r * ps[j * Q + t];
            for (int k = lane; k <= j; k += 32) Cs[i * n + k] -= r * Cs[j * n + k];
            __syncwarp();
        }
        double s = 0.0;
        for (int t = lane; t < Q; t += 32) s += W[t] * ps[i * Q + t] * ps[i * Q + t];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const double is = 1.0 / sqrt(s);
        for (int t = lane; t < Q; t += 32) ps[i * Q + t] *= is;
        for (int k = lane; k <= i; k += 32) Cs[i * n + k] *= is;
        __syncwarp();
    }
    for (int t = lane; t < n * n; t += 32) C[(size_t)e * n * n + t] = Cs[t];
    for (int i = lane; i < n; i += 32) psic[(size_t)e * n + i] = Cs[i * n];
}

// ---- level tables ---------------------------------------------------------------------------
template <int D, int NM>
__device__ __forceinline__ void eval_basis(const double x[D], int e, int n, int nmax, const double* __restrict__ xc,
                                           const double* __restrict__ Lh, const int* __restrict__ exps,
                                           const double* __restrict__ C, double psi[NM], double gpsi[NM][D]) {
    double chi[NM], g[NM][D];
    monomials<D, NM>(x, xc + e * 3, Lh + e * 3, exps, n, chi, g);
    const double* Ce = C + (size_t)e * nmax * nmax;
    for (int i = 0; i < n; ++i) {
        double v = 0.0, gv[D];
        for (int d = 0; d < D; ++d) gv[d] = 0.0;
        for (int k = 0; k <= i; ++k) {
            const double c = Ce[i * nmax + k];
            v += c * chi[k];
            for (int d = 0; d < D; ++d) gv[d] += c * g[k][d];
        }
        psi[i] = v;
        for (int d = 0; d < D; ++d) gpsi[i][d] = gv[d];
    }
}

// Frame velocity v_r = omega x x of a rotating frame at the point x (z = 0 in 2-D).
template <int D>
__device__ __forceinline__ void frame_velocity(const U5& om, const double x[D], double* vr) {
    const double x3[3] = {x[0], x[1], D == 3 ? x[D - 1] : 0.0};
    vr[0] = om.v[1] * x3[2] - om.v[2] * x3[1];
    vr[1] = om.v[2] * x3[0] - om.v[0] * x3[2];
    vr[2] = om.v[0] * x3[1] - om.v[1] * x3[0];
}

template <int D, int NM>
__global__ void k_vol_tables(int E, int n, int nmax, int q, const double* __restrict__ ex, const double* __restrict__ gl,
                             const double* __restrict__ xc, const double* __restrict__ Lh,
                             const int* __restrict__ exps, const double* __restrict__ C, double* vpsi, double* vgw,
                             U5 om, double* vvr) {
    int Q = 1;
    for (int d = 0; d < D; ++d) Q *= q;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)E * Q) return;
    const int e = (int)(idx / Q), t = (int)(idx % Q);
    const double* X = ex + (size_t)e * (1 << D) * D;
    double xi[D], x[D], J[D][D], psi[NM], g[NM][D];
    const double w = vol_point<D>(gl, q, t, xi);
    map_point<D>(X, xi, x, J);
    const double W = w * det_of<D>(J);
    eval_basis<D, NM>(x, e, n, nmax, xc, Lh, exps, C, psi, g);
    for (int i = 0; i < n; ++i) vpsi[((size_t)e * Q + t) * n + i] = psi[i];
    for (int d = 0; d < D; ++d)
        for (int i = 0; i < n; ++i) vgw[(((size_t)e * D + d) * Q + t) * n + i] = W * g[i][d];
    if (vvr) frame_velocity<D>(om, x, vvr + idx * 3);
}

template <int D, int NM>
__global__ void k_face_tables(int F, int F_int, int n, int nmax, int q, const int* __restrict__ fL,
                              const int* __restrict__ ffL, const int* __restrict__ fR, const double* __restrict__ ex,
                              const double* __restrict__ gl, const double* __restrict__ xc,
                              const double* __restrict__ Lh, const int* __restrict__ exps,
                              const double* __restrict__ C, const double* __restrict__ ewn, int has_wn,
                              const int* __restrict__ fbc, double* fnrm, double* famag, double* fpsiL,
                              double* fpsiR, double* fwn, U5 om, double* fvr) {
    int QF = 1;
    for (int d = 0; d < D - 1; ++d) QF *= q;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)F * QF) return;
    const int f = (int)(idx / QF), t = (int)(idx % QF);
    const int eL = fL[f], lf = ffL[f];
    const double* X = ex + (size_t)eL * (1 << D) * D;
    double xi[D], x[D], J[D][D], a[3], psi[NM], g[NM][D];
    const double w = face_point<D>(gl, q, lf, t, xi);
    map_point<D>(X, xi, x, J);
    cof_col<D>(J, lf >> 1, a);
    const double sgn = (lf & 1) ? 1.0 : -1.0;
    for (int k = 0; k < 3; ++k) a[k] *= sgn * w;
    const double am = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    famag[idx] = am;
    for (int k = 0; k < 3; ++k) fnrm[idx * 3 + k] = a[k] / am;
    if (f >= F_int) {
        // reflection normal of the slip wall: node body normals interpolated with the
        // multilinear shape functions at this face point and normalised; a symmetry plane
        // reflects about its own (flat) normal
        double nw[3] = {a[0] / am, a[1] / am, a[2] / am};
        if (has_wn && fbc[f] == EMG_BC_WALL) {
            double v[3] = {0.0, 0.0, 0.0};
            const double* Wn = ewn + (size_t)eL * (1 << D) * D;
            for (int nd = 0; nd < (1 << D); ++nd) {
                double Na = 1.0;
                for (int d = 0; d < D; ++d) Na *= 0.5 * (1.0 + xi[d] * ref_coord(nd, d));
                for (int d = 0; d < D; ++d) v[d] += Na * Wn[nd * D + d];
            }
            const double vm = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            if (vm > 0.0)
                for (int k = 0; k < 3; ++k) nw[k] = v[k] / vm;
        }
        const int64_t bi = (int64_t)(f - F_int) * QF + t;
        for (int k = 0; k < 3; ++k) fwn[bi * 3 + k] = nw[k];
    }
    if (fvr) frame_velocity<D>(om, x, fvr + idx * 3);
    eval_basis<D, NM>(x, eL, n, nmax, xc, Lh, exps, C, psi, g);
    for (int i = 0; i < n; ++i) fpsiL[idx * n + i] = psi[i];
    if (f < F_int) {
        eval_basis<D, NM>(x, fR[f], n, nmax, xc, Lh, exps, C, psi, g);
        for (int i = 0; i < n; ++i) fpsiR[idx * n + i] = psi[i];
    }
}

// ---- host side -------------------------------------------------------------------------------
static void gauss_legendre(int q, double* x, double* w) {
    // Newton iteration on P_q from the Chebyshev guesses; P_q and P_q' by the three-term recurrence.
    for (int i = 0; i < q; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (q + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= q; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            const double pq = q == 0 ? 1.0 : p1;
            const double pm = q == 1 ? 1.0 : p0;
            dp = q * (z * pq - pm) / (z * z - 1.0);
            const double dz = pq / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-17) break;
        }
        x[q - 1 - i] = z;
        w[q - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

static std::vector<std::array<int, 3>> basis_exponents(int dim, int p) {
    std::vector<std::array<int, 3>> out;
    for (int k = 0; k <= p; ++k) {
        if (dim == 2) {
            for (int a = k; a >= 0; --a) out.push_back({a, k - a, 0});
        } else {
            for (int a = k; a >= 0; --a)
                for (int b = k - a; b >= 0; --b) out.push_back({a, b, k - a - b});
        }
    }
    return out;
}

template <class T>
static T* dalloc(emg_ctx* c, size_t count) {
    void* p = nullptr;
    if (count == 0) count = 1;
    // stream-ordered: neither this nor the free in emg_destroy waits for other streams' work
    if (cudaMallocAsync(&p, count * sizeof(T), c->stream) != cudaSuccess) return nullptr;
    cudaMemsetAsync(p, 0, count * sizeof(T), c->stream);
    c->allocs.push_back(p);
    c->bytes += (int64_t)(count * sizeof(T));
    return static_cast<T*>(p);
}

#define EMG_ALLOC(ptr, T, count)                                              \
    do {                                                                      \
        (ptr) = dalloc<T>(c, (size_t)(count));                                \
        if (!(ptr)) {                                                         \
            c->err = "cudaMalloc failed for " #ptr;                           \
            return EMG_ERR_OOM;                                               \
        }                                                                     \
    } while (0)

struct FaceKey {
    int64_t k[4];
    int e, f;
};

template <int D, int NM>
static emg_status build_tables(emg_ctx* c, int nmax, const int* exps_d) {
    const int E = (int)c->E;
    U5 om{};
    for (int k = 0; k < 3; ++k) om.v[k] = c->prm.omega[k];
    for (int p = 0; p <= c->p_max; ++p) {
        LevelDev& L = c->lv[p];
        const int thr = 128;
        int64_t nv = (int64_t)E * L.Q;
        { ProfScope _ps(c, PC_SETUP); k_vol_tables<D, NM><<<(unsigned)((nv + thr - 1) / thr), thr, 0, c->stream>>>(
            E, L.N, nmax, L.q, c->elem_x, c->gl, c->xc, c->Lh, exps_d, c->C, L.vpsi, L.vgw, om, L.vvr); }
        EMG_CHECK_LAUNCH(c);
        int64_t nf = c->F * L.QF;
        { ProfScope _ps(c, PC_SETUP); k_face_tables<D, NM><<<(unsigned)((nf + thr - 1) / thr), thr, 0, c->stream>>>(
            (int)c->F, (int)c->F_int, L.N, nmax, L.q, c->face_L, c->face_fL, c->face_R, c->elem_x, c->gl, c->xc,
            c->Lh, exps_d, c->C, c->elem_wn, c->has_wn, c->face_bc, L.fnrm, L.famag, L.fpsiL, L.fpsiR, L.fwn, om,
            L.fvr); }
        EMG_CHECK_LAUNCH(c);
    }
    return EMG_OK;
}

// Device bytes that setup_device_mesh allocates, item by item (admission control).
int64_t estimate_bytes(int dim, int64_t E, int64_t F, int64_t F_int, int p_max, int m, int prec, bool rot) {
    const int nf = 2 * dim, nn = 1 << dim;
    const int nmax = n_modes(dim, p_max);
    const int64_t Fi1 = std::max<int64_t>(F_int, 1), Fb1 = std::max<int64_t>(F - F_int, 1);
    int64_t b = 4 * F * 4 + 2 * E * nf * 4 + 2 * E * nn * dim * 8;           // faces, element maps, x, body normals
    b += E * (3 + 3 + 1 + 1 + 1 + (int64_t)nmax * nmax + nmax) * 8 + 8 * 16 * 8 + (int64_t)nmax * 3 * 4;
    for (int p = 0; p <= p_max; ++p) {
        const int64_t N = n_modes(dim, p), q = p + 2, Q = ipow((int)q, dim), QF = ipow((int)q, dim - 1), B = 5 * N;
        b += E * Q * N * (1 + dim) * 8;                                         // vpsi, vgw
        b += F * QF * (3 + 1 + N + 5 + 25) * 8 + Fi1 * QF * (N + 25) * 8 + Fb1 * QF * 3 * 8;
        b += 6 * E * B * 8;                                                     // v, v0, tau, un, r, r2
        if (rot) b += (E * Q + F * QF) * 3 * 8;                                 // frame velocities
        if (p > 0) {
            if (blocks_f32(prec))
                b += E * B * B * 4 + E * Q * N * (1 + dim) * 4 + F * QF * (N + 25) * 4 + Fi1 * QF * (N + 25) * 4;
            else
                b += E * B * B * 8;
            b += E * B * 4;                                                     // pivots
        }
    }
    const int64_t K0 = 5 * E;
    b += E * 8 + E * (1 + nf) * 25 * 8 + (m + 1) * K0 * 8 + 2 * K0 * 8 + ((int64_t)(m + 1) * m + 2 * m + 3) * 8;
    b += 3 * 2 * 160 * (MAX_KRYLOV + 8) * 8 + 16 + (int64_t)sizeof(DevScalars);
    b += 2 * E * 5 * nmax * 8 + E * 8;                                          // staging for component calls
    return b;
}

emg_status setup_device_mesh(emg_ctx* c, const emg_mesh_desc* m) {
    const int D = m->dim;
    const int64_t E = m->n_elems;
    const int nn = 1 << D, nf = 2 * D;
    // -- face matching (host): sort the face node sets --
    std::vector<FaceKey> keys;
    std::vector<int> bE, bF, bC;
    keys.reserve((size_t)E * nf);
    for (int64_t e = 0; e < E; ++e) {
        for (int f = 0; f < nf; ++f) {
            const int bc = m->face_bc[e * nf + f];
            if (bc >= 0) {
                if (bc != EMG_BC_WALL && bc != EMG_BC_FARFIELD && bc != EMG_BC_SYMMETRY) {
                    c->err = "unsupported boundary code " + std::to_string(bc);
                    return EMG_ERR_ARG;
                }
                bE.push_back((int)e), bF.push_back(f), bC.push_back(bc);
                continue;
            }
            FaceKey k;
            int cnt = 0;
            const int axis = f >> 1;
            const double side = (f & 1) ? 1.0 : -1.0;
            for (int a = 0; a < nn; ++a)
                if (ref_coord(a, axis) == side) k.k[cnt++] = m->elem_nodes[e * nn + a];
            for (int i = cnt; i < 4; ++i) k.k[i] = -1;
            std::sort(k.k, k.k + cnt);
            k.e = (int)e;
            k.f = f;
            keys.push_back(k);
        }
    }
    std::sort(keys.begin(), keys.end(), [](const FaceKey& a, const FaceKey& b) {
        for (int i = 0; i < 4; ++i)
            if (a.k[i] != b.k[i]) return a.k[i] < b.k[i];
        return a.e < b.e;
    });
    std::vector<int> hL, hfL, hR, hbc;
    for (size_t i = 0; i < keys.size();) {
        if (i + 1 < keys.size() && std::equal(keys[i].k, keys[i].k + 4, keys[i + 1].k)) {
            if (i + 2 < keys.size() && std::equal(keys[i].k, keys[i].k + 4, keys[i + 2].k)) {
                c->err = "a face is shared by more than two elements";
                return EMG_ERR_ARG;
            }
            hL.push_back(keys[i].e), hfL.push_back(keys[i].f), hR.push_back(keys[i + 1].e), hbc.push_back(-1);
            i += 2;
        } else {
            c->err = "interior face of element " + std::to_string(keys[i].e) + " has no neighbour";
            return EMG_ERR_ARG;
        }
    }
    const int64_t F_int = (int64_t)hL.size();
    for (size_t i = 0; i < bE.size(); ++i) hL.push_back(bE[i]), hfL.push_back(bF[i]), hR.push_back(-1), hbc.push_back(bC[i]);
    const int64_t F = (int64_t)hL.size();
    std::vector<int> efc((size_t)E * nf, -1), enb((size_t)E * nf, -1);
    for (int64_t f = 0; f < F; ++f) efc[(size_t)hL[f] * nf + hfL[f]] = (int)(f << 1);
    for (size_t i = 0; i < keys.size(); i += 2) {
        const int f = (int)(i / 2);
        efc[(size_t)keys[i + 1].e * nf + keys[i + 1].f] = (f << 1) | 1;
        enb[(size_t)keys[i].e * nf + keys[i].f] = keys[i + 1].e;
        enb[(size_t)keys[i + 1].e * nf + keys[i + 1].f] = keys[i].e;
    }
    c->E = E;
    c->F = F;
    c->F_int = F_int;
    c->n_nodes = m->n_nodes;
    c->dim = D;
    // -- admission --
    const int m_kr = c->prm.krylov_m;
    const int64_t need = estimate_bytes(D, E, F, F_int, c->p_max, m_kr, c->prm.prec, c->rot);
    size_t fr = 0, tot = 0;
    EMG_CUDA_TRY(c, cudaMemGetInfo(&fr, &tot));
    if (need > (int64_t)fr) {
        c->err = "admission: needs " + std::to_string(need) + " bytes, " + std::to_string(fr) + " free";
        return EMG_ERR_OOM;
    }
    // -- mesh arrays --
    const int nmax = n_modes(D, c->p_max);
    std::vector<double> hx((size_t)E * nn * D);
    for (int64_t e = 0; e < E; ++e)
        for (int a = 0; a < nn; ++a) {
            const int64_t nd = m->elem_nodes[e * nn + a];
            if (nd < 0 || nd >= m->n_nodes) {
                c->err = "element node index out of range";
                return EMG_ERR_ARG;
            }
            for (int d = 0; d < D; ++d) hx[((size_t)e * nn + a) * D + d] = m->xyz[(size_t)d * m->n_nodes + nd];
        }
    EMG_ALLOC(c->face_L, int, F);
    EMG_ALLOC(c->face_fL, int, F);
    EMG_ALLOC(c->face_R, int, F);
    EMG_ALLOC(c->face_bc, int, F);
    EMG_ALLOC(c->elem_face, int, E * nf);
    EMG_ALLOC(c->elem_nbr, int, E * nf);
    EMG_ALLOC(c->elem_x, double, E * nn * D);
    EMG_ALLOC(c->elem_wn, double, E * nn * D);
    if (m->wall_normal) {
        std::vector<double> hw((size_t)E * nn * D);
        for (int64_t e = 0; e < E; ++e)
            for (int a = 0; a < nn; ++a)
                for (int d = 0; d < D; ++d)
                    hw[((size_t)e * nn + a) * D + d] =
                        m->wall_normal[(size_t)d * m->n_nodes + m->elem_nodes[e * nn + a]];
        EMG_CUDA_TRY(c, cudaMemcpyAsync(c->elem_wn, hw.data(), hw.size() * 8, cudaMemcpyHostToDevice, c->stream));
        EMG_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        c->has_wn = 1;
    }
    EMG_ALLOC(c->xc, double, E * 3);
    EMG_ALLOC(c->Lh, double, E * 3);
    EMG_ALLOC(c->vol, double, E);
    EMG_ALLOC(c->surf, double, E);
    EMG_ALLOC(c->h, double, E);
    EMG_ALLOC(c->C, double, E * nmax * nmax);
    EMG_ALLOC(c->psic, double, E * nmax);
    EMG_ALLOC(c->gl, double, 8 * 16);
    EMG_CUDA_TRY(c, cudaMemcpyAsync(c->face_L, hL.data(), F * 4, cudaMemcpyHostToDevice, c->stream));
    EMG_CUDA_TRY(c, cudaMemcpyAsync(c->face_fL, hfL.data(), F * 4, cudaMemcpyHostToDevice, c->stream));
    EMG_CUDA_TRY(c, cudaMemcpyAsync(c->face_R, hR.data(), F * 4, cudaMemcpyHostToDevice, c->stream));
    EMG_CUDA_TRY(c, cudaMemcpyAsync(c->face_bc, hbc.data(), F * 4, cudaMemcpyHostToDevice, c->stream));
    EMG_CUDA_TRY(c, cudaMemcpyAsync(c->elem_face, efc.data(), E * nf * 4, cudaMemcpyHostToDevice, c->stream));
    EMG_CUDA_TRY(c, cudaMemcpyAsync(c->elem_nbr, enb.data(), E * nf * 4, cudaMemcpyHostToDevice, c->stream));
    EMG_CUDA_TRY(c, cudaMemcpyAsync(c->elem_x, hx.data(), hx.size() * 8, cudaMemcpyHostToDevice, c->stream));
    std::vector<double> hgl(8 * 16, 0.0);
    for (int q = 1; q <= 7; ++q) gauss_legendre(q, &hgl[q * 16], &hgl[q * 16 + 8]);
    EMG_CUDA_TRY(c, cudaMemcpyAsync(c->gl, hgl.data(), hgl.size() * 8, cudaMemcpyHostToDevice, c->stream));
    auto ex = basis_exponents(D, c->p_max);
    std::vector<int> hexp(ex.size() * 3);
    for (size_t k = 0; k < ex.size(); ++k)
        for (int d = 0; d < 3; ++d) hexp[k * 3 + d] = ex[k][d];
    int* exps_d = nullptr;
    EMG_ALLOC(exps_d, int, hexp.size());
    EMG_CUDA_TRY(c, cudaMemcpyAsync(exps_d, hexp.data(), hexp.size() * 4, cudaMemcpyHostToDevice, c->stream));
    // -- levels --
    for (int p = 0; p <= c->p_max; ++p) {
        LevelDev& L = c->lv[p];
        L.p = p;
        L.N = n_modes(D, p);
        L.q = p + 2;
        L.Q = ipow(L.q, D);
        L.QF = ipow(L.q, D - 1);
        L.B = 5 * L.N;
        const int64_t S = E * 5 * L.N;
        EMG_ALLOC(L.vpsi, double, E * L.Q * L.N);
        EMG_ALLOC(L.vgw, double, E * D * L.Q * L.N);
        EMG_ALLOC(L.fnrm, double, F * L.QF * 3);
        EMG_ALLOC(L.famag, double, F * L.QF);
        EMG_ALLOC(L.fpsiL, double, F * L.QF * L.N);
        EMG_ALLOC(L.fpsiR, double, std::max<int64_t>(F_int, 1) * L.QF * L.N);
        EMG_ALLOC(L.fwn, double, std::max<int64_t>(F - F_int, 1) * L.QF * 3);
        EMG_ALLOC(L.v, double, S);
        EMG_ALLOC(L.v0, double, S);
        EMG_ALLOC(L.tau, double, S);
        EMG_ALLOC(L.un, double, S);
        EMG_ALLOC(L.r, double, S);
        EMG_ALLOC(L.r2, double, S);
        EMG_ALLOC(L.fhat, double, F * L.QF * 5);
        EMG_ALLOC(L.fjl, double, F * L.QF * 25);
        EMG_ALLOC(L.fjr, double, std::max<int64_t>(F_int, 1) * L.QF * 25);
        if (c->rot) {
            EMG_ALLOC(L.vvr, double, E * L.Q * 3);
            EMG_ALLOC(L.fvr, double, F * L.QF * 3);
        }
        if (p > 0) {
            if (blocks_f32(c->prm.prec)) {
                EMG_ALLOC(L.blk32, float, E * L.B * L.B);
                EMG_ALLOC(L.vpsi32, float, E * L.Q * L.N);
                EMG_ALLOC(L.vgw32, float, E * D * L.Q * L.N);
                EMG_ALLOC(L.fpsiL32, float, F * L.QF * L.N);
                EMG_ALLOC(L.fpsiR32, float, std::max<int64_t>(F_int, 1) * L.QF * L.N);
                EMG_ALLOC(L.fjl32, float, F * L.QF * 25);
                EMG_ALLOC(L.fjr32, float, std::max<int64_t>(F_int, 1) * L.QF * 25);
            } else {
                EMG_ALLOC(L.blk, double, E * L.B * L.B);
            }
            EMG_ALLOC(L.piv, int, E * L.B);
        }
    }
    // -- Krylov / EXP1 --
    const int64_t K0 = 5 * E;
    EMG_ALLOC(c->dt, double, E);
    EMG_ALLOC(c->bsr, double, E * (1 + nf) * 25);
    EMG_ALLOC(c->V, double, (m_kr + 1) * K0);
    EMG_ALLOC(c->w, double, 2 * K0);
    EMG_ALLOC(c->H, double, (m_kr + 1) * m_kr);
    EMG_ALLOC(c->hcol, double, m_kr + 2);
    EMG_ALLOC(c->y, double, m_kr + 1);
    c->red_blocks = 2 * 160;
    EMG_ALLOC(c->partial, double, 3 * c->red_blocks * (MAX_KRYLOV + 8));
    EMG_ALLOC(c->bar, unsigned int, 4);
    EMG_ALLOC(c->sc, DevScalars, 1);
    c->sc_host = pinned_scalars_acquire();
    if (!c->sc_host) {
        c->err = "page-locked host memory for the cycle scalars";
        return EMG_ERR_OOM;
    }
    const int Bmax = 5 * nmax;
    EMG_ALLOC(c->stage_in, double, E * Bmax);
    EMG_ALLOC(c->stage_in2, double, E * Bmax);
    EMG_ALLOC(c->stage_small, double, E);
    // -- device geometry, basis, tables --
    const int qg = c->p_max + 2;
    if (D == 2) {
        { ProfScope _ps(c, PC_SETUP); k_geometry<2><<<(unsigned)((E + 127) / 128), 128, 0, c->stream>>>((int)E, c->elem_x, c->gl, qg, c->vol, c->xc,
                                                                         c->Lh, c->surf, c->h); }
    } else {
        { ProfScope _ps(c, PC_SETUP); k_geometry<3><<<(unsigned)((E + 127) / 128), 128, 0, c->stream>>>((int)E, c->elem_x, c->gl, qg, c->vol, c->xc,
                                                                         c->Lh, c->surf, c->h); }
    }
    EMG_CHECK_LAUNCH(c);
    const int Qg = ipow(qg, D);
    const size_t smem = ((size_t)nmax * Qg + Qg + (size_t)nmax * nmax) * 8;
    if (smem > 200 * 1024) {
        c->err = "basis set-up does not fit in shared memory";
        return EMG_ERR_ARG;
    }
    emg_status st = EMG_OK;
    if (D == 2) {
        cudaFuncSetAttribute(k_basis<2, 15>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        { ProfScope _ps(c, PC_SETUP); k_basis<2, 15><<<(unsigned)E, 32, smem, c->stream>>>((int)E, nmax, qg, c->elem_x, c->gl, c->xc, c->Lh, exps_d,
                                                           c->C, c->psic); }
        EMG_CHECK_LAUNCH(c);
        st = build_tables<2, 15>(c, nmax, exps_d);
    } else {
        cudaFuncSetAttribute(k_basis<3, 35>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        { ProfScope _ps(c, PC_SETUP); k_basis<3, 35><<<(unsigned)E, 32, smem, c->stream>>>((int)E, nmax, qg, c->elem_x, c->gl, c->xc, c->Lh, exps_d,
                                                           c->C, c->psic); }
        EMG_CHECK_LAUNCH(c);
        st = build_tables<3, 35>(c, nmax, exps_d);
    }
    if (st != EMG_OK) return st;
    if (blocks_f32(c->prm.prec)) {
        for (int p = 1; p <= c->p_max; ++p) {
            c->lv[p].tc_asm = use_tc_assembly(D, p, c->prm.prec, c->prm.block_kernels);
            c->lv[p].tc_gj = use_tc_inverse(c->lv[p].B, c->prm.block_kernels);
        }
        st = build_float_tables(c);
        if (st != EMG_OK) return st;
        st = tune_gj(c);
        if (st != EMG_OK) return st;
    }
    std::vector<double> hv(E);
    EMG_CUDA_TRY(c, cudaMemcpyAsync(hv.data(), c->vol, E * 8, cudaMemcpyDeviceToHost, c->stream));
    EMG_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    double tot_v = 0.0;
    for (int64_t e = 0; e < E; ++e) {
        if (!(hv[e] > 0.0)) {
            c->err = "element " + std::to_string(e) + " has non-positive volume";
            return EMG_ERR_ARG;
        }
        tot_v += hv[e];
    }
    c->domain_volume = tot_v;
    return EMG_OK;
}

}  // namespace emg
