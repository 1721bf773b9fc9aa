// Device physics: Euler flux (Eq. euler, omega = 0), Roe flux (Sec. 3.1, Roe 1981,
// no entropy fix), slip-wall and Riemann-invariant far-field ghost states (Sec. 3.3),
// all templated on the scalar so that the same code yields values (double) and exact
// derivatives by forward-mode automatic differentiation (Dual<M, S>), as the paper does
// for dF~/dU_L, dF~/dU_R and dU_ghost/dU_L.  S is the dual's base type: double for the
// FP64 form and for the p = 0 Jacobian, float for the preconditioner blocks of the FP32
// block form.
#pragma once

#include <cuda_runtime.h>

namespace emg {

// ---- forward-mode dual numbers ------------------------------------------------------
// A product that is never fused into a later addition (float); plain for double.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return a * b; }

template <int M, class S = double>
struct Dual {
    S v;
    S d[M];
};

template <int M, class S = double>
__device__ __forceinline__ Dual<M, S> dconst(double a) {
    Dual<M, S> r;
    r.v = (S)a;
#pragma unroll
    for (int i = 0; i < M; ++i) r.d[i] = (S)0;
    return r;
}

template <int M, class S>
__device__ __forceinline__ Dual<M, S> operator+(const Dual<M, S>& a, const Dual<M, S>& b) {
    Dual<M, S> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int i = 0; i < M; ++i) r.d[i] = a.d[i] + b.d[i];
    return r;
}
template <int M, class S>
__device__ __forceinline__ Dual<M, S> operator-(const Dual<M, S>& a, const Dual<M, S>& b) {
    Dual<M, S> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int i = 0; i < M; ++i) r.d[i] = a.d[i] - b.d[i];
    return r;
}
template <int M, class S>
__device__ __forceinline__ Dual<M, S> operator-(const Dual<M, S>& a) {
    Dual<M, S> r;
    r.v = -a.v;
#pragma unroll
    for (int i = 0; i < M; ++i) r.d[i] = -a.d[i];
    return r;
}
template <int M, class S>
__device__ __forceinline__ Dual<M, S> operator*(const Dual<M, S>& a, const Dual<M, S>& b) {
    Dual<M, S> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int i = 0; i < M; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
template <int M, class S>
__device__ __forceinline__ Dual<M, S> operator/(const Dual<M, S>& a, const Dual<M, S>& b) {
    Dual<M, S> r;
    const S ib = (S)1 / b.v;
    r.v = a.v * ib;
#pragma unroll
    for (int i = 0; i < M; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
    return r;
}
template <int M, class S>
__device__ __forceinline__ Dual<M, S> operator*(double a, const Dual<M, S>& b) {
    Dual<M, S> r;
    const S s = (S)a;
    r.v = s * b.v;
#pragma unroll
    for (int i = 0; i < M; ++i) r.d[i] = s * b.d[i];
    return r;
}
template <int M, class S>
__device__ __forceinline__ Dual<M, S> operator*(const Dual<M, S>& b, double a) { return a * b; }
template <int M, class S>
__device__ __forceinline__ Dual<M, S> operator+(const Dual<M, S>& b, double a) {
    Dual<M, S> r = b;
    r.v += (S)a;
    return r;
}
template <int M, class S>
__device__ __forceinline__ Dual<M, S> operator-(const Dual<M, S>& b, double a) {
    Dual<M, S> r = b;
    r.v -= (S)a;
    return r;
}
template <int M, class S>
__device__ __forceinline__ Dual<M, S> operator-(double a, const Dual<M, S>& b) {
    return dconst<M, S>(a) - b;
}

// Float duals (the float32 block forms' face Jacobians): every product and sum rounded on its
// own, never contracted into a fused multiply-add, so that one derivative direction gives the
// same bits whether it is carried alone or beside others (the compiler may otherwise fuse
// differently once seeds of 0 and 1 are known constants).
template <int M>
__device__ __forceinline__ Dual<M, float> operator*(const Dual<M, float>& a, const Dual<M, float>& b) {
    Dual<M, float> r;
    r.v = __fmul_rn(a.v, b.v);
#pragma unroll
    for (int i = 0; i < M; ++i) r.d[i] = __fadd_rn(__fmul_rn(a.d[i], b.v), __fmul_rn(a.v, b.d[i]));
    return r;
}
template <int M>
__device__ __forceinline__ Dual<M, float> operator/(const Dual<M, float>& a, const Dual<M, float>& b) {
    Dual<M, float> r;
    const float ib = 1.0f / b.v;
    r.v = __fmul_rn(a.v, ib);
#pragma unroll
    for (int i = 0; i < M; ++i) r.d[i] = __fmul_rn(__fsub_rn(a.d[i], __fmul_rn(r.v, b.d[i])), ib);
    return r;
}
template <int M>
__device__ __forceinline__ Dual<M, float> operator*(double a, const Dual<M, float>& b) {
    Dual<M, float> r;
    const float s = (float)a;
    r.v = __fmul_rn(s, b.v);
#pragma unroll
    for (int i = 0; i < M; ++i) r.d[i] = __fmul_rn(s, b.d[i]);
    return r;
}
template <int M>
__device__ __forceinline__ Dual<M, float> operator*(const Dual<M, float>& b, double a) { return a * b; }

__device__ __forceinline__ double sqrt_(double a) { return sqrt(a); }
__device__ __forceinline__ double abs_(double a) { return fabs(a); }
__device__ __forceinline__ double powr_(double a, double e) { return pow(a, e); }
__device__ __forceinline__ double val(double a) { return a; }
__device__ __forceinline__ double inv_(double a) { return 1.0 / a; }

template <int M, class S>
__device__ __forceinline__ Dual<M, S> sqrt_(const Dual<M, S>& a) {
    Dual<M, S> r;
    r.v = sqrt(a.v);
    const S h = (S)0.5 / r.v;
#pragma unroll
    for (int i = 0; i < M; ++i) r.d[i] = mul_rn(a.d[i], h);
    return r;
}
// |x| with d|x|/dx = sign(x), sign(0) = +1 (matches the analytic continuation x*sign(Re x)).
template <int M, class S>
__device__ __forceinline__ Dual<M, S> abs_(const Dual<M, S>& a) {
    return a.v >= (S)0 ? a : -a;
}
template <int M, class S>
__device__ __forceinline__ Dual<M, S> powr_(const Dual<M, S>& a, double e) {
    Dual<M, S> r;
    r.v = pow(a.v, (S)e);
    const S g = (S)e * r.v / a.v;
#pragma unroll
    for (int i = 0; i < M; ++i) r.d[i] = mul_rn(a.d[i], g);
    return r;
}
template <int M, class S>
__device__ __forceinline__ double val(const Dual<M, S>& a) { return (double)a.v; }
template <int M, class S>
__device__ __forceinline__ Dual<M, S> inv_(const Dual<M, S>& a) { return dconst<M, S>(1.0) / a; }
__device__ __forceinline__ double dconst_like(double, double a) { return a; }
template <int M, class S>
__device__ __forceinline__ Dual<M, S> dconst_like(const Dual<M, S>&, double a) { return dconst<M, S>(a); }

// ---- Euler ----------------------------------------------------------------------------
// U = (rho, rho u, rho v, rho w, rho E); n has three components (n_z = 0 in 2-D).

template <class T>
__device__ __forceinline__ void primitives(const T U[5], double g, T& rho, T v[3], T& p) {
    rho = U[0];
    T ir = inv_(rho);
    v[0] = U[1] * ir;
    v[1] = U[2] * ir;
    v[2] = U[3] * ir;
    p = (g - 1.0) * (U[4] - 0.5 * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
}

// Normal flux F(U).n from U and its velocity and pressure
template <class T>
__device__ __forceinline__ void flux_n_vp(const T U[5], const T v[3], const T& p, const double n[3], T F[5]) {
    T qn = v[0] * n[0] + v[1] * n[1] + v[2] * n[2];
    T mq = U[0] * qn;
    F[0] = mq;
    F[1] = mq * v[0] + p * n[0];
    F[2] = mq * v[1] + p * n[1];
    F[3] = mq * v[2] + p * n[2];
    F[4] = (U[4] + p) * qn;
}

// Normal flux F(U).n
template <class T>
__device__ __forceinline__ void flux_n(const T U[5], const double n[3], double g, T F[5]) {
    T rho, v[3], p;
    primitives(U, g, rho, v, p);
    flux_n_vp(U, v, p, n, F);
}

// Primitives and 1/rho (computed once: velocity, enthalpy and flux all use it)
template <class T>
__device__ __forceinline__ void primitives_ir(const T U[5], double g, T& ir, T v[3], T& p) {
    ir = inv_(U[0]);
    v[0] = U[1] * ir;
    v[1] = U[2] * ir;
    v[2] = U[3] * ir;
    p = (g - 1.0) * (U[4] - 0.5 * U[0] * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
}

// Cartesian flux component k (double only; used by the volume integral).
__device__ __forceinline__ void flux_k(const double U[5], double g, double F[3][5]) {
    const double ir = 1.0 / U[0];
    const double v0 = U[1] * ir, v1 = U[2] * ir, v2 = U[3] * ir;
    const double p = (g - 1.0) * (U[4] - 0.5 * (U[1] * v0 + U[2] * v1 + U[3] * v2));
    const double vv[3] = {v0, v1, v2};
    const double H = U[4] + p;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        F[k][0] = U[1 + k];
        F[k][1] = U[1] * vv[k];
        F[k][2] = U[2] * vv[k];
        F[k][3] = U[3] * vv[k];
        F[k][1 + k] += p;
        F[k][4] = H * vv[k];
    }
}

// Roe flux; with ROT the face moves with normal speed vrn (a rotating frame: v_r . n): the
// normal fluxes carry the relative normal velocity, F_n - vrn U (mass and momentum with
// v - v_r, energy rho E (v - v_r) + p v), and the waves' speeds are shifted by -vrn; the
// Roe averages, wave strengths and eigenvectors are those of the stationary face.
template <class T, bool ROT = false>
__device__ __forceinline__ void roe_flux(const T UL[5], const T UR[5], const double n[3], double g, T F[5],
                                         double vrn = 0.0) {
    T irL, vL[3], pL, irR, vR[3], pR;
    primitives_ir(UL, g, irL, vL, pL);
    primitives_ir(UR, g, irR, vR, pR);
    const T rL = UL[0], rR = UR[0];
    T HL = (UL[4] + pL) * irL;
    T HR = (UR[4] + pR) * irR;
    T sL = sqrt_(rL), sR = sqrt_(rR);
    T iden = inv_(sL + sR);
    T u[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) u[k] = (sL * vL[k] + sR * vR[k]) * iden;
    T H = (sL * HL + sR * HR) * iden;
    T rho = sL * sR;
    T q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    T c2 = (g - 1.0) * (H - 0.5 * q2);
    T c = sqrt_(c2);
    T ic2 = inv_(c2);
    T qn = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
    T drho = rR - rL;
    T dp = pR - pL;
    T dv[3] = {vR[0] - vL[0], vR[1] - vL[1], vR[2] - vL[2]};
    T dqn = dv[0] * n[0] + dv[1] * n[1] + dv[2] * n[2];
    T rc = rho * c;
    T a1 = (dp - rc * dqn) * (0.5 * ic2);
    T a5 = (dp + rc * dqn) * (0.5 * ic2);
    T a2 = drho - dp * ic2;
    T dvt[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) dvt[k] = dv[k] - dqn * n[k];
    T l1, l2, l5;
    if constexpr (ROT) {
        const T qr = qn - vrn;
        l1 = abs_(qr - c), l2 = abs_(qr), l5 = abs_(qr + c);
    } else {
        l1 = abs_(qn - c), l2 = abs_(qn), l5 = abs_(qn + c);
    }
    T w1 = l1 * a1, w2 = l2 * a2, w5 = l5 * a5, ws = l2 * rho;
    T FL[5], FR[5];
    flux_n_vp(UL, vL, pL, n, FL);
    flux_n_vp(UR, vR, pR, n, FR);
    if constexpr (ROT) {
#pragma unroll
        for (int a = 0; a < 5; ++a) {
            FL[a] = FL[a] - vrn * UL[a];
            FR[a] = FR[a] - vrn * UR[a];
        }
    }
    T d0 = w1 + w2 + w5;
    F[0] = 0.5 * (FL[0] + FR[0] - d0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        T dk = w1 * (u[k] - c * n[k]) + w2 * u[k] + ws * dvt[k] + w5 * (u[k] + c * n[k]);
        F[1 + k] = 0.5 * (FL[1 + k] + FR[1 + k] - dk);
    }
    T udvt = u[0] * dvt[0] + u[1] * dvt[1] + u[2] * dvt[2];
    T d4 = w1 * (H - c * qn) + w2 * (0.5 * q2) + ws * udvt + w5 * (H + c * qn);
    F[4] = 0.5 * (FL[4] + FR[4] - d4);
}

template <class T>
__device__ __forceinline__ void wall_ghost(const T UL[5], const double n[3], T G[5]) {
    T mn = UL[1] * n[0] + UL[2] * n[1] + UL[3] * n[2];
    G[0] = UL[0];
    G[1] = UL[1] - 2.0 * mn * n[0];
    G[2] = UL[2] - 2.0 * mn * n[1];
    G[3] = UL[3] - 2.0 * mn * n[2];
    G[4] = UL[4];
}

// Slip wall at rest in a rotating frame: the velocity relative to the frame (v - v_r) mirrored
// about n, density and pressure kept (the kinetic energy changes with the absolute velocity).
template <class T>
__device__ __forceinline__ void wall_ghost_rel(const T UL[5], const double n[3], const double vr[3], double g,
                                               T G[5]) {
    T ir = inv_(UL[0]);
    T v[3] = {UL[1] * ir, UL[2] * ir, UL[3] * ir};
    T p = (g - 1.0) * (UL[4] - 0.5 * UL[0] * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
    T wn = (v[0] - vr[0]) * n[0] + (v[1] - vr[1]) * n[1] + (v[2] - vr[2]) * n[2];
    T vg[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) vg[k] = v[k] - 2.0 * wn * n[k];
    G[0] = UL[0];
#pragma unroll
    for (int k = 0; k < 3; ++k) G[1 + k] = UL[0] * vg[k];
    G[4] = p * (1.0 / (g - 1.0)) + 0.5 * UL[0] * (vg[0] * vg[0] + vg[1] * vg[1] + vg[2] * vg[2]);
}

// Subsonic characteristic far field: R+ = q_n,L + 2c_L/(g-1) from inside, R- = q_n,inf -
// 2c_inf/(g-1) from outside; entropy and tangential velocity from the upwind side.
template <class T>
__device__ __forceinline__ void farfield_ghost(const T UL[5], const double n[3], const double Ui[5], double g,
                                               T G[5]) {
    T rL, vL[3], pL;
    primitives(UL, g, rL, vL, pL);
    const double ri = Ui[0];
    const double vi[3] = {Ui[1] / ri, Ui[2] / ri, Ui[3] / ri};
    const double pi = (g - 1.0) * (Ui[4] - 0.5 * ri * (vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2]));
    const double ci = sqrt(g * pi / ri);
    const double qni = vi[0] * n[0] + vi[1] * n[1] + vi[2] * n[2];
    T cL = sqrt_(g * pL * inv_(rL));
    T qnL = vL[0] * n[0] + vL[1] * n[1] + vL[2] * n[2];
    T Rp = qnL + (2.0 / (g - 1.0)) * cL;
    const double Rm = qni - 2.0 * ci / (g - 1.0);
    T qnb = 0.5 * (Rp + Rm);
    T cb = (0.25 * (g - 1.0)) * (Rp - Rm);
    T s, vb[3];
    if (val(qnb) < 0.0) {
        s = dconst_like(qnb, pi / pow(ri, g));
#pragma unroll
        for (int k = 0; k < 3; ++k) vb[k] = (qnb - qni) * n[k] + vi[k];
    } else {
        s = pL * inv_(powr_(rL, g));
#pragma unroll
        for (int k = 0; k < 3; ++k) vb[k] = vL[k] + (qnb - qnL) * n[k];
    }
    T rb = powr_(cb * cb * inv_(g * s), 1.0 / (g - 1.0));
    T pb = rb * cb * cb * (1.0 / g);
    G[0] = rb;
    G[1] = rb * vb[0];
    G[2] = rb * vb[1];
    G[3] = rb * vb[2];
    G[4] = pb * (1.0 / (g - 1.0)) + 0.5 * rb * (vb[0] * vb[0] + vb[1] * vb[1] + vb[2] * vb[2]);
}

// The far field of a rotating frame: the stationary-frame condition on velocities relative to
// the frame (v - v_r for the interior state and the free stream, which is given in the
// absolute frame), the ghost's velocity taken back to the absolute frame.
template <class T>
__device__ __forceinline__ void farfield_ghost_rel(const T UL[5], const double n[3], const double Ui[5], double g,
                                                   const double vr[3], T G[5]) {
    T ir = inv_(UL[0]);
    T v[3] = {UL[1] * ir, UL[2] * ir, UL[3] * ir};
    T q2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    T Ur[5];
    Ur[0] = UL[0];
    T w[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        w[k] = v[k] - vr[k];
        Ur[1 + k] = UL[0] * w[k];
    }
    // same pressure: rho E_rel = rho E - rho |v|^2 / 2 + rho |v - v_r|^2 / 2
    Ur[4] = UL[4] - 0.5 * UL[0] * q2 + 0.5 * UL[0] * (w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double Uir[5];
    {
        const double ri = Ui[0];
        double vi[3], wi[3];
        for (int k = 0; k < 3; ++k) {
            vi[k] = Ui[1 + k] / ri;
            wi[k] = vi[k] - vr[k];
        }
        Uir[0] = ri;
        for (int k = 0; k < 3; ++k) Uir[1 + k] = ri * wi[k];
        Uir[4] = Ui[4] - 0.5 * ri * (vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2]) +
                 0.5 * ri * (wi[0] * wi[0] + wi[1] * wi[1] + wi[2] * wi[2]);
    }
    T Gr[5];
    farfield_ghost(Ur, n, Uir, g, Gr);
    T ig = inv_(Gr[0]);
    T wg[3] = {Gr[1] * ig, Gr[2] * ig, Gr[3] * ig};
    T vb[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) vb[k] = wg[k] + vr[k];
    G[0] = Gr[0];
#pragma unroll
    for (int k = 0; k < 3; ++k) G[1 + k] = Gr[0] * vb[k];
    G[4] = Gr[4] - 0.5 * Gr[0] * (wg[0] * wg[0] + wg[1] * wg[1] + wg[2] * wg[2]) +
           0.5 * Gr[0] * (vb[0] * vb[0] + vb[1] * vb[1] + vb[2] * vb[2]);
}

}  // namespace emg
