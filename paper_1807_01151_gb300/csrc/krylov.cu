// EXP1 on the p = 0 level (Eqs. EXP1, Phi1, vm, final):
//   u_0 <- u_0 + phi_1(A) N,   A = DT J_0,  N = DT R~_0(u_0),  DT = diag(dt_e),
// with phi_1(A) N ~= beta V_k phi_1(H_k) e_1 from k Arnoldi steps.  Orthogonalisation is
// classical Gram-Schmidt applied twice (CGS2), whose dot products are one batched
// reduction per pass; every reduction sums fixed per-block partials in a fixed order, so
// results do not depend on scheduling.  phi_1(H_k) e_1 is the last column of
// exp([[H_k, e_1], [0, 0]]), computed in one CTA by [13/13] Pade scaling-and-squaring
// (Higham, SIAM J. Matrix Anal. Appl. 26 (2005) 1179).  The device decides happy
// breakdown itself, so the loop needs no host round trip.
#include <cmath>

#include "common.cuh"

namespace emg {

constexpr int RED_THREADS = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    return s;  // valid in thread 0
}

// Reduce partial[0..nb-1][col] in a fixed order; result valid in thread 0... broadcast via shared.
__device__ __forceinline__ double reduce_partials(const double* partial, int nb, int stride, int col, double* sh) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += partial[(size_t)b * stride + col];
    double s = block_sum(v, sh);
    __syncthreads();
    if (threadIdx.x == 0) sh[32] = s;
    __syncthreads();
    return sh[32];
}

// w = dt * (J_0 x): BSR with one diagonal and 2d neighbour blocks per element row.
__global__ void k_spmv0(int E, int NF, const double* __restrict__ bsr, const int* __restrict__ nbr,
                        const double* __restrict__ dt, const double* __restrict__ x, double* __restrict__ y,
                        const DevScalars* __restrict__ sc) {
    if (sc->broken) return;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)E * 5) return;
    const int e = (int)(idx / 5), a = (int)(idx % 5);
    const double* row = bsr + (size_t)e * (1 + NF) * 25;
    double s = 0.0;
#pragma unroll
    for (int b = 0; b < 5; ++b) s += row[a * 5 + b] * x[(size_t)e * 5 + b];
    for (int lf = 0; lf < NF; ++lf) {
        const int nb = nbr[(size_t)e * NF + lf];
        if (nb < 0) continue;
        const double* blk = row + (1 + lf) * 25;
#pragma unroll
        for (int b = 0; b < 5; ++b) s += blk[a * 5 + b] * x[(size_t)nb * 5 + b];
    }
    y[idx] = dt[e] * s;
}

// v0 = dt * r (unnormalised start vector) and per-block partial sums of its squares.
__global__ void k_start(int64_t K0, const double* __restrict__ r, const double* __restrict__ dt,
                        double* __restrict__ v0, double* __restrict__ partial, int stride) {
    __shared__ double sh[40];
    double acc = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < K0; k += (int64_t)gridDim.x * blockDim.x) {
        const double v = dt[k / 5] * r[k];
        v0[k] = v;
        acc += v * v;
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[(size_t)blockIdx.x * stride] = s;
}

__global__ void k_start_norm(int64_t K0, double* __restrict__ v0, const double* __restrict__ partial, int nb,
                             int stride, DevScalars* sc) {
    __shared__ double sh[40];
    const double bb = reduce_partials(partial, nb, stride, 0, sh);
    const double beta = sqrt(bb);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->beta = beta;
        sc->broken = (beta == 0.0 || !isfinite(beta)) ? 1 : 0;
        sc->m_used = 0;
        if (!isfinite(beta)) sc->nonfinite = 1;
    }
    if (beta == 0.0 || !isfinite(beta)) return;
    const double ib = 1.0 / beta;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < K0; k += (int64_t)gridDim.x * blockDim.x)
        v0[k] *= ib;
}

// partial[blk][i] = sum over the block's slice of V[i] . w  (i < nv); partial[blk][nv] = w . w
__global__ void k_dots(int64_t K0, int nv, const double* __restrict__ V, const double* __restrict__ w,
                       double* __restrict__ partial, int stride, int with_ww, const DevScalars* __restrict__ sc) {
    if (sc->broken) return;
    __shared__ double sh[40];
    for (int i = 0; i < nv + with_ww; ++i) {
        const double* vi = i < nv ? V + (size_t)i * K0 : w;
        double acc = 0.0;
        for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < K0;
             k += (int64_t)gridDim.x * blockDim.x)
            acc += vi[k] * w[k];
        const double s = block_sum(acc, sh);
        if (threadIdx.x == 0) partial[(size_t)blockIdx.x * stride + i] = s;
    }
}

// h_i = sum of partials; w -= sum_i h_i V[i]; block 0 stores/accumulates h into hcol.
// pass 0 also records w0 = ||w|| before orthogonalisation; pass 1 leaves per-block
// partial sums of the squares of the updated w in partial2.
__global__ void k_orth(int64_t K0, int nv, const double* __restrict__ V, double* __restrict__ w,
                       const double* __restrict__ partial, int nb, int stride, int pass, double* __restrict__ hcol,
                       double* __restrict__ partial2, DevScalars* sc) {
    if (sc->broken) return;
    __shared__ double sh[40];
    __shared__ double hs[MAX_KRYLOV + 2];
    for (int i = 0; i < nv + (pass == 0 ? 1 : 0); ++i) {
        const double s = reduce_partials(partial, nb, stride, i, sh);
        if (threadIdx.x == 0) hs[i] = s;
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int i = 0; i < nv; ++i) hcol[i] = pass == 0 ? hs[i] : hcol[i] + hs[i];
        if (pass == 0) sc->w0 = sqrt(hs[nv]);
    }
    double acc = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < K0; k += (int64_t)gridDim.x * blockDim.x) {
        double s = w[k];
        for (int i = 0; i < nv; ++i) s -= hs[i] * V[(size_t)i * K0 + k];
        w[k] = s;
        acc += s * s;
    }
    if (pass == 1) {
        const double s = block_sum(acc, sh);
        if (threadIdx.x == 0) partial2[blockIdx.x] = s;
    }
}

// h_{j+1,j} = ||w||; happy breakdown if h_{j+1,j} <= 1e-12 ||A v_j||; else v_{j+1} = w / h.
__global__ void k_normalize(int64_t K0, int j, int m, double* __restrict__ V, const double* __restrict__ w,
                            const double* __restrict__ partial2, int nb, const double* __restrict__ hcol,
                            double* __restrict__ H, DevScalars* sc) {
    if (sc->broken) return;
    __shared__ double sh[40];
    const double hn = sqrt(reduce_partials(partial2, nb, 1, 0, sh));
    const bool brk = !(hn > 1e-12 * sc->w0);
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hcol[i];
        H[(size_t)(j + 1) * m + j] = hn;
        sc->m_used = j + 1;
        sc->hsub = hn;
        if (!isfinite(hn)) sc->nonfinite = 1;
    }
    if (brk) {
        // every block reaches the same decision from the same reduced value
        __syncthreads();
        if (threadIdx.x == 0) atomicExch(&sc->broken, 1);
        return;
    }
    const double ih = 1.0 / hn;
    double* vn = V + (size_t)(j + 1) * K0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < K0; k += (int64_t)gridDim.x * blockDim.x)
        vn[k] = w[k] * ih;
}

struct Pade13 {
    double b[14];
};

// C = A B on n x n shared matrices with leading dimension ld.
__device__ __forceinline__ void smm(const double* A, const double* B, double* C, int n, int ld) {
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        const int i = t / n, j = t % n;
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += A[i * ld + k] * B[k * ld + j];
        C[i * ld + j] = s;
    }
    __syncthreads();
}

// y = beta * [exp([[H, e1], [0, 0]])]_{0:k, k}
__global__ void k_phi(int m, const double* __restrict__ H, double* __restrict__ y, Pade13 pc, DevScalars* sc) {
    extern __shared__ double sm[];
    const int k = sc->m_used;
    const double beta = sc->beta;
    if (k == 0) return;
    const int n = k + 1, ld = n;
    const int nn = ld * n;
    double* M = sm;
    double* M2 = M + nn;
    double* M4 = M2 + nn;
    double* M6 = M4 + nn;
    double* T1 = M6 + nn;
    double* T2 = T1 + nn;
    double* U = T2 + nn;
    double* Vv = U + nn;
    __shared__ double s_norm;
    __shared__ int s_piv;
    for (int t = threadIdx.x; t < nn; t += blockDim.x) {
        const int i = t / n, j = t % n;
        double v = 0.0;
        if (i < k && j < k) v = H[(size_t)i * m + j];
        if (i == 0 && j == k) v = 1.0;
        M[i * ld + j] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double mx = 0.0;
        for (int j = 0; j < n; ++j) {
            double cs = 0.0;
            for (int i = 0; i < n; ++i) cs += fabs(M[i * ld + j]);
            mx = fmax(mx, cs);
        }
        s_norm = mx;
    }
    __syncthreads();
    const double theta13 = 5.371920351148152;
    int s = 0;
    if (s_norm > theta13) s = (int)ceil(log2(s_norm / theta13));
    const double sc2 = ldexp(1.0, -s);
    for (int t = threadIdx.x; t < nn; t += blockDim.x) M[t] *= sc2;
    __syncthreads();
    smm(M, M, M2, n, ld);
    smm(M2, M2, M4, n, ld);
    smm(M4, M2, M6, n, ld);
    const double* b = pc.b;
    for (int t = threadIdx.x; t < nn; t += blockDim.x) {
        T1[t] = b[13] * M6[t] + b[11] * M4[t] + b[9] * M2[t];
        T2[t] = b[12] * M6[t] + b[10] * M4[t] + b[8] * M2[t];
    }
    __syncthreads();
    smm(M6, T1, U, n, ld);   // U = M6 (b13 M6 + b11 M4 + b9 M2)
    smm(M6, T2, Vv, n, ld);  // V = M6 (b12 M6 + b10 M4 + b8 M2)
    for (int t = threadIdx.x; t < nn; t += blockDim.x) {
        const int i = t / n, j = t % n;
        const double id = (i == j) ? 1.0 : 0.0;
        T1[t] = U[t] + b[7] * M6[t] + b[5] * M4[t] + b[3] * M2[t] + b[1] * id;
        Vv[t] = Vv[t] + b[6] * M6[t] + b[4] * M4[t] + b[2] * M2[t] + b[0] * id;
    }
    __syncthreads();
    smm(M, T1, U, n, ld);    // U = M (...)
    // solve (V - U) X = (V + U); A in T1, RHS/X in T2
    for (int t = threadIdx.x; t < nn; t += blockDim.x) {
        T1[t] = Vv[t] - U[t];
        T2[t] = Vv[t] + U[t];
    }
    __syncthreads();
    for (int c = 0; c < n; ++c) {
        if (threadIdx.x == 0) {
            int pr = c;
            double best = fabs(T1[c * ld + c]);
            for (int r = c + 1; r < n; ++r)
                if (fabs(T1[r * ld + c]) > best) {
                    best = fabs(T1[r * ld + c]);
                    pr = r;
                }
            s_piv = pr;
        }
        __syncthreads();
        const int pr = s_piv;
        if (pr != c)
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                double t0 = T1[c * ld + j];
                T1[c * ld + j] = T1[pr * ld + j];
                T1[pr * ld + j] = t0;
                t0 = T2[c * ld + j];
                T2[c * ld + j] = T2[pr * ld + j];
                T2[pr * ld + j] = t0;
            }
        __syncthreads();
        const double ip = 1.0 / T1[c * ld + c];
        for (int t = threadIdx.x; t < (n - c - 1) * (n + n); t += blockDim.x) {
            const int r = c + 1 + t / (2 * n);
            const int j = t % (2 * n);
            const double l = T1[r * ld + c] * ip;
            if (j < n) {
                if (j > c) T1[r * ld + j] -= l * T1[c * ld + j];
            } else {
                T2[r * ld + (j - n)] -= l * T2[c * ld + (j - n)];
            }
        }
        __syncthreads();
        for (int r = c + 1 + threadIdx.x; r < n; r += blockDim.x) T1[r * ld + c] = 0.0;
        __syncthreads();
    }
    for (int c = n - 1; c >= 0; --c) {
        const double ip = 1.0 / T1[c * ld + c];
        for (int j = threadIdx.x; j < n; j += blockDim.x) T2[c * ld + j] *= ip;
        __syncthreads();
        for (int t = threadIdx.x; t < c * n; t += blockDim.x) {
            const int r = t / n, j = t % n;
            T2[r * ld + j] -= T1[r * ld + c] * T2[c * ld + j];
        }
        __syncthreads();
    }
    // squaring: X <- X^2, s times (X in T2)
    double* X = T2;
    double* Y = U;
    for (int it = 0; it < s; ++it) {
        smm(X, X, Y, n, ld);
        double* t = X;
        X = Y;
        Y = t;
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) y[i] = beta * X[i * ld + k];
}

// out = u0 + V[0:k]^T y  (out = u0 when the start vector was zero)
__global__ void k_combine(int64_t K0, const double* __restrict__ u0, const double* __restrict__ V,
                          const double* __restrict__ y, const DevScalars* __restrict__ sc, double* __restrict__ out) {
    const int k = sc->m_used;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < K0; t += (int64_t)gridDim.x * blockDim.x) {
        double s = u0[t];
        for (int j = 0; j < k; ++j) s += V[(size_t)j * K0 + t] * y[j];
        out[t] = s;
    }
}

static Pade13 pade13() {
    Pade13 p;
    const int m = 13;
    p.b[0] = 1.0;
    for (int k = 1; k <= m; ++k) p.b[k] = p.b[k - 1] * (double)(m - k + 1) / ((double)(2 * m - k + 1) * k);
    return p;
}

emg_status launch_exp1(emg_ctx* c, const double* u0, const double* tau0, const double* dt, double* out) {
    LevelDev& L = c->lv[0];
    const int64_t K0 = 5 * c->E;
    const int m = c->prm.krylov_m;
    const int nb = c->red_blocks;
    const int stride = MAX_KRYLOV + 8;
    double* part2 = c->partial + (size_t)nb * stride;  // separate tail for the norm partials
    emg_status st = launch_residual(c, 0, u0, tau0, L.r);
    if (st != EMG_OK) return st;
    st = launch_face_jacobian(c, 0, u0);
    if (st != EMG_OK) return st;
    st = launch_bsr0(c);
    if (st != EMG_OK) return st;
    { ProfScope _ps(c, PC_ARNOLDI); k_start<<<nb, RED_THREADS, 0, c->stream>>>(K0, L.r, dt, c->V, c->partial, stride); }
    EMG_CHECK_LAUNCH(c);
    { ProfScope _ps(c, PC_ARNOLDI); k_start_norm<<<nb, RED_THREADS, 0, c->stream>>>(K0, c->V, c->partial, nb, stride, c->sc); }
    EMG_CHECK_LAUNCH(c);
    const unsigned gs = (unsigned)((K0 + 255) / 256);
    const int NF = 2 * c->dim;
    for (int j = 0; j < m; ++j) {
        { ProfScope _ps(c, PC_ARNOLDI); k_spmv0<<<gs, 256, 0, c->stream>>>((int)c->E, NF, c->bsr, c->elem_nbr, dt, c->V + (size_t)j * K0, c->w,
                                           c->sc); }
        { ProfScope _ps(c, PC_ARNOLDI); k_dots<<<nb, RED_THREADS, 0, c->stream>>>(K0, j + 1, c->V, c->w, c->partial, stride, 1, c->sc); }
        { ProfScope _ps(c, PC_ARNOLDI); k_orth<<<nb, RED_THREADS, 0, c->stream>>>(K0, j + 1, c->V, c->w, c->partial, nb, stride, 0, c->hcol, part2,
                                                  c->sc); }
        { ProfScope _ps(c, PC_ARNOLDI); k_dots<<<nb, RED_THREADS, 0, c->stream>>>(K0, j + 1, c->V, c->w, c->partial, stride, 0, c->sc); }
        { ProfScope _ps(c, PC_ARNOLDI); k_orth<<<nb, RED_THREADS, 0, c->stream>>>(K0, j + 1, c->V, c->w, c->partial, nb, stride, 1, c->hcol, part2,
                                                  c->sc); }
        { ProfScope _ps(c, PC_ARNOLDI); k_normalize<<<nb, RED_THREADS, 0, c->stream>>>(K0, j, m, c->V, c->w, part2, nb, c->hcol, c->H, c->sc); }
        EMG_CHECK_LAUNCH(c);
    }
    const int n = m + 1;
    const size_t smem = (size_t)8 * n * n * sizeof(double);
    EMG_CUDA_TRY(c, cudaFuncSetAttribute(k_phi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    { ProfScope _ps(c, PC_PHI); k_phi<<<1, 256, smem, c->stream>>>(m, c->H, c->y, pade13(), c->sc); }
    EMG_CHECK_LAUNCH(c);
    { ProfScope _ps(c, PC_COMBINE); k_combine<<<nb, 256, 0, c->stream>>>(K0, u0, c->V, c->y, c->sc, out); }
    EMG_CHECK_LAUNCH(c);
    return EMG_OK;
}

}  // namespace emg
