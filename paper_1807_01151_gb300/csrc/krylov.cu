// EXP1 on the p = 0 level (Eqs. EXP1, Phi1, vm, final):
//   u_0 <- u_0 + phi_1(A) N,   A = DT J_0,  N = DT R~_0(u_0),  DT = diag(dt_e),
// with phi_1(A) N ~= beta V_k phi_1(H_k) e_1 from k Arnoldi steps.  Orthogonalisation is
// classical Gram-Schmidt applied twice (CGS2), whose dot products are one batched
// reduction per pass; every reduction sums fixed per-block partials in a fixed order, so
// results do not depend on scheduling.  phi_1(H_k) e_1 is the last column of
// exp([[H_k, e_1], [0, 0]]), computed in one CTA by [13/13] Pade scaling-and-squaring
// (Higham, SIAM J. Matrix Anal. Appl. 26 (2005) 1179).  The device decides happy
// breakdown itself, so the loop needs no host round trip.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include <functional>
#include <mutex>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace emg {

// ---- persistent Arnoldi: one cooperative launch for the whole Krylov loop ------------------
// Grid barrier on a monotonic arrival counter in global memory (zeroed before the launch):
// at its e-th barrier a block adds one and waits until the counter reaches e * nblocks, so
// the last arrival releases everyone without a reset.  Waits are bounded: after `budget`
// clock cycles the block records a timeout in sc->timeout and the kernel returns (the host
// maps it to EMG_ERR_TIMEOUT); nothing spins forever.
struct GridBar {
    unsigned int count;
    unsigned int unused;
};

__device__ __forceinline__ bool grid_sync(GridBar* bar, unsigned nblocks, unsigned* epoch, long long budget,
                                          DevScalars* sc, int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned target = (*epoch + 1u) * nblocks;
        *epoch += 1u;
        __threadfence();
        const unsigned arrived = atomicAdd(&bar->count, 1u) + 1u;
        int ok = 1;
        if (arrived < target) {
            volatile unsigned int* vc = &bar->count;
            const long long t0 = clock64();
            while (*vc < target) {
                if (clock64() - t0 > budget) {
                    atomicExch(&sc->timeout, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(20);
            }
        }
        __threadfence();
        *s_ok = ok && !*((volatile int*)&sc->timeout);
    }
    __syncthreads();
    return *s_ok != 0;
}

constexpr int ARN_THREADS = 256;
constexpr int ARN_PER_THREAD = 1;   // spread the FP64 work over every SM (FP64 is slow per SM)

// Blocks of the persistent Arnoldi launch: about ARN_PER_THREAD entries per thread, at most
// what is co-resident (per_sm per SM) and at most `cap`.
static int64_t arnoldi_blocks(int64_t K0, int nsm, int per_sm, int64_t cap) {
    int64_t nb = (K0 + (int64_t)ARN_THREADS * ARN_PER_THREAD - 1) / ((int64_t)ARN_THREADS * ARN_PER_THREAD);
    const int64_t resident = (int64_t)nsm * (per_sm < 1 ? 1 : per_sm);
    if (nb > resident) nb = resident;
    if (nb > cap) nb = cap;
    return nb < 1 ? 1 : nb;
}
constexpr int ARN_CHUNK = 8;  // vectors per dot-product sweep
static_assert(ARN_CHUNK == 8, "warp_sum8 reduces eight columns");

constexpr int ARN_MAXCOL = MAX_KRYLOV + 8;
constexpr int ARN_WARPS = ARN_THREADS / 32;
constexpr int ARN_SUB = 8;    // threads per column in the cross-block reduction

// Arithmetic of the Arnoldi process in the basis' precision T (double, or float for the float32
// Krylov form): explicit fused multiply-adds (so that every form of the process computes the
// same bits), and the happy-breakdown threshold h_{j+1,j} <= tol ||A v_j|| at that precision.
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <class T>
__device__ __forceinline__ T arn_breakdown_tol();
template <>
__device__ __forceinline__ double arn_breakdown_tol<double>() { return 1e-12; }
template <>
__device__ __forceinline__ float arn_breakdown_tol<float>() { return 1e-5f; }

// Warp sums of the 8 values v[0..8) of every lane with 9 shuffle-adds per lane: at each of
// the first three levels a lane keeps half of its columns and receives its partner's
// partial sums of them (a transposing butterfly), then two plain levels.  Afterwards lane l
// holds the warp sum of column 4 b4(l) + 2 b3(l) + b2(l) (b_k = bit k of l); returns it.
// The order of the additions is fixed.
template <class T>
__device__ __forceinline__ T warp_sum8(const T v[8], int lane, int* col) {
    const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4;
    T a[4], b[2];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const T send = u16 ? v[c] : v[c + 4];
        const T keep = u16 ? v[c + 4] : v[c];
        a[c] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const T send = u8 ? a[c] : a[c + 2];
        const T keep = u8 ? a[c + 2] : a[c];
        b[c] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    const T send = u4 ? b[0] : b[1];
    T x = (u4 ? b[1] : b[0]) + __shfl_xor_sync(0xffffffffu, send, 4);
    x += __shfl_xor_sync(0xffffffffu, x, 2);
    x += __shfl_xor_sync(0xffffffffu, x, 1);
    *col = (u16 ? 4 : 0) + (u8 ? 2 : 0) + (u4 ? 1 : 0);
    return x;
}

// Block-reduce v[0..n) (n <= ARN_CHUNK): warp shuffles, then one barrier; dst[0..n) from
// threads 0..n-1 (fixed order).
template <class T>
__device__ __forceinline__ void block_reduce_store(T v[ARN_CHUNK], int n, T* dst,
                                                   T (*sh)[ARN_MAXCOL]) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (n == 1) {
        T x = v[0];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sh[warp][0] = x;
    } else {
        int c = 0;
        const T x = warp_sum8<T>(v, lane, &c);
        if ((lane & 3) == 0) sh[warp][c] = x;
    }
    __syncthreads();
    if (threadIdx.x < n) {
        T s = 0.0;
        for (int w = 0; w < ARN_WARPS; ++w) s += sh[w][threadIdx.x];
        dst[threadIdx.x] = s;
    }
    __syncthreads();
}

// out_sh[c] = sum over blocks b of part[b * stride + c], c < ncol, identical in every block:
// ARN_SUB threads per column sum a fixed stride of blocks (eight loads issued together, then
// added in order), then a fixed shuffle tree.
template <class T>
__device__ __forceinline__ void reduce_cols(const T* part, int nb, int stride, int ncol, T* out_sh,
                                            T (*sh)[ARN_MAXCOL]) {
    const int sub = threadIdx.x % ARN_SUB;
    for (int c0 = 0; c0 < ncol; c0 += ARN_THREADS / ARN_SUB) {
        const int c = c0 + threadIdx.x / ARN_SUB;
        T v = 0.0;
        if (c < ncol) {
            for (int b0 = sub; b0 < nb; b0 += 8 * ARN_SUB) {
                T x[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int b = b0 + u * ARN_SUB;
                    x[u] = b < nb ? __ldcg(part + (size_t)b * stride + c) : 0.0;   // other blocks' data: L2
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) v += x[u];
            }
        }
        for (int o = ARN_SUB / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, ARN_SUB);
        if (sub == 0 && c < ncol) out_sh[c] = v;
    }
    __syncthreads();
}

// dst[i] (i < nv) = V[i] . w over this block's slice, plus w . w at index nv if with_ww
// (warp shuffles per chunk of columns, one barrier for all of them).
template <class T>
__device__ __forceinline__ void slice_dots(const T* V, const T* w, int64_t K0, int64_t k0, int64_t k1,
                                           int nv, int with_ww, T* dst, T (*sh)[ARN_MAXCOL]) {
    const int ncol = nv + with_ww;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c0 = 0; c0 < ncol; c0 += ARN_CHUNK) {
        T v[ARN_CHUNK];
#pragma unroll
        for (int i = 0; i < ARN_CHUNK; ++i) v[i] = 0.0;
        for (int64_t k = k0 + threadIdx.x; k < k1; k += ARN_THREADS) {
            const T wk = w[k];
#pragma unroll
            for (int i = 0; i < ARN_CHUNK; ++i) {
                const int col = c0 + i;
                if (col < nv) v[i] = fma_t(V[(size_t)col * K0 + k], wk, v[i]);
                else if (col == nv && with_ww) v[i] = fma_t(wk, wk, v[i]);
            }
        }
        int c = 0;
        const T x = warp_sum8<T>(v, lane, &c);
        if ((lane & 3) == 0 && c0 + c < ncol) sh[warp][c0 + c] = x;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < ncol; c += ARN_THREADS) {
        T s = 0.0;
        for (int wv = 0; wv < ARN_WARPS; ++wv) s += sh[wv][c];
        dst[c] = s;
    }
}

// out[k] = scale * dt_e * (J_0 x)_k for this block's rows; x may belong to other blocks
// (read through L2) and is either a vector or, when xr != nullptr, dt .* xr computed on the fly.
template <class T>
__device__ __forceinline__ void spmv_rows(int64_t k0, int64_t k1, int NF, const double* __restrict__ bsr,
                                          const int* __restrict__ nbr, const double* __restrict__ dt,
                                          const T* x, const double* __restrict__ xr, T scale,
                                          T* __restrict__ out) {
    for (int64_t k = k0 + threadIdx.x; k < k1; k += ARN_THREADS) {
        const int e = (int)(k / 5), a = (int)(k % 5);
        const double* row = bsr + (size_t)e * (1 + NF) * 25;
        T s = 0.0;
        if (xr) {
            const double de = dt[e];
#pragma unroll
            for (int b = 0; b < 5; ++b) s = fma_t((T)row[a * 5 + b], (T)(de * xr[(size_t)e * 5 + b]), s);
            for (int lf = 0; lf < NF; ++lf) {
                const int n = nbr[(size_t)e * NF + lf];
                if (n < 0) continue;
                const double dn = dt[n];
                const double* blk = row + (1 + lf) * 25;
#pragma unroll
                for (int b = 0; b < 5; ++b) s = fma_t((T)blk[a * 5 + b], (T)(dn * xr[(size_t)n * 5 + b]), s);
            }
        } else {
#pragma unroll
            for (int b = 0; b < 5; ++b) s = fma_t((T)row[a * 5 + b], __ldcg(x + (size_t)e * 5 + b), s);
            for (int lf = 0; lf < NF; ++lf) {
                const int n = nbr[(size_t)e * NF + lf];
                if (n < 0) continue;
                const double* blk = row + (1 + lf) * 25;
#pragma unroll
                for (int b = 0; b < 5; ++b) s = fma_t((T)blk[a * 5 + b], __ldcg(x + (size_t)n * 5 + b), s);   // other blocks
            }
        }
        out[k] = (T)dt[e] * (scale * s);
    }
}

// Row k of A x = DT J_0 x for the vector x (other blocks' entries read through L2).
template <class T>
__device__ __forceinline__ T a_row(int64_t k, int NF, const double* __restrict__ bsr, const int* __restrict__ nbr,
                                        const double* __restrict__ dt, const T* x) {
    const int e = (int)(k / 5), a = (int)(k % 5);
    const double* row = bsr + (size_t)e * (1 + NF) * 25;
    T s = 0.0;
#pragma unroll
    for (int b = 0; b < 5; ++b) s = fma_t((T)row[a * 5 + b], __ldcg(x + (size_t)e * 5 + b), s);
    for (int lf = 0; lf < NF; ++lf) {
        const int n = nbr[(size_t)e * NF + lf];
        if (n < 0) continue;
        const double* blk = row + (1 + lf) * 25;
#pragma unroll
        for (int b = 0; b < 5; ++b) s = fma_t((T)blk[a * 5 + b], __ldcg(x + (size_t)n * 5 + b), s);
    }
    return (T)dt[e] * s;
}

// The two halves of Krylov step j, shared by the persistent kernel and the barrier-free
// kernels (the same blocks and the same arithmetic in the same order: bitwise the same
// results).  CGS2 with two reductions per step: the first sweep gives h1 = V^T w and w.w,
// the second h2 = V^T w1 and w1.w1 (w1 = w - V h1); with V orthonormal the subdiagonal is
// h_{j+1,j} = (w1.w1 - h2.h2)^(1/2), so no third reduction is needed.  The next product is
// A v_{j+1} = (A w1 - A V h2) / h_{j+1,j}: A w1 uses the neighbours' w1 (final at the second
// reduction) and A V h2 = V (H~_j h2), from the Arnoldi relation A v_i = sum_l h_{l,i} v_l,
// uses this block's rows only (h2 is at rounding level, so the correction is small).

// First half: h1 from the first sweep's partials; w <- w1 = w - V h1 on this block's rows;
// the second sweep into partB.
template <class T>
__device__ __forceinline__ void arn_half1(int j, int64_t K0, int64_t k0, int64_t k1, int nb, int stride,
                                          const T* V, T* w, const T* partA, T* partB_blk,
                                          T* h1, T (*sh)[ARN_MAXCOL]) {
    reduce_cols<T>(partA, nb, stride, j + 2, h1, sh);
    for (int64_t k = k0 + threadIdx.x; k < k1; k += ARN_THREADS) {
        T s = w[k];
        for (int i = 0; i <= j; ++i) s = fma_t(-h1[i], V[(size_t)i * K0 + k], s);
        w[k] = s;
    }
    __syncthreads();
    slice_dots<T>(V, w, K0, k0, k1, j + 1, 1, partB_blk, sh);
}

// Second half: h2 and w1.w1; h_{j+1,j}; Hessenberg column j (into this block's copy Hs, and by
// block 0 into H with the flags); unless the process ends (breakdown or j + 1 = m): v_{j+1},
// the next product into wn and the next step's first sweep into partA.  Returns whether the
// process continues (the same in every block).  Hs is the block's shared copy of H (row
// stride ARN_HLD), complete up to column j - 1 on entry.
constexpr int ARN_HLD = 41;   // row stride of the shared Hessenberg copy (m <= 40)
template <class T>
__device__ __forceinline__ bool arn_half2(int j, int m, int64_t K0, int64_t k0, int64_t k1, int nb, int stride,
                                          int NF, const double* __restrict__ bsr, const int* __restrict__ nbr,
                                          const double* __restrict__ dt, T* V, const T* w1, T* wn,
                                          double* H, T* Hs, const T* partB, T* partA_blk,
                                          const T* h1, T* h2, T* cs, DevScalars* sc,
                                          T (*sh)[ARN_MAXCOL]) {
    reduce_cols<T>(partB, nb, stride, j + 2, h2, sh);
    T hh = 0.0;
    for (int i = 0; i <= j; ++i) hh = fma_t(h2[i], h2[i], hh);
    const T hn = sqrt(fmax(h2[j + 1] - hh, (T)0));
    const T w0 = sqrt(h1[j + 1]);
    const bool brk = !(hn > arn_breakdown_tol<T>() * w0);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = h1[i] + h2[i];
        H[(size_t)(j + 1) * m + j] = hn;
        sc->m_used = j + 1;
        sc->hsub = hn;
        sc->w0 = w0;
        if (!isfinite(hn)) sc->nonfinite = 1;
        if (brk) sc->broken = 1;
    }
    if (brk || j + 1 == m) return false;   // uniform: every block reduced the same values
    for (int i = threadIdx.x; i <= j + 1; i += ARN_THREADS) Hs[i * ARN_HLD + j] = i <= j ? h1[i] + h2[i] : hn;
    __syncthreads();
    const T ih = (T)1 / hn;
    // c = H~_j h2 over l = 0..j+1
    for (int l = threadIdx.x; l <= j + 1; l += ARN_THREADS) {
        T c = 0.0;
        for (int i = (l > 0 ? l - 1 : 0); i <= j; ++i) c = fma_t(Hs[l * ARN_HLD + i], h2[i], c);
        cs[l] = c;
    }
    __syncthreads();
    T* vn = V + (size_t)(j + 1) * K0;
    for (int64_t k = k0 + threadIdx.x; k < k1; k += ARN_THREADS) {
        T s = w1[k];
        T t = a_row<T>(k, NF, bsr, nbr, dt, w1);
        for (int i = 0; i <= j; ++i) {
            const T vi = V[(size_t)i * K0 + k];
            s = fma_t(-h2[i], vi, s);
            t = fma_t(-cs[i], vi, t);
        }
        const T v = s * ih;
        vn[k] = v;
        t = fma_t(-cs[j + 1], v, t);
        wn[k] = t * ih;
    }
    __syncthreads();
    slice_dots<T>(V, wn, K0, k0, k1, j + 2, 1, partA_blk, sh);
    return true;
}

// ---- the persistent process with this thread's Krylov rows in registers -------------------
// When every thread owns at most one row (chunk <= ARN_THREADS) and m <= MV, the persistent
// kernel keeps the thread's entries of v_0 .. v_j in registers for the whole process instead of
// reading them back from V at every sweep and dot product (V is still written: the combination
// step reads it).  The sweeps, dot products and reductions are those of arn_half1, arn_half2 and
// slice_dots in the same order, so the results are bitwise the memory form's (and the
// barrier-free kernels', which share that form).  Loops over i <= j run over the register
// array with a uniform early exit, so every index is a compile-time one.
template <class T, int MV>
__device__ __forceinline__ void slice_dots_rv(const T (&vrow)[MV], T wk, bool has, int nv, T* dst,
                                              T (*sh)[ARN_MAXCOL]) {
    const int ncol = nv + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int c0 = 0; c0 < MV + 1; c0 += ARN_CHUNK) {
        if (c0 >= ncol) break;   // uniform
        T v[ARN_CHUNK];
#pragma unroll
        for (int i = 0; i < ARN_CHUNK; ++i) v[i] = 0.0;
        if (has) {
#pragma unroll
            for (int i = 0; i < ARN_CHUNK; ++i) {
                const int col = c0 + i;
                if (col < MV && col < nv)
                    v[i] = fma_t(vrow[col < MV ? col : 0], wk, v[i]);
                else if (col == nv)
                    v[i] = fma_t(wk, wk, v[i]);
            }
        }
        int c = 0;
        const T x = warp_sum8<T>(v, lane, &c);
        if ((lane & 3) == 0 && c0 + c < ncol) sh[warp][c0 + c] = x;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < ncol; c += ARN_THREADS) {
        T s = 0.0;
        for (int wv = 0; wv < ARN_WARPS; ++wv) s += sh[wv][c];
        dst[c] = s;
    }
}

template <class T, int MV>
__device__ __forceinline__ void arn_half1_rv(int j, int nb, int stride, const T (&vrow)[MV], bool has, int64_t k,
                                             T* w, T& wk, const T* partA, T* partB_blk,
                                             T* h1, T (*sh)[ARN_MAXCOL]) {
    reduce_cols<T>(partA, nb, stride, j + 2, h1, sh);
    T s = 0.0;
    if (has) {
        s = w[k];
#pragma unroll
        for (int i = 0; i < MV; ++i) {
            if (i > j) break;   // uniform
            s = fma_t(-h1[i], vrow[i], s);
        }
        w[k] = s;
    }
    wk = s;
    __syncthreads();
    slice_dots_rv<T, MV>(vrow, s, has, j + 1, partB_blk, sh);
}

template <class T, int MV>
__device__ __forceinline__ bool arn_half2_rv(int j, int m, int64_t K0, int64_t k, bool has, int nb, int stride,
                                             int NF, const double* __restrict__ bsr, const int* __restrict__ nbr,
                                             const double* __restrict__ dt, T* V, T (&vrow)[MV], T w1k,
                                             const T* w1, T* wn, double* H, T* Hs, const T* partB,
                                             T* partA_blk, const T* h1, T* h2, T* cs,
                                             DevScalars* sc, T (*sh)[ARN_MAXCOL]) {
    reduce_cols<T>(partB, nb, stride, j + 2, h2, sh);
    T hh = 0.0;
    for (int i = 0; i <= j; ++i) hh = fma_t(h2[i], h2[i], hh);
    const T hn = sqrt(fmax(h2[j + 1] - hh, (T)0));
    const T w0 = sqrt(h1[j + 1]);
    const bool brk = !(hn > arn_breakdown_tol<T>() * w0);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = h1[i] + h2[i];
        H[(size_t)(j + 1) * m + j] = hn;
        sc->m_used = j + 1;
        sc->hsub = hn;
        sc->w0 = w0;
        if (!isfinite(hn)) sc->nonfinite = 1;
        if (brk) sc->broken = 1;
    }
    if (brk || j + 1 == m) return false;   // uniform: every block reduced the same values
    for (int i = threadIdx.x; i <= j + 1; i += ARN_THREADS) Hs[i * ARN_HLD + j] = i <= j ? h1[i] + h2[i] : hn;
    __syncthreads();
    const T ih = (T)1 / hn;
    for (int l = threadIdx.x; l <= j + 1; l += ARN_THREADS) {
        T c = 0.0;
        for (int i = (l > 0 ? l - 1 : 0); i <= j; ++i) c = fma_t(Hs[l * ARN_HLD + i], h2[i], c);
        cs[l] = c;
    }
    __syncthreads();
    T wnk = 0.0;
    if (has) {
        T s = w1k;
        T t = a_row<T>(k, NF, bsr, nbr, dt, w1);
#pragma unroll
        for (int i = 0; i < MV; ++i) {
            if (i > j) break;   // uniform
            const T vi = vrow[i];
            s = fma_t(-h2[i], vi, s);
            t = fma_t(-cs[i], vi, t);
        }
        const T v = s * ih;
        V[(size_t)(j + 1) * K0 + k] = v;
#pragma unroll
        for (int i = 0; i < MV; ++i)
            if (i == j + 1) vrow[i] = v;
        t = fma_t(-cs[j + 1], v, t);
        wnk = t * ih;
        wn[k] = wnk;
    }
    __syncthreads();
    slice_dots_rv<T, MV>(vrow, wnk, has, j + 2, partA_blk, sh);
    return true;
}

template <class T, int MV>
__global__ void __launch_bounds__(ARN_THREADS, 2) k_arnoldi_rv(int64_t K0, int E, int NF, int m,
                                                               const double* __restrict__ bsr,
                                                               const int* __restrict__ nbr,
                                                               const double* __restrict__ dt,
                                                               const double* __restrict__ r, T* __restrict__ V,
                                                               T* __restrict__ wbuf, double* __restrict__ H,
                                                               T* __restrict__ partA, T* __restrict__ partB,
                                                               T* __restrict__ partC, int stride, GridBar* bar,
                                                               long long budget, DevScalars* sc) {
    __shared__ T sh[ARN_WARPS][ARN_MAXCOL];
    __shared__ T h1[ARN_MAXCOL], h2[ARN_MAXCOL], cs[ARN_MAXCOL], red[8];
    __shared__ T Hs[(ARN_HLD + 1) * ARN_HLD];
    __shared__ int s_ok;
    unsigned epoch = 0;
    const unsigned nb = gridDim.x;
    const int64_t chunk = (K0 + nb - 1) / nb;   // <= ARN_THREADS (checked by the launcher)
    const int64_t k0 = (int64_t)blockIdx.x * chunk;
    const int64_t k1 = (k0 + chunk) < K0 ? (k0 + chunk) : K0;
    const int64_t k = k0 + threadIdx.x;
    const bool has = k < k1;
    T vrow[MV];
#pragma unroll
    for (int i = 0; i < MV; ++i) vrow[i] = 0.0;
    {
        T v[ARN_CHUNK] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (has) {
            const T x = dt[k / 5] * r[k];
            v[0] = fma_t(x, x, v[0]);
        }
        block_reduce_store<T>(v, 1, partC + (size_t)blockIdx.x * stride, sh);
    }
    if (!grid_sync(bar, nb, &epoch, budget, sc, &s_ok)) return;
    reduce_cols<T>(partC, nb, stride, 1, red, sh);
    const T beta = sqrt(red[0]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->beta = beta;
        sc->m_used = 0;
        sc->broken = (beta == 0.0 || !isfinite(beta)) ? 1 : 0;
        if (!isfinite(beta)) sc->nonfinite = 1;
    }
    if (beta == 0.0 || !isfinite(beta)) return;   // uniform across blocks
    const T ib = (T)1 / beta;
    if (has) {
        vrow[0] = dt[k / 5] * r[k] * ib;
        V[k] = vrow[0];
    }
    spmv_rows<T>(k0, k1, NF, bsr, nbr, dt, nullptr, r, ib, wbuf);   // A v_1 from the inputs: no barrier
    __syncthreads();
    slice_dots_rv<T, MV>(vrow, has ? wbuf[k] : 0.0, has, 1, partA + (size_t)blockIdx.x * stride, sh);
    for (int j = 0; j < m; ++j) {
        T* w = wbuf + (size_t)(j & 1) * K0;
        if (!grid_sync(bar, nb, &epoch, budget, sc, &s_ok)) return;
        T w1k = 0.0;
        arn_half1_rv<T, MV>(j, (int)nb, stride, vrow, has, k, w, w1k, partA, partB + (size_t)blockIdx.x * stride, h1, sh);
        if (!grid_sync(bar, nb, &epoch, budget, sc, &s_ok)) return;
        if (!arn_half2_rv<T, MV>(j, m, K0, k, has, (int)nb, stride, NF, bsr, nbr, dt, V, vrow, w1k, w,
                              wbuf + (size_t)((j + 1) & 1) * K0, H, Hs, partB, partA + (size_t)blockIdx.x * stride, h1,
                              h2, cs, sc, sh))
            break;
    }
}
constexpr int ARN_RV = 32;   // Krylov rows held in registers by k_arnoldi_rv (m <= 32)

// Two grid barriers per Krylov step (one per reduction).
template <class T>
__global__ void __launch_bounds__(ARN_THREADS) k_arnoldi(int64_t K0, int E, int NF, int m,
                                                         const double* __restrict__ bsr, const int* __restrict__ nbr,
                                                         const double* __restrict__ dt, const double* __restrict__ r,
                                                         T* __restrict__ V, T* __restrict__ wbuf,
                                                         double* __restrict__ H, T* __restrict__ partA,
                                                         T* __restrict__ partB, T* __restrict__ partC,
                                                         int stride, GridBar* bar, long long budget, DevScalars* sc) {
    __shared__ T sh[ARN_WARPS][ARN_MAXCOL];
    __shared__ T h1[ARN_MAXCOL], h2[ARN_MAXCOL], cs[ARN_MAXCOL], red[8];
    __shared__ T Hs[(ARN_HLD + 1) * ARN_HLD];
    __shared__ int s_ok;
    unsigned epoch = 0;   // barriers passed (thread 0's copy is the one used)
    const unsigned nb = gridDim.x;
    const int64_t chunk = (K0 + nb - 1) / nb;
    const int64_t k0 = (int64_t)blockIdx.x * chunk;
    const int64_t k1 = (k0 + chunk) < K0 ? (k0 + chunk) : K0;
    // start vector v_1 = N / ||N||, N = dt * r
    {
        T v[ARN_CHUNK] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int64_t k = k0 + threadIdx.x; k < k1; k += ARN_THREADS) {
            const T x = dt[k / 5] * r[k];
            v[0] = fma_t(x, x, v[0]);
        }
        block_reduce_store<T>(v, 1, partC + (size_t)blockIdx.x * stride, sh);
    }
    if (!grid_sync(bar, nb, &epoch, budget, sc, &s_ok)) return;
    reduce_cols<T>(partC, nb, stride, 1, red, sh);
    const T beta = sqrt(red[0]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->beta = beta;
        sc->m_used = 0;
        sc->broken = (beta == 0.0 || !isfinite(beta)) ? 1 : 0;
        if (!isfinite(beta)) sc->nonfinite = 1;
    }
    if (beta == 0.0 || !isfinite(beta)) return;   // uniform across blocks
    const T ib = (T)1 / beta;
    for (int64_t k = k0 + threadIdx.x; k < k1; k += ARN_THREADS) V[k] = dt[k / 5] * r[k] * ib;
    spmv_rows<T>(k0, k1, NF, bsr, nbr, dt, nullptr, r, ib, wbuf);   // A v_1 from the inputs: no barrier
    __syncthreads();
    slice_dots<T>(V, wbuf, K0, k0, k1, 1, 1, partA + (size_t)blockIdx.x * stride, sh);
    for (int j = 0; j < m; ++j) {
        T* w = wbuf + (size_t)(j & 1) * K0;
        if (!grid_sync(bar, nb, &epoch, budget, sc, &s_ok)) return;
        arn_half1<T>(j, K0, k0, k1, (int)nb, stride, V, w, partA, partB + (size_t)blockIdx.x * stride, h1, sh);
        if (!grid_sync(bar, nb, &epoch, budget, sc, &s_ok)) return;
        if (!arn_half2<T>(j, m, K0, k0, k1, (int)nb, stride, NF, bsr, nbr, dt, V, w, wbuf + (size_t)((j + 1) & 1) * K0, H,
                       Hs, partB, partA + (size_t)blockIdx.x * stride, h1, h2, cs, sc, sh))
            break;
    }
}

// ---- the same Arnoldi process without grid barriers ----------------------------------------
// Kernel boundaries take the place of the persistent kernel's grid barriers: a start kernel
// (norm partials of N), an init kernel (beta, v_1, A v_1, first dot sweep) and two kernels
// per Krylov step (the two halves above).  Each block does exactly the persistent kernel's work on the same slice, with the
// same block count, so the Krylov basis and H are bitwise the same; no block ever waits for
// another, so nothing depends on the blocks being co-resident (several contexts sharing the
// device).  h1 travels between kernels through hcol[]; a kernel that finds the process
// ended (breakdown or a zero start vector) returns at once.
template <class T>
struct ArnArgs {
    int64_t K0;
    int NF, m, stride;
    const double* bsr;
    const int* nbr;
    const double* dt;
    const double* r;
    T* V;
    T* wbuf;
    double* H;
    double* hcol;
    T* partA;
    T* partB;
    T* partC;
    DevScalars* sc;
};

__device__ __forceinline__ void arn_slice(int64_t K0, int64_t* k0, int64_t* k1) {
    const unsigned nb = gridDim.x;
    const int64_t chunk = (K0 + nb - 1) / nb;
    *k0 = (int64_t)blockIdx.x * chunk;
    *k1 = (*k0 + chunk) < K0 ? (*k0 + chunk) : K0;
}

template <class T>
__global__ void __launch_bounds__(ARN_THREADS) k_arn_start(ArnArgs<T> A) {
    __shared__ T sh[ARN_WARPS][ARN_MAXCOL];
    int64_t k0, k1;
    arn_slice(A.K0, &k0, &k1);
    T v[ARN_CHUNK] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t k = k0 + threadIdx.x; k < k1; k += ARN_THREADS) {
        const T x = A.dt[k / 5] * A.r[k];
        v[0] = fma_t(x, x, v[0]);
    }
    block_reduce_store<T>(v, 1, A.partC + (size_t)blockIdx.x * A.stride, sh);
}

template <class T>
__global__ void __launch_bounds__(ARN_THREADS) k_arn_init(ArnArgs<T> A) {
    __shared__ T sh[ARN_WARPS][ARN_MAXCOL];
    __shared__ T red[8];
    int64_t k0, k1;
    arn_slice(A.K0, &k0, &k1);
    const int nb = (int)gridDim.x;
    reduce_cols<T>(A.partC, nb, A.stride, 1, red, sh);
    const T beta = sqrt(red[0]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.sc->beta = beta;
        A.sc->m_used = 0;
        A.sc->broken = (beta == 0.0 || !isfinite(beta)) ? 1 : 0;
        if (!isfinite(beta)) A.sc->nonfinite = 1;
    }
    if (beta == 0.0 || !isfinite(beta)) return;
    const T ib = (T)1 / beta;
    for (int64_t k = k0 + threadIdx.x; k < k1; k += ARN_THREADS) A.V[k] = A.dt[k / 5] * A.r[k] * ib;
    spmv_rows<T>(k0, k1, A.NF, A.bsr, A.nbr, A.dt, nullptr, A.r, ib, A.wbuf);
    __syncthreads();
    slice_dots<T>(A.V, A.wbuf, A.K0, k0, k1, 1, 1, A.partA + (size_t)blockIdx.x * A.stride, sh);
}

// step j, first half (h1 reaches the second half through hcol[])
template <class T>
__global__ void __launch_bounds__(ARN_THREADS) k_arn_half1(ArnArgs<T> A, int j) {
    __shared__ T sh[ARN_WARPS][ARN_MAXCOL];
    __shared__ T h1[ARN_MAXCOL];
    if (*((volatile int*)&A.sc->broken)) return;
    int64_t k0, k1;
    arn_slice(A.K0, &k0, &k1);
    T* w = A.wbuf + (size_t)(j & 1) * A.K0;
    arn_half1<T>(j, A.K0, k0, k1, (int)gridDim.x, A.stride, A.V, w, A.partA, A.partB + (size_t)blockIdx.x * A.stride,
              h1, sh);
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < j + 2; i += ARN_THREADS) A.hcol[i] = h1[i];
}

// step j, second half
template <class T>
__global__ void __launch_bounds__(ARN_THREADS) k_arn_half2(ArnArgs<T> A, int j) {
    __shared__ T sh[ARN_WARPS][ARN_MAXCOL];
    __shared__ T h1[ARN_MAXCOL], h2[ARN_MAXCOL], cs[ARN_MAXCOL];
    __shared__ T Hs[(ARN_HLD + 1) * ARN_HLD];
    if (*((volatile int*)&A.sc->broken)) return;
    int64_t k0, k1;
    arn_slice(A.K0, &k0, &k1);
    for (int i = threadIdx.x; i < j + 2; i += ARN_THREADS) h1[i] = __ldcg(A.hcol + i);
    // columns 0..j-1 of H (written by earlier kernels)
    for (int t = threadIdx.x; t < (j + 1) * j; t += ARN_THREADS) {
        const int r = t / (j > 0 ? j : 1), cc = t % (j > 0 ? j : 1);
        Hs[r * ARN_HLD + cc] = __ldcg(A.H + (size_t)r * A.m + cc);
    }
    __syncthreads();
    const T* w1 = A.wbuf + (size_t)(j & 1) * A.K0;
    T* wn = A.wbuf + (size_t)((j + 1) & 1) * A.K0;
    arn_half2<T>(j, A.m, A.K0, k0, k1, (int)gridDim.x, A.stride, A.NF, A.bsr, A.nbr, A.dt, A.V, w1, wn, A.H, Hs,
              A.partB, A.partA + (size_t)blockIdx.x * A.stride, h1, h2, cs, A.sc, sh);
}

// Self-test of the bounded wait: one block waits at a barrier sized for two blocks, so
// the arrival it waits for never comes and the wait must give up by itself.
__global__ void k_barrier_selftest(GridBar* bar, long long budget, DevScalars* sc) {
    __shared__ int s_ok;
    unsigned epoch = 0;
    grid_sync(bar, 2u, &epoch, budget, sc, &s_ok);
}

emg_status selftest_barrier_timeout(emg_ctx* c, int* timed_out) {
    GridBar* bar = reinterpret_cast<GridBar*>(c->bar);
    EMG_CUDA_TRY(c, cudaMemsetAsync(bar, 0, sizeof(GridBar), c->stream));
    {
        ProfScope _ps(c, PC_CONTROL);
        k_barrier_selftest<<<1, 32, 0, c->stream>>>(bar, 200000000LL, c->sc);   // ~0.1 s of SM clock
    }
    EMG_CHECK_LAUNCH(c);
    int flag = 0;
    EMG_CUDA_TRY(c, cudaMemcpyAsync(&flag, &c->sc->timeout, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    EMG_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    *timed_out = flag;
    EMG_CUDA_TRY(c, cudaMemsetAsync(&c->sc->timeout, 0, sizeof(int), c->stream));
    EMG_CUDA_TRY(c, cudaMemsetAsync(bar, 0, sizeof(GridBar), c->stream));
    return EMG_OK;
}

struct Pade13 {
    double b[14];
};

constexpr int PHI_CLUSTER = 8;   // blocks (one per SM) sharing the dense products of k_phi

// C = A B on n x n shared matrices with leading dimension ld, split over the cluster: block
// r forms a contiguous range of the entries (each entry summed in k order by one thread,
// as on a single block) and stores it into C of every block of the cluster.  The first
// barrier keeps the stores from overwriting a C that a slower block still reads.
__device__ __forceinline__ void smm(const double* A, const double* B, double* C, int n, int ld) {
    cg::cluster_group cl = cg::this_cluster();
    const int nr = (int)cl.num_blocks(), rk = (int)cl.block_rank();
    const int tot = n * n, per = (tot + nr - 1) / nr;
    const int t0 = rk * per, t1 = (t0 + per) < tot ? (t0 + per) : tot;
    cl.sync();
    for (int t = t0 + (int)threadIdx.x; t < t1; t += (int)blockDim.x) {
        const int i = t / n, j = t % n;
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += A[i * ld + k] * B[k * ld + j];
        for (int r = 0; r < nr; ++r) cl.map_shared_rank(C, r)[i * ld + j] = s;
    }
    cl.sync();
}

// EST = false: y = beta * [exp([[H_k, e1], [0, 0]])]_{0:k, k} with k = sc->m_used (the
// phi_1 weights of Eq. final).
// EST = true: the Krylov tolerance test after Arnoldi step jstep (k = jstep + 1 steps, unless the
// process has already ended): X = exp([[H_k, e1, 0], [0, 0, 1], [0, 0, 0]]) holds phi_1(H_k)e1
// and phi_2(H_k)e1 in its last two columns; when h_{k+1,k} |(phi_2(H_k)e1)_k| <= tol
// ||phi_1(H_k)e1|| the process ends with k steps (sc->broken = 1).
// A cluster of PHI_CLUSTER blocks: the dense products (bound by one SM's FP64 rate on a
// single block) are shared out; the cheap element-wise steps and the small pivoted solve
// are repeated in every block on its own copies, so every block holds the same matrices
// and block 0 writes the result.
template <bool EST>
__global__ void __cluster_dims__(PHI_CLUSTER, 1, 1)
    k_phi(int m, int jstep, double tol, const double* __restrict__ H, double* __restrict__ y, Pade13 pc,
          DevScalars* sc) {
    extern __shared__ double sm[];
    const int k = EST ? jstep + 1 : sc->m_used;
    const double beta = sc->beta;
    if (k == 0) return;
    // uniform over the cluster: every block reads the same flags written by earlier kernels
    if (EST && (*((volatile int*)&sc->broken) || sc->m_used != k)) return;
    const int n = EST ? k + 2 : k + 1, ld = n;
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
        const int i = t / n, jj = t % n;
        double v = 0.0;
        if (i < k && jj < k && i <= jj + 1) v = H[(size_t)i * m + jj];   // the Hessenberg band only
        if (i == 0 && jj == k) v = 1.0;
        if (EST && i == k && jj == k + 1) v = 1.0;
        M[i * ld + jj] = v;
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
    // squarings: a non-finite norm (the Krylov data are not finite) takes none, and the count
    // is capped (2^-1100 underflows every double)
    int s = 0;
    if (isfinite(s_norm) && s_norm > theta13) s = (int)fmin(ceil(log2(s_norm / theta13)), 1100.0);
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
        if (threadIdx.x < 32) {
            // pivot: the first row (lowest index) of largest |T1[r][c]|, r >= c, by one warp
            double best = -1.0;
            int bi = c;
            for (int r = c + (int)threadIdx.x; r < n; r += 32) {
                const double v = fabs(T1[r * ld + c]);
                if (v > best) {
                    best = v;
                    bi = r;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
            }
            if (threadIdx.x == 0) s_piv = bi;
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
    if (cg::this_cluster().block_rank() == 0) {
        if (EST) {
            if (threadIdx.x == 0) {
                double nrm = 0.0;
                for (int i = 0; i < k; ++i) nrm += X[i * ld + k] * X[i * ld + k];
                const double err = H[(size_t)k * m + (k - 1)] * fabs(X[(k - 1) * ld + k + 1]);
                if (err <= tol * sqrt(nrm)) sc->broken = 1;
            }
        } else {
            for (int i = threadIdx.x; i < k; i += blockDim.x) y[i] = beta * X[i * ld + k];
        }
    }
}

// out = u0 + V[0:k]^T y  (out = u0 when the start vector was zero)
template <class TV>
__global__ void k_combine(int64_t K0, const double* __restrict__ u0, const TV* __restrict__ V,
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

// ---- ordering of cooperative launches across contexts ---------------------------------------
// The Arnoldi kernel spins at grid barriers until every one of its blocks is resident.  Two
// such kernels of different contexts (streams) running at once could each hold part of the
// device while waiting for the rest.  All cooperative launches on a device are therefore
// chained through one event: each waits for the previous one before it starts.
namespace {
struct CoopGate {
    std::mutex mu;
    cudaEvent_t ev = nullptr;
    bool recorded = false;
};
CoopGate g_gate[64];
}  // namespace

emg_status coop_ordered(int device, cudaStream_t st, const std::function<cudaError_t()>& launch, std::string* err) {
    CoopGate& g = g_gate[device & 63];
    std::lock_guard<std::mutex> lk(g.mu);
    cudaError_t e = cudaSuccess;
    if (!g.ev) e = cudaEventCreateWithFlags(&g.ev, cudaEventDisableTiming);
    if (e == cudaSuccess && g.recorded) e = cudaStreamWaitEvent(st, g.ev, 0);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(g.ev, st);
    if (e != cudaSuccess) {
        if (err) *err = std::string("cooperative launch: ") + cudaGetErrorString(e);
        return EMG_ERR_CUDA;
    }
    g.recorded = true;
    return EMG_OK;
}

// EXP1 inputs on p = 0: R~_0(u0) and the block rows of J_0.
emg_status launch_exp1_prepare(emg_ctx* c, const double* u0, const double* tau0) {
    emg_status st = launch_residual(c, 0, u0, tau0, c->lv[0].r);
    if (st != EMG_OK) return st;
    st = launch_face_jacobian(c, 0, u0);
    if (st != EMG_OK) return st;
    return launch_bsr0(c);
}

emg_status launch_exp1(emg_ctx* c, const double* u0, const double* tau0, const double* dt, double* out) {
    emg_status st = launch_exp1_prepare(c, u0, tau0);
    if (st != EMG_OK) return st;
    return launch_exp1_krylov(c, u0, dt, out);
}

// Arnoldi (one persistent cooperative kernel), phi_1 of the Hessenberg matrix, combination.
// While a graph is being captured the ordering of cooperative launches is left to the
// caller (the graph replay is ordered as a whole).
template <class T>
static emg_status exp1_krylov(emg_ctx* c, const double* u0, const double* dt, double* out) {
    LevelDev& L = c->lv[0];
    const int64_t K0 = 5 * c->E;
    const int m = c->prm.krylov_m;
    // one cooperative launch: every block must be co-resident for the grid barriers
    int per_sm = 0, nsm = 0, per_sm_rv = 0;
    EMG_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_arnoldi<T>, ARN_THREADS, 0));
    EMG_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_rv, k_arnoldi_rv<T, ARN_RV>, ARN_THREADS, 0));
    EMG_CUDA_TRY(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
    const int64_t nb = arnoldi_blocks(K0, nsm, per_sm, c->red_blocks);
    // rows in registers: one row per thread at most, every block co-resident, m <= ARN_RV
    const bool rows_in_regs = m <= ARN_RV && (K0 + nb - 1) / nb <= ARN_THREADS && nb <= (int64_t)nsm * per_sm_rv;
    const int stride = MAX_KRYLOV + 8;
    // the basis, products and partials in T (float: the same arrays, half of each used)
    T* partA = reinterpret_cast<T*>(c->partial);
    T* partB = partA + (size_t)c->red_blocks * stride;
    T* partC = partB + (size_t)c->red_blocks * stride;
    GridBar* bar = reinterpret_cast<GridBar*>(c->bar);
    EMG_CUDA_TRY(c, cudaMemsetAsync(bar, 0, sizeof(GridBar), c->stream));
    int64_t K0a = K0;
    int Ea = (int)c->E, NFa = 2 * c->dim, ma = m, stra = stride;
    const double* bsr = c->bsr;
    const int* nbr = c->elem_nbr;
    const double* rr = L.r;
    T* Vv = reinterpret_cast<T*>(c->V);
    T* ww = reinterpret_cast<T*>(c->w);
    double* HH = c->H;
    const double tol = c->prm.krylov_tol;
    if (!c->prm.coop_krylov || tol > 0.0) {
        // barrier-free form (same blocks, same arithmetic): 2 + 2m plain launches; with a
        // Krylov tolerance, the test of each step follows it (it may end the process)
        ArnArgs<T> A{K0, 2 * c->dim, m, stride, bsr, nbr, dt, rr, Vv, ww, HH, c->hcol, partA, partB, partC, c->sc};
        const unsigned g = (unsigned)nb;
        const size_t smem_est = (size_t)8 * (m + 2) * (m + 2) * sizeof(double);
        if (tol > 0.0)
            EMG_CUDA_TRY(c, cudaFuncSetAttribute(k_phi<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_est));
        { ProfScope _ps(c, PC_ARNOLDI); k_arn_start<T><<<g, ARN_THREADS, 0, c->stream>>>(A); }
        { ProfScope _ps(c, PC_ARNOLDI); k_arn_init<T><<<g, ARN_THREADS, 0, c->stream>>>(A); }
        for (int j = 0; j < m; ++j) {
            { ProfScope _ps(c, PC_ARNOLDI); k_arn_half1<T><<<g, ARN_THREADS, 0, c->stream>>>(A, j); }
            { ProfScope _ps(c, PC_ARNOLDI); k_arn_half2<T><<<g, ARN_THREADS, 0, c->stream>>>(A, j); }
            if (tol > 0.0 && j + 1 < m) {
                ProfScope _ps(c, PC_PHI);
                k_phi<true><<<PHI_CLUSTER, 256, smem_est, c->stream>>>(m, j, tol, c->H, c->y, pade13(), c->sc);
            }
        }
        EMG_CHECK_LAUNCH(c);
    } else {
        long long budget = 4000000000LL;   // about two seconds of SM clock per barrier wait
        DevScalars* scp = c->sc;
        void* args[] = {&K0a, &Ea, &NFa, &ma, (void*)&bsr, (void*)&nbr, (void*)&dt, (void*)&rr, &Vv, &ww, &HH,
                        &partA, &partB, &partC, &stra, &bar, &budget, &scp};
        {
            ProfScope _ps(c, PC_ARNOLDI);
            auto launch = [&]() {
                const void* fn = rows_in_regs ? (const void*)k_arnoldi_rv<T, ARN_RV> : (const void*)k_arnoldi<T>;
                return cudaLaunchCooperativeKernel(fn, dim3((unsigned)nb), dim3(ARN_THREADS), args, 0, c->stream);
            };
            if (c->capturing) {
                EMG_CUDA_TRY(c, launch());
            } else {
                emg_status so = coop_ordered(c->device, c->stream, launch, &c->err);
                if (so != EMG_OK) return so;
            }
        }
    }
    const int n = m + 1;
    const size_t smem = (size_t)8 * n * n * sizeof(double);
    EMG_CUDA_TRY(c, cudaFuncSetAttribute(k_phi<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    {
        ProfScope _ps(c, PC_PHI);
        k_phi<false><<<PHI_CLUSTER, 256, smem, c->stream>>>(m, 0, 0.0, c->H, c->y, pade13(), c->sc);
    }
    EMG_CHECK_LAUNCH(c);
    {
        ProfScope _ps(c, PC_COMBINE);
        k_combine<T><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(296, (K0 + 255) / 256)), 256, 0, c->stream>>>(
            K0, u0, Vv, c->y, c->sc, out);
    }
    EMG_CHECK_LAUNCH(c);
    return EMG_OK;
}

// The Krylov process in FP64, or in float32 arithmetic for the basis, products and reductions
// (emg_params.krylov_f32; the Hessenberg matrix, phi_1 and the combination stay FP64).
emg_status launch_exp1_krylov(emg_ctx* c, const double* u0, const double* dt, double* out) {
    return c->prm.krylov_f32 ? exp1_krylov<float>(c, u0, dt, out) : exp1_krylov<double>(c, u0, dt, out);
}

// ---- EXP1 step without any allocation --------------------------------------------------------
// For callers that must not allocate device memory once they are running (an application
// whose memory is handed out by its own pool, or a loop that may not take the device-wide
// synchronisation of cudaMalloc/cudaFree): the Krylov basis, the packed block rows, the
// reduction partials, the Hessenberg matrix and the barrier live in one file-scope device
// array of fixed size, so the call itself allocates nothing.
constexpr int64_t NA_MAX_ELEMS = 8192;
constexpr int NA_MAX_M = 40;
constexpr int NA_MAX_NF = 6;
constexpr int NA_BLOCKS = 320;
constexpr int NA_STRIDE = MAX_KRYLOV + 8;
constexpr int64_t NA_K0 = 5 * NA_MAX_ELEMS;
constexpr size_t NA_OFF_V = 0;
constexpr size_t NA_OFF_W = NA_OFF_V + (size_t)(NA_MAX_M + 1) * NA_K0;
constexpr size_t NA_OFF_BSR = NA_OFF_W + 2 * (size_t)NA_K0;
constexpr size_t NA_OFF_NBR = NA_OFF_BSR + (size_t)NA_MAX_ELEMS * (1 + NA_MAX_NF) * 25;
constexpr size_t NA_OFF_H = NA_OFF_NBR + (size_t)NA_MAX_ELEMS * NA_MAX_NF / 2;
constexpr size_t NA_OFF_Y = NA_OFF_H + (size_t)(NA_MAX_M + 1) * NA_MAX_M;
constexpr size_t NA_OFF_PART = NA_OFF_Y + NA_MAX_M + 8;
constexpr size_t NA_OFF_SC = NA_OFF_PART + (size_t)3 * NA_BLOCKS * NA_STRIDE;
constexpr size_t NA_OFF_BAR = NA_OFF_SC + 16;
static_assert(sizeof(DevScalars) <= 16 * sizeof(double), "cycle scalars outgrew their slot");
constexpr size_t NA_DOUBLES = NA_OFF_BAR + 8;   // about 26 MB

static __device__ __align__(256) double g_exp1_scratch[NA_DOUBLES];
static_assert(sizeof(DevScalars) <= 16 * sizeof(double), "scalars do not fit their slot");

// Device address of g_exp1_scratch for each device, looked up once per device (std::call_once,
// so concurrent first calls from several host threads are safe) with that device current.
static double* g_exp1_scratch_addr[64] = {};
static cudaError_t g_exp1_scratch_err[64] = {};
static std::once_flag g_exp1_scratch_once[64];

// Packs the block rows and narrows the neighbour table.  A neighbour index outside
// [-1, E) is replaced by -1 (so nothing out of range is ever read) and flagged.
__global__ void k_pack_bsr(int64_t E, int NF, const double* __restrict__ diag, const double* __restrict__ off,
                           const int64_t* __restrict__ nbr, double* __restrict__ bsr, int* __restrict__ nbr32,
                           DevScalars* sc) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= E * (1 + NF) * 25) return;
    const int64_t e = idx / ((1 + NF) * 25);
    const int r = (int)(idx % ((1 + NF) * 25));
    const int blk = r / 25, t = r % 25;
    bsr[idx] = blk == 0 ? diag[e * 25 + t] : off[(e * NF + blk - 1) * 25 + t];
    if (r < NF) {
        const int64_t nb = nbr[e * NF + r];
        const bool ok = nb >= -1 && nb < E;
        nbr32[e * NF + r] = ok ? (int)nb : -1;
        if (!ok) sc->bad_index = 1;
    }
}

}  // namespace emg

extern "C" emg_status emg_exp1_step_noalloc(int32_t dim, int64_t n_elems, const double* diag, const double* off,
                                            const int64_t* nbr, const double* r0, const double* dt,
                                            const double* u0, int32_t krylov_m, void* cuda_stream,
                                            double* u_out, int32_t* krylov_dim) {
    using namespace emg;
    if ((dim != 2 && dim != 3) || n_elems < 1 || n_elems > NA_MAX_ELEMS || krylov_m < 1 || krylov_m > NA_MAX_M ||
        !diag || !off || !nbr || !r0 || !dt || !u0 || !u_out)
        return EMG_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return EMG_ERR_CUDA;
    std::call_once(g_exp1_scratch_once[dev], [dev]() {
        void* p = nullptr;
        g_exp1_scratch_err[dev] = cudaGetSymbolAddress(&p, g_exp1_scratch);
        if (g_exp1_scratch_err[dev] == cudaSuccess && !p) g_exp1_scratch_err[dev] = cudaErrorInvalidSymbol;
        g_exp1_scratch_addr[dev] = static_cast<double*>(p);
    });
    if (g_exp1_scratch_err[dev] != cudaSuccess) return EMG_ERR_CUDA;
    double* S = g_exp1_scratch_addr[dev];
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int NF = 2 * dim;
    const int64_t E = n_elems, K0 = 5 * E;
    double* V = S + NA_OFF_V;
    double* w = S + NA_OFF_W;
    double* bsr = S + NA_OFF_BSR;
    int* nbr32 = reinterpret_cast<int*>(S + NA_OFF_NBR);
    double* H = S + NA_OFF_H;
    double* y = S + NA_OFF_Y;
    double* partA = S + NA_OFF_PART;
    double* partB = partA + (size_t)NA_BLOCKS * NA_STRIDE;
    double* partC = partB + (size_t)NA_BLOCKS * NA_STRIDE;
    DevScalars* sc = reinterpret_cast<DevScalars*>(S + NA_OFF_SC);
    GridBar* bar = reinterpret_cast<GridBar*>(S + NA_OFF_BAR);
    // the previous call's contents remain: clear the flags, the barrier and the Hessenberg
    // matrix (whose row stride is this call's krylov_m)
    if (cudaMemsetAsync(sc, 0, sizeof(DevScalars), st) != cudaSuccess) return EMG_ERR_CUDA;
    if (cudaMemsetAsync(bar, 0, sizeof(GridBar), st) != cudaSuccess) return EMG_ERR_CUDA;
    if (cudaMemsetAsync(H, 0, (size_t)(NA_MAX_M + 1) * NA_MAX_M * sizeof(double), st) != cudaSuccess)
        return EMG_ERR_CUDA;
    const int64_t npack = E * (1 + NF) * 25;
    k_pack_bsr<<<(unsigned)((npack + 255) / 256), 256, 0, st>>>(E, NF, diag, off, nbr, bsr, nbr32, sc);
    if (cudaGetLastError() != cudaSuccess) return EMG_ERR_CUDA;
    {
        // the neighbour table is checked before anything reads through it
        int bad = 0;
        if (cudaMemcpyAsync(&bad, &sc->bad_index, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return EMG_ERR_CUDA;
        if (bad) return EMG_ERR_ARG;
    }
    int per_sm = 0, nsm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_arnoldi<double>, ARN_THREADS, 0) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return EMG_ERR_CUDA;
    const int64_t nb = arnoldi_blocks(K0, nsm, per_sm, NA_BLOCKS);
    int64_t K0a = K0;
    int Ea = (int)E, NFa = NF, ma = krylov_m, stra = NA_STRIDE;
    const double* bsrc = bsr;
    const int* nbrc = nbr32;
    long long budget = 4000000000LL;
    void* args[] = {&K0a, &Ea, &NFa, &ma, (void*)&bsrc, (void*)&nbrc, (void*)&dt, (void*)&r0, &V, &w, &H,
                    &partA, &partB, &partC, &stra, &bar, &budget, &sc};
    auto launch = [&]() {
        return cudaLaunchCooperativeKernel((const void*)k_arnoldi<double>, dim3((unsigned)nb), dim3(ARN_THREADS), args, 0, st);
    };
    if (coop_ordered(dev, st, launch, nullptr) != EMG_OK) return EMG_ERR_CUDA;
    const int n = krylov_m + 1;
    const size_t smem = (size_t)8 * n * n * sizeof(double);
    if (cudaFuncSetAttribute(k_phi<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return EMG_ERR_CUDA;
    k_phi<false><<<PHI_CLUSTER, 256, smem, st>>>(krylov_m, 0, 0.0, H, y, pade13(), sc);
    k_combine<double><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(296, (K0 + 255) / 256)), 256, 0, st>>>(
        K0, u0, V, y, sc, u_out);
    if (cudaGetLastError() != cudaSuccess) return EMG_ERR_CUDA;
    DevScalars hs;
    if (cudaMemcpyAsync(&hs, sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return EMG_ERR_CUDA;
    if (krylov_dim) *krylov_dim = hs.m_used;
    if (hs.timeout) return EMG_ERR_TIMEOUT;
    if (hs.nonfinite) return EMG_ERR_NONFINITE;
    return EMG_OK;
}

namespace emg {
}  // namespace emg
