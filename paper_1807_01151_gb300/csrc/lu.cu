// Batched element-block solves of the PRK smoother (Eq. prk_scalar), FP64 form, and the
// stage GEMV of the float32 forms:
//  * k_lu: LU factorisation with partial pivoting of every P_e = I/dtau_e - D_e, one CTA
//    per element with the block in shared memory; factors stored column-major so that the
//    substitutions read contiguous columns (k_lu_gmem: the same in global memory for blocks
//    larger than shared memory).
//  * k_stage: one warp per element: y = P_e^{-1} r_e (row swaps, unit-lower forward and
//    upper backward substitution), u^(k) = u^n + beta_k y.
//  * k_stage_gemv: the same stage with the explicit inverse of the float32 forms (gj.cu).
// T is the block precision (double for the FP64 form, float for the FP32 block form);
// the residual r, u^n and u^(k) are always double.
#include "blocks.cuh"
#include "common.cuh"

namespace emg {
template <int B, class T>
struct LuCfg {
    static constexpr int LD = B + 1;                 // padded row stride in shared memory
    static constexpr size_t SMEM = (size_t)B * LD * sizeof(T);
};

template <int B, class T>
__global__ void __launch_bounds__(256) k_lu(int E, T* __restrict__ blk, int* __restrict__ piv) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T* a = reinterpret_cast<T*>(smraw);
    constexpr int LD = LuCfg<B, T>::LD;
    __shared__ int s_piv;
    const int e = blockIdx.x;
    const int tid = threadIdx.x, nth = blockDim.x;
    T* g = blk + (size_t)e * B * B;
    for (int t = tid; t < B * B; t += nth) a[(t / B) * LD + (t % B)] = g[t];
    __syncthreads();
    for (int k = 0; k < B; ++k) {
        if (tid < 32) {
            auto best = piv_key((T)0) - 1;   // every key is >= -1: a NaN row is taken only if no row is a number
            int bi = k;
            for (int r = k + tid; r < B; r += 32) {
                const auto v = piv_key(a[r * LD + k]);
                if (v > best) {
                    best = v;
                    bi = r;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const auto ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
            }
            if (tid == 0) {
                s_piv = bi;
                piv[(size_t)e * B + k] = bi;
            }
        }
        __syncthreads();
        const int pr = s_piv;
        if (pr != k)
            for (int cc = tid; cc < B; cc += nth) {
                const T t0 = a[k * LD + cc];
                a[k * LD + cc] = a[pr * LD + cc];
                a[pr * LD + cc] = t0;
            }
        __syncthreads();
        if (k + 1 + tid < B) {   // only the threads that scale a row pay for the division
            const T inv = (T)1 / a[k * LD + k];
            for (int r = k + 1 + tid; r < B; r += nth) a[r * LD + k] *= inv;
        }
        __syncthreads();
        // trailing update on a 32-wide column x 8-row thread grid (no index division)
        const int tx = tid & 31, ty = tid >> 5;
        for (int r = k + 1 + ty; r < B; r += 8) {
            const T l = a[r * LD + k];
            for (int cc = k + 1 + tx; cc < B; cc += 32) a[r * LD + cc] -= l * a[k * LD + cc];
        }
        __syncthreads();
    }
    // column-major out: g[col * B + row]
    for (int t = tid; t < B * B; t += nth) {
        const int cc = t / B, r = t % B;
        g[t] = a[r * LD + cc];
    }
}

// The same factorisation for blocks that do not fit in shared memory (B = 175 in float64):
// the block is factored in place in global memory (it stays in L2 while its CTA works on it),
// row-major during the elimination, then transposed in place to the column-major layout the
// substitutions read.  Pivot choice and tie rule as in k_lu.
template <int B, class T>
__global__ void __launch_bounds__(256) k_lu_gmem(int E, T* __restrict__ blk, int* __restrict__ piv) {
    __shared__ int s_piv;
    const int e = blockIdx.x;
    const int tid = threadIdx.x, nth = blockDim.x;
    T* a = blk + (size_t)e * B * B;
    for (int k = 0; k < B; ++k) {
        if (tid < 32) {
            auto best = piv_key((T)0) - 1;
            int bi = k;
            for (int r = k + tid; r < B; r += 32) {
                const auto v = piv_key(a[(size_t)r * B + k]);
                if (v > best) {
                    best = v;
                    bi = r;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const auto ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
            }
            if (tid == 0) {
                s_piv = bi;
                piv[(size_t)e * B + k] = bi;
            }
        }
        __syncthreads();
        const int pr = s_piv;
        if (pr != k)
            for (int cc = tid; cc < B; cc += nth) {
                const T t0 = a[(size_t)k * B + cc];
                a[(size_t)k * B + cc] = a[(size_t)pr * B + cc];
                a[(size_t)pr * B + cc] = t0;
            }
        __syncthreads();
        if (k + 1 + tid < B) {
            const T inv = (T)1 / a[(size_t)k * B + k];
            for (int r = k + 1 + tid; r < B; r += nth) a[(size_t)r * B + k] *= inv;
        }
        __syncthreads();
        const int tx = tid & 31, ty = tid >> 5;
        for (int r = k + 1 + ty; r < B; r += 8) {
            const T l = a[(size_t)r * B + k];
            for (int cc = k + 1 + tx; cc < B; cc += 32) a[(size_t)r * B + cc] -= l * a[(size_t)k * B + cc];
        }
        __syncthreads();
    }
    // row-major -> column-major, in place
    for (int t = tid; t < B * B; t += nth) {
        const int r = t / B, cc = t % B;
        if (r < cc) {
            const T t0 = a[(size_t)r * B + cc];
            a[(size_t)r * B + cc] = a[(size_t)cc * B + r];
            a[(size_t)cc * B + r] = t0;
        }
    }
}

template <int B, class T>
__global__ void __launch_bounds__(128) k_stage(int E, const T* __restrict__ lu, const int* __restrict__ piv,
                                               const double* __restrict__ r, const double* __restrict__ un,
                                               double beta, double* __restrict__ out) {
    __shared__ T ys[4][B];
    __shared__ T rd[4][B];   // reciprocals of U's diagonal
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int e = blockIdx.x * 4 + warp;
    if (e >= E) return;
    T* y = ys[warp];
    const T* M = lu + (size_t)e * B * B;
    // the B divisions of the back substitution, done once and in parallel across the lanes
    // (a division costs a warp-wide multi-instruction sequence on the FP64 pipe)
    for (int t = lane; t < B; t += 32) {
        y[t] = (T)r[(size_t)e * B + t];
        rd[warp][t] = (T)1 / M[(size_t)t * B + t];
    }
    __syncwarp();
    if (lane == 0) {
        const int* pv = piv + (size_t)e * B;
        for (int k = 0; k < B; ++k) {
            const int p = pv[k];
            if (p != k) {
                const T t0 = y[k];
                y[k] = y[p];
                y[p] = t0;
            }
        }
    }
    __syncwarp();
    for (int j = 0; j < B; ++j) {
        const T yj = y[j];
        const T* col = M + (size_t)j * B;
        for (int rr = j + 1 + lane; rr < B; rr += 32) y[rr] -= col[rr] * yj;
        __syncwarp();
    }
    for (int j = B - 1; j >= 0; --j) {
        const T* col = M + (size_t)j * B;
        const T xj = y[j] * rd[warp][j];
        __syncwarp();
        for (int rr = lane; rr < j; rr += 32) y[rr] -= col[rr] * xj;
        if (lane == 0) y[j] = xj;
        __syncwarp();
    }
    for (int t = lane; t < B; t += 32) out[(size_t)e * B + t] = un[(size_t)e * B + t] + beta * (double)y[t];
}

// u^(k) = u^n + beta P_e^{-1} r_e with P_e^{-1} column-major: one warp per element, each
// lane owns rows lane, lane+32, ...; every column is a coalesced read.
template <int B, class T>
__global__ void __launch_bounds__(128) k_stage_gemv(int E, const T* __restrict__ inv, const double* __restrict__ r,
                                                    const double* __restrict__ un, double beta,
                                                    double* __restrict__ out) {
    constexpr int RPL = (B + 31) / 32;
    __shared__ T rs[4][B];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int e = blockIdx.x * 4 + warp;
    if (e >= E) return;
    for (int t = lane; t < B; t += 32) rs[warp][t] = (T)r[(size_t)e * B + t];
    __syncwarp();
    T acc[RPL];
#pragma unroll
    for (int t = 0; t < RPL; ++t) acc[t] = (T)0;
    const T* M = inv + (size_t)e * B * B;
#pragma unroll 4
    for (int j = 0; j < B; ++j) {
        const T rj = rs[warp][j];
        const T* col = M + (size_t)j * B;
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
            const int i = lane + 32 * t;
            if (i < B) acc[t] += __ldg(col + i) * rj;
        }
    }
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
        const int i = lane + 32 * t;
        if (i < B) out[(size_t)e * B + i] = un[(size_t)e * B + i] + beta * (double)acc[t];
    }
}


template <class T>
static emg_status lu_dispatch(emg_ctx* c, int B, T* blk, int* piv) {
    const unsigned E = (unsigned)c->E;
    switch (B) {
#define EMG_LU_CASE(BB)                                                                                      \
    case BB: {                                                                                               \
        const size_t sm = LuCfg<BB, T>::SMEM;                                                                \
        if (sm > 227 * 1024) {                                                                               \
            ProfScope _ps(c, PC_LU);                                                                         \
            k_lu_gmem<BB, T><<<E, 256, 0, c->stream>>>((int)E, blk, piv);                                   \
            EMG_CHECK_LAUNCH(c);                                                                             \
            return EMG_OK;                                                                                   \
        }                                                                                                    \
        EMG_CUDA_TRY(c, cudaFuncSetAttribute(k_lu<BB, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)); \
        {                                                                                                    \
            ProfScope _ps(c, PC_LU);                                                                         \
            k_lu<BB, T><<<E, 256, sm, c->stream>>>((int)E, blk, piv);                                        \
        }                                                                                                    \
        EMG_CHECK_LAUNCH(c);                                                                                 \
        return EMG_OK;                                                                                       \
    }
        EMG_BSIZES(EMG_LU_CASE)
#undef EMG_LU_CASE
        default:
            c->err = "unsupported block size";
            return EMG_ERR_ARG;
    }
}

template <class T>
static emg_status stage_dispatch(emg_ctx* c, int B, const T* lu, const int* piv, const double* r, const double* un,
                                 double beta, double* out) {
    const unsigned E = (unsigned)c->E;
    switch (B) {
#define EMG_ST_CASE(BB)                                                                          \
    case BB: {                                                                                   \
        ProfScope _ps(c, PC_STAGE);                                                              \
        k_stage<BB, T><<<(E + 3) / 4, 128, 0, c->stream>>>((int)E, lu, piv, r, un, beta, out);   \
    }                                                                                            \
        EMG_CHECK_LAUNCH(c);                                                                     \
        return EMG_OK;
        EMG_BSIZES(EMG_ST_CASE)
#undef EMG_ST_CASE
        default:
            c->err = "unsupported block size";
            return EMG_ERR_ARG;
    }
}

emg_status launch_lu(emg_ctx* c, int p) { return lu_dispatch<double>(c, c->lv[p].B, c->lv[p].blk, c->lv[p].piv); }

emg_status launch_stage(emg_ctx* c, int p, const double* r, const double* un, double beta, double* out) {
    LevelDev& L = c->lv[p];
    return stage_dispatch<double>(c, L.B, L.blk, L.piv, r, un, beta, out);
}

emg_status launch_stage32(emg_ctx* c, int p, const double* r, const double* un, double beta, double* out) {
    LevelDev& L = c->lv[p];
    const unsigned E = (unsigned)c->E;
    switch (L.B) {
#define EMG_GV_CASE(BB)                                                                                  \
    case BB: {                                                                                           \
        ProfScope _ps(c, PC_STAGE);                                                                      \
        k_stage_gemv<BB, float><<<(E + 3) / 4, 128, 0, c->stream>>>((int)E, L.blk32, r, un, beta, out);  \
    }                                                                                                    \
        EMG_CHECK_LAUNCH(c);                                                                             \
        return EMG_OK;
        EMG_BSIZES(EMG_GV_CASE)
#undef EMG_GV_CASE
        default:
            c->err = "unsupported block size";
            return EMG_ERR_ARG;
    }
}

}  // namespace emg
