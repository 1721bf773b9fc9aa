// Batched element-block solves of the PRK smoother (Eq. prk_scalar):
//  * k_lu: LU factorisation with partial pivoting of every P_e = I/dtau_e - D_e, one CTA
//    per element with the block in shared memory; factors stored column-major so that the
//    substitutions read contiguous columns.
//  * k_stage: one warp per element: y = P_e^{-1} r_e (row swaps, unit-lower forward and
//    upper backward substitution), u^(k) = u^n + beta_k y.
// T is the block precision (double for the FP64 form, float for the FP32 block form);
// the residual r, u^n and u^(k) are always double.
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
            T best = (T)-1;
            int bi = k;
            for (int r = k + tid; r < B; r += 32) {
                const T v = fabs(a[r * LD + k]);
                if (v > best) {
                    best = v;
                    bi = r;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const T ob = __shfl_xor_sync(0xffffffffu, best, o);
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
        const T inv = (T)1 / a[k * LD + k];
        for (int r = k + 1 + tid; r < B; r += nth) a[r * LD + k] *= inv;
        __syncthreads();
        const int m = B - k - 1;
        for (int t = tid; t < m * m; t += nth) {
            const int r = k + 1 + t / m, cc = k + 1 + t % m;
            a[r * LD + cc] -= a[r * LD + k] * a[k * LD + cc];
        }
        __syncthreads();
    }
    // column-major out: g[col * B + row]
    for (int t = tid; t < B * B; t += nth) {
        const int cc = t / B, r = t % B;
        g[t] = a[r * LD + cc];
    }
}

template <int B, class T>
__global__ void __launch_bounds__(128) k_stage(int E, const T* __restrict__ lu, const int* __restrict__ piv,
                                               const double* __restrict__ r, const double* __restrict__ un,
                                               double beta, double* __restrict__ out) {
    __shared__ T ys[4][B];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int e = blockIdx.x * 4 + warp;
    if (e >= E) return;
    T* y = ys[warp];
    for (int t = lane; t < B; t += 32) y[t] = (T)r[(size_t)e * B + t];
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
    const T* M = lu + (size_t)e * B * B;
    for (int j = 0; j < B; ++j) {
        const T yj = y[j];
        const T* col = M + (size_t)j * B;
        for (int rr = j + 1 + lane; rr < B; rr += 32) y[rr] -= col[rr] * yj;
        __syncwarp();
    }
    for (int j = B - 1; j >= 0; --j) {
        const T* col = M + (size_t)j * B;
        const T xj = y[j] / col[j];
        __syncwarp();
        for (int rr = lane; rr < j; rr += 32) y[rr] -= col[rr] * xj;
        if (lane == 0) y[j] = xj;
        __syncwarp();
    }
    for (int t = lane; t < B; t += 32) out[(size_t)e * B + t] = un[(size_t)e * B + t] + beta * (double)y[t];
}

#define EMG_BSIZES(X) X(15) X(30) X(50) X(75) X(20) X(100) X(175)

template <class T>
static emg_status lu_dispatch(emg_ctx* c, int B, T* blk, int* piv) {
    const unsigned E = (unsigned)c->E;
    switch (B) {
#define EMG_LU_CASE(BB)                                                                                      \
    case BB: {                                                                                               \
        const size_t sm = LuCfg<BB, T>::SMEM;                                                                \
        if (sm > 227 * 1024) {                                                                               \
            c->err = "block of size " #BB " does not fit in shared memory in this precision";                \
            return EMG_ERR_ARG;                                                                              \
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

emg_status launch_lu32(emg_ctx* c, int p) { return lu_dispatch<float>(c, c->lv[p].B, c->lv[p].blk32, c->lv[p].piv); }

emg_status launch_stage(emg_ctx* c, int p, const double* r, const double* un, double beta, double* out) {
    LevelDev& L = c->lv[p];
    return stage_dispatch<double>(c, L.B, L.blk, L.piv, r, un, beta, out);
}

emg_status launch_stage32(emg_ctx* c, int p, const double* r, const double* un, double beta, double* out) {
    LevelDev& L = c->lv[p];
    return stage_dispatch<float>(c, L.B, L.blk32, L.piv, r, un, beta, out);
}

}  // namespace emg
