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

// Register-tiled Gauss-Jordan inversion with partial pivoting (FP32 block form).
// 256 threads = 32 (tx) x 8 (ty); thread (tx, ty) keeps rows ty + 8i and columns
// tx + 32j of the block in registers for the whole elimination.  Per pivot step only the
// pivot column (colk), the scaled pivot row (rowk) and, on a row interchange, the two
// swapped rows pass through shared memory.  The inverse is written column-major through
// a transposing shared tile so that the global stores are coalesced.
template <int B>
struct GjTile {
    static constexpr int RS = (B + 7) / 8;    // row slots per thread
    static constexpr int CS = (B + 31) / 32;  // column slots per thread
    static constexpr int LD = (B % 2) ? B + 2 : B + 1;   // odd stride of the output tile
    static constexpr size_t SMEM = (size_t)B * LD * sizeof(float);
};

template <int B>
__global__ void __launch_bounds__(256) k_gj_tile(int E, float* __restrict__ blk) {
    constexpr int RS = GjTile<B>::RS, CS = GjTile<B>::CS, LD = GjTile<B>::LD;
    constexpr int RP = 8 * RS, CP = 32 * CS;   // zero-padded extents: no bounds checks inside
    extern __shared__ __align__(16) unsigned char smraw[];
    float* tile = reinterpret_cast<float*>(smraw);
    __shared__ float colk[RP], rowk[CP], rowx[CP], rowy[CP];
    __shared__ int s_p;
    __shared__ int ipiv[B], colidx[B], pos[B];
    const int e = blockIdx.x;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    float* g = blk + (size_t)e * B * B;
    float a[RS][CS];
#pragma unroll
    for (int i = 0; i < RS; ++i)
#pragma unroll
        for (int j = 0; j < CS; ++j) {
            const int r = ty + 8 * i, c = tx + 32 * j;
            a[i][j] = (r < B && c < B) ? g[r * B + c] : 0.0f;
        }
    for (int t = threadIdx.x; t < RP; t += 256) colk[t] = 0.0f;
    for (int t = threadIdx.x; t < CP; t += 256) rowk[t] = rowx[t] = rowy[t] = 0.0f;
    __syncthreads();
    // fully unrolled for B <= 100: k, its row slot and column slot are compile-time,
    // so the register tile is indexed without runtime selects
    constexpr int UNR = B <= 100 ? B : 1;
#pragma unroll UNR
    for (int k = 0; k < B; ++k) {
        const int ki = k >> 3, kj = k >> 5;
        // (1) the pivot column, from the lane that owns column k in every warp
        if (tx == (k & 31)) {
#pragma unroll
            for (int i = 0; i < RS; ++i) {
                const int r = ty + 8 * i;
                float v = 0.0f;
#pragma unroll
                for (int j = 0; j < CS; ++j)
                    if (j == kj) {
                        v = a[i][j];
                        a[i][j] = 0.0f;   // column k is rebuilt by the update (in-place scheme)
                    }
                colk[r] = v;
            }
        }
        __syncthreads();
        // (2) pivot: largest |colk[r]|, r >= k, lowest index on ties
        if (threadIdx.x < 32) {
            float best = -1.0f;
            int bi = k;
            for (int r = k + tx; r < B; r += 32) {
                const float v = fabsf(colk[r]);
                if (v > best) {
                    best = v;
                    bi = r;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
            }
            if (tx == 0) {
                s_p = bi;
                ipiv[k] = bi;
            }
        }
        __syncthreads();
        const int p = s_p;
        // (3) interchange rows k and p
        if (p != k) {
            const int pi = p >> 3;
            if (ty == (k & 7)) {
#pragma unroll
                for (int j = 0; j < CS; ++j) {
                    float v = 0.0f;
#pragma unroll
                    for (int i = 0; i < RS; ++i)
                        if (i == ki) v = a[i][j];
                    rowx[tx + 32 * j] = v;
                }
            }
            if (ty == (p & 7)) {
#pragma unroll
                for (int j = 0; j < CS; ++j) {
                    float v = 0.0f;
#pragma unroll
                    for (int i = 0; i < RS; ++i)
                        if (i == pi) v = a[i][j];
                    rowy[tx + 32 * j] = v;
                }
            }
            if (threadIdx.x == 0) {
                const float t0 = colk[k];
                colk[k] = colk[p];
                colk[p] = t0;
            }
            __syncthreads();
            if (ty == (k & 7)) {
#pragma unroll
                for (int j = 0; j < CS; ++j) {
                    const float v = rowy[tx + 32 * j];
#pragma unroll
                    for (int i = 0; i < RS; ++i)
                        if (i == ki) a[i][j] = v;
                }
            }
            if (ty == (p & 7)) {
#pragma unroll
                for (int j = 0; j < CS; ++j) {
                    const float v = rowx[tx + 32 * j];
#pragma unroll
                    for (int i = 0; i < RS; ++i)
                        if (i == pi) a[i][j] = v;
                }
            }
        }
        // (4) the scaled pivot row (in-place Gauss-Jordan: column k becomes the inverse's)
        const float inv = 1.0f / colk[k];
        if (ty == (k & 7)) {
#pragma unroll
            for (int j = 0; j < CS; ++j) {
                float v = 0.0f;
#pragma unroll
                for (int i = 0; i < RS; ++i)
                    if (i == ki) v = a[i][j];
                const int c = tx + 32 * j;
                rowk[c] = (c == k ? 1.0f : v) * inv;
            }
        }
        __syncthreads();
        // (5) eliminate column k from every other row (padded rows have colk = 0)
        float rk[CS];
#pragma unroll
        for (int j = 0; j < CS; ++j) rk[j] = rowk[tx + 32 * j];
#pragma unroll
        for (int i = 0; i < RS; ++i) {
            if (ty + 8 * i == k) {
#pragma unroll
                for (int j = 0; j < CS; ++j) a[i][j] = rk[j];
            } else {
                const float f = colk[ty + 8 * i];
#pragma unroll
                for (int j = 0; j < CS; ++j) a[i][j] -= f * rk[j];
            }
        }
        __syncthreads();
    }
    // Undo the row interchanges as column interchanges in reverse order: position j of the
    // inverse holds working column colidx[j]; thread-owned column c goes to pos[c].
    if (threadIdx.x == 0) {
        for (int j = 0; j < B; ++j) colidx[j] = j;
        for (int k = B - 1; k >= 0; --k) {
            const int t0 = colidx[k];
            colidx[k] = colidx[ipiv[k]];
            colidx[ipiv[k]] = t0;
        }
        for (int j = 0; j < B; ++j) pos[colidx[j]] = j;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RS; ++i)
#pragma unroll
        for (int j = 0; j < CS; ++j) {
            const int r = ty + 8 * i, c = tx + 32 * j;
            if (r < B && c < B) tile[pos[c] * LD + r] = a[i][j];
        }
    __syncthreads();
    for (int t = threadIdx.x; t < B * B; t += 256) g[t] = tile[(t / B) * LD + (t % B)];
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

// FP32 block form: explicit inverse (Gauss-Jordan), applied by k_stage_gemv.
emg_status launch_lu32(emg_ctx* c, int p) {
    LevelDev& L = c->lv[p];
    const unsigned E = (unsigned)c->E;
    switch (L.B) {
#define EMG_GJ_CASE(BB)                                                                                      \
    case BB: {                                                                                               \
        const size_t sm = GjTile<BB>::SMEM;                                                                  \
        EMG_CUDA_TRY(c, cudaFuncSetAttribute(k_gj_tile<BB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)); \
        {                                                                                                    \
            ProfScope _ps(c, PC_LU);                                                                         \
            k_gj_tile<BB><<<E, 256, sm, c->stream>>>((int)E, L.blk32);                                       \
        }                                                                                                    \
        EMG_CHECK_LAUNCH(c);                                                                                 \
        return EMG_OK;                                                                                       \
    }
        EMG_BSIZES(EMG_GJ_CASE)
#undef EMG_GJ_CASE
        default:
            c->err = "unsupported block size";
            return EMG_ERR_ARG;
    }
}

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
