// Column-owner (unblocked) Gauss-Jordan inverses of the float32 block forms, plain and rotating,
// one variant per warp count; launched through gj_dispatch (gj.cu).
#include "blocks.cuh"
#include "common.cuh"
#include "gj.cuh"

namespace emg {

// Column-owner form of the same Gauss-Jordan inversion: W warps per element; lane tx owns
// rows tx + 32i, warp w owns columns w + W j.  At step k only the warp owning column k
// searches for the pivot (its lanes hold the whole column) and publishes the column and
// the pivot row index; every warp then takes the pivot row's entries for its own columns
// from lane (p mod 32) by shuffles.  One barrier per step (the published column is double
// buffered).  Pivot choice, tie rule and every multiply-add are those of k_gj_tile, so
// both forms give bitwise the same inverse.
template <int B, int W>
struct GjCols {
    static constexpr int RS = (B + 31) / 32;   // row slots per thread
    static constexpr int CS = (B + W - 1) / W; // column slots per thread
    static constexpr int LD = (B % 2) ? B + 2 : B + 1;
    static constexpr size_t SMEM = (size_t)B * LD * sizeof(float);
};

template <int B, int W>
__global__ void __launch_bounds__(32 * W) k_gj_cols(int E, float* __restrict__ blk) {
    using G = GjCols<B, W>;
    constexpr int RS = G::RS, CS = G::CS, LD = G::LD, T = 32 * W;
    extern __shared__ __align__(16) unsigned char smraw[];
    float* tile = reinterpret_cast<float*>(smraw);
    __shared__ float colk[2][32 * RS];
    __shared__ int s_p[2];
    __shared__ int perm[B], invp[B];
    const int e = blockIdx.x;
    const int tx = threadIdx.x & 31, w = threadIdx.x >> 5;
    float* g = blk + (size_t)e * B * B;
    for (int t = threadIdx.x; t < B * B; t += T) tile[(t / B) * LD + (t % B)] = g[t];
    __syncthreads();
    float a[RS][CS];
#pragma unroll
    for (int i = 0; i < RS; ++i)
#pragma unroll
        for (int j = 0; j < CS; ++j) {
            const int r = tx + 32 * i, c = w + W * j;
            a[i][j] = (r < B && c < B) ? tile[r * LD + c] : 0.0f;
        }
    unsigned used = 0u;   // bit i: row tx + 32 i has been a pivot row
#pragma unroll 1
    for (int k = 0; k < B; ++k) {
        const int kb = k & 1, wk = k % W, jk = k / W;
        if (w == wk) {
            // (1) column k (then zeroed: in-place scheme), pivot among the unused rows
            float v[RS];
            int best = -1;
            int bi = B, lo = B;
#pragma unroll
            for (int i = 0; i < RS; ++i) {
                float x = 0.0f;
#pragma unroll
                for (int j = 0; j < CS; ++j)
                    if (j == jk) {
                        x = a[i][j];
                        a[i][j] = 0.0f;
                    }
                v[i] = x;
                const int r = tx + 32 * i;
                if (r < B && !((used >> i) & 1u)) {
                    const int m = piv_key(x);
                    if (m > best) {
                        best = m;
                        bi = r;
                    }
                    if (r < lo) lo = r;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const int ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                const int ol = __shfl_xor_sync(0xffffffffu, lo, o);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
                lo = ol < lo ? ol : lo;
            }
            // no comparable candidate (a non-finite column): the lowest unused row
            const int p = bi < B ? bi : lo;
#pragma unroll
            for (int i = 0; i < RS; ++i) colk[kb][tx + 32 * i] = v[i];
            if (tx == 0) {
                s_p[kb] = p;
                perm[k] = p;
            }
        }
        __syncthreads();
        // (2) every warp: the scaled pivot row on its own columns, then the elimination
        const int p = s_p[kb];
        const float inv = 1.0f / colk[kb][p];
        const int pl = p & 31, pi = p >> 5;
        if (tx == pl) used |= 1u << pi;
        float f[RS];
#pragma unroll
        for (int i = 0; i < RS; ++i) f[i] = colk[kb][tx + 32 * i];
#pragma unroll
        for (int j = 0; j < CS; ++j) {
            float x = 0.0f;
#pragma unroll
            for (int i = 0; i < RS; ++i)
                if (i == pi) x = a[i][j];
            x = __shfl_sync(0xffffffffu, x, pl);
            const float rk = (w + W * j == k ? 1.0f : x) * inv;
#pragma unroll
            for (int i = 0; i < RS; ++i) {
                if (tx + 32 * i == p)
                    a[i][j] = rk;
                else
                    a[i][j] -= f[i] * rk;
            }
        }
    }
    // Row r of the working matrix holds row invp[r] of the inverse, and its column k holds
    // column perm[k]; written column-major through the shared tile.
    __syncthreads();
    for (int t = threadIdx.x; t < B; t += T) invp[perm[t]] = t;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RS; ++i)
#pragma unroll
        for (int j = 0; j < CS; ++j) {
            const int r = tx + 32 * i, c = w + W * j;
            if (r < B && c < B) tile[perm[c] * LD + invp[r]] = a[i][j];
        }
    __syncthreads();
    for (int t = threadIdx.x; t < B * B; t += T) g[t] = tile[(t / B) * LD + (t % B)];
}

// Rotating column-owner form: the layout of k_gj_cols, but after every W pivot steps each
// thread rotates its column slots by one, so that the pivot column of a step is always in
// register slot 0 of its owner warp (no runtime-indexed register access).  The pivot row
// slot (p / 32) is warp-uniform: it is taken by branching, not by select chains.  The
// multiply-adds and the pivot choice are those of k_gj_tile (bitwise the same inverse).
template <int B, int W>
__global__ void __launch_bounds__(32 * W) k_gj_rot(int E, float* __restrict__ blk) {
    using G = GjCols<B, W>;
    constexpr int RS = G::RS, CS = G::CS, LD = G::LD, T = 32 * W;
    extern __shared__ __align__(16) unsigned char smraw[];
    float* tile = reinterpret_cast<float*>(smraw);
    __shared__ float colk[2][32 * RS];
    __shared__ int s_p[2];
    __shared__ int perm[B], invp[B];
    const int e = blockIdx.x;
    const int tx = threadIdx.x & 31, w = threadIdx.x >> 5;
    float* g = blk + (size_t)e * B * B;
    for (int t = threadIdx.x; t < B * B; t += T) tile[(t / B) * LD + (t % B)] = g[t];
    __syncthreads();
    float a[RS][CS];
#pragma unroll
    for (int i = 0; i < RS; ++i)
#pragma unroll
        for (int j = 0; j < CS; ++j) {
            const int r = tx + 32 * i, c = w + W * j;
            a[i][j] = (r < B && c < B) ? tile[r * LD + c] : 0.0f;
        }
    unsigned used = 0u;
#pragma unroll 1
    for (int kb = 0; kb < CS; ++kb) {
#pragma unroll 1
        for (int wk = 0; wk < W; ++wk) {
            const int k = kb * W + wk;
            if (k >= B) break;   // uniform
            const int buf = k & 1;
            if (w == wk) {
                // (1) column k is slot 0 of this warp; zero it (in-place scheme) and pivot
                float v[RS];
                int best = -1;
                int bi = B, lo = B;
#pragma unroll
                for (int i = 0; i < RS; ++i) {
                    v[i] = a[i][0];
                    a[i][0] = 0.0f;
                    const int r = tx + 32 * i;
                    if (r < B && !((used >> i) & 1u)) {
                        const int m = piv_key(v[i]);
                        if (m > best) {
                            best = m;
                            bi = r;
                        }
                        if (r < lo) lo = r;
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const int ob = __shfl_xor_sync(0xffffffffu, best, o);
                    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                    const int ol = __shfl_xor_sync(0xffffffffu, lo, o);
                    if (ob > best || (ob == best && oi < bi)) {
                        best = ob;
                        bi = oi;
                    }
                    lo = ol < lo ? ol : lo;
                }
                const int p = bi < B ? bi : lo;   // lowest unused row if the column is not finite
#pragma unroll
                for (int i = 0; i < RS; ++i) colk[buf][tx + 32 * i] = v[i];
                if (tx == 0) {
                    s_p[buf] = p;
                    perm[k] = p;
                }
            }
            __syncthreads();
            // (2) the scaled pivot row on this warp's columns, by shuffles from lane p mod 32
            const int p = s_p[buf];
            const float inv = 1.0f / colk[buf][p];
            const int pl = p & 31, pi = p >> 5;
            if (tx == pl) used |= 1u << pi;
            float rk[CS];
#pragma unroll
            for (int c = 0; c < RS; ++c)
                if (pi == c) {   // warp-uniform branch
#pragma unroll
                    for (int j = 0; j < CS; ++j) rk[j] = __shfl_sync(0xffffffffu, a[c][j], pl) * inv;
                }
            if (w == wk) rk[0] = inv;   // column k: 1 / a_pk
            // (3) eliminate column k from every other row; row p becomes the scaled row
            float f[RS];
#pragma unroll
            for (int i = 0; i < RS; ++i) f[i] = (tx + 32 * i == p) ? 0.0f : colk[buf][tx + 32 * i];
#pragma unroll
            for (int i = 0; i < RS; ++i)
#pragma unroll
                for (int j = 0; j < CS; ++j) a[i][j] -= f[i] * rk[j];
            if (tx == pl) {
#pragma unroll
                for (int c = 0; c < RS; ++c)
                    if (pi == c) {
#pragma unroll
                        for (int j = 0; j < CS; ++j) a[c][j] = rk[j];
                    }
            }
        }
        // rotate the column slots: the next group's pivot columns move to slot 0
#pragma unroll
        for (int i = 0; i < RS; ++i) {
            const float t0 = a[i][0];
#pragma unroll
            for (int j = 0; j < CS - 1; ++j) a[i][j] = a[i][j + 1];
            a[i][CS - 1] = t0;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < B; t += T) invp[perm[t]] = t;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RS; ++i)
#pragma unroll
        for (int j = 0; j < CS; ++j) {
            const int r = tx + 32 * i, c = w + W * j;
            if (r < B && c < B) tile[perm[c] * LD + invp[r]] = a[i][j];
        }
    __syncthreads();
    for (int t = threadIdx.x; t < B * B; t += T) g[t] = tile[(t / B) * LD + (t % B)];
}

template <int B, int W>
cudaError_t gj_cols_go(unsigned E, float* blk, cudaStream_t st) {
    const size_t sm = GjCols<B, W>::SMEM;
    cudaError_t e = cudaFuncSetAttribute(k_gj_cols<B, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_gj_cols<B, W><<<E, 32 * W, sm, st>>>((int)E, blk);
    return cudaGetLastError();
}

template <int B, int W>
cudaError_t gj_rot_go(unsigned E, float* blk, cudaStream_t st) {
    const size_t sm = GjCols<B, W>::SMEM;
    cudaError_t e = cudaFuncSetAttribute(k_gj_rot<B, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_gj_rot<B, W><<<E, 32 * W, sm, st>>>((int)E, blk);
    return cudaGetLastError();
}

#define EMG_GJ_COLS_INST(BB)                                                        \
    template cudaError_t gj_cols_go<BB, 1>(unsigned, float*, cudaStream_t);         \
    template cudaError_t gj_cols_go<BB, 2>(unsigned, float*, cudaStream_t);         \
    template cudaError_t gj_cols_go<BB, 4>(unsigned, float*, cudaStream_t);         \
    template cudaError_t gj_cols_go<BB, 8>(unsigned, float*, cudaStream_t);         \
    template cudaError_t gj_cols_go<BB, 16>(unsigned, float*, cudaStream_t);        \
    template cudaError_t gj_rot_go<BB, 1>(unsigned, float*, cudaStream_t);          \
    template cudaError_t gj_rot_go<BB, 2>(unsigned, float*, cudaStream_t);          \
    template cudaError_t gj_rot_go<BB, 4>(unsigned, float*, cudaStream_t);          \
    template cudaError_t gj_rot_go<BB, 8>(unsigned, float*, cudaStream_t);          \
    template cudaError_t gj_rot_go<BB, 16>(unsigned, float*, cudaStream_t);
EMG_BSIZES(EMG_GJ_COLS_INST)
#undef EMG_GJ_COLS_INST

}  // namespace emg
