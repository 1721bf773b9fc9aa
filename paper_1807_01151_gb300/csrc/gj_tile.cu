// Register-tiled (unblocked) Gauss-Jordan inverse of the float32 block forms, one variant per
// pivot-loop unrolling; launched through gj_dispatch (gj.cu).
#include "blocks.cuh"
#include "common.cuh"
#include "gj.cuh"

namespace emg {

// Register-tiled Gauss-Jordan inversion with partial pivoting (FP32 block form).
// 256 threads = 32 (tx) x 8 (ty); thread (tx, ty) keeps rows ty + 8i and columns
// tx + 32j of the block in registers for the whole elimination.  Pivoting is implicit:
// rows never move; step k takes the unused row p with the largest |a_pk| (lowest index on
// ties) as its pivot row, and the permutation is applied when the inverse is stored.  Per
// step only the pivot column and the scaled pivot row pass through shared memory, double
// buffered, so a step needs two barriers.  Every warp finds the pivot itself from the
// shared column (the same data in the same order, hence the same row).  The inverse is
// written column-major through a transposing shared tile so that the stores coalesce.
template <int B>
struct GjTile {
    static constexpr int RS = (B + 7) / 8;    // row slots per thread
    static constexpr int CS = (B + 31) / 32;  // column slots per thread
    static constexpr int LD = (B % 2) ? B + 2 : B + 1;   // odd stride of the output tile
    static constexpr size_t SMEM = (size_t)B * LD * sizeof(float);
};

template <int B, int UNR>
__global__ void __launch_bounds__(256) k_gj_tile(int E, float* __restrict__ blk) {
    constexpr int RS = GjTile<B>::RS, CS = GjTile<B>::CS, LD = GjTile<B>::LD;
    constexpr int RP = 8 * RS, CP = 32 * CS;   // zero-padded extents: no bounds checks inside
    constexpr int MW = (B + 31) / 32;          // words of the used-row mask
    extern __shared__ __align__(16) unsigned char smraw[];
    float* tile = reinterpret_cast<float*>(smraw);
    __shared__ float colk[2][RP], rowk[2][CP];
    __shared__ int perm[B], invp[B];
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
    unsigned used[MW];
#pragma unroll
    for (int m = 0; m < MW; ++m) used[m] = 0u;
    // UNR steps per unrolled body: a variant parameter (the arithmetic is the same for every
    // UNR; full unrolling makes k compile-time but the code can outgrow the instruction cache)
#pragma unroll UNR
    for (int k = 0; k < B; ++k) {
        const int kb = k & 1, kj = k >> 5;
        float* ck = colk[kb];
        float* rk_s = rowk[kb];
        // (1) the pivot column, from the lane that owns column k (column k is then rebuilt
        //     by the update: in-place scheme)
        if (tx == (k & 31)) {
#pragma unroll
            for (int i = 0; i < RS; ++i) {
                float v = 0.0f;
#pragma unroll
                for (int j = 0; j < CS; ++j)
                    if (j == kj) {
                        v = a[i][j];
                        a[i][j] = 0.0f;
                    }
                ck[ty + 8 * i] = v;
            }
        }
        __syncthreads();
        // (2) every warp: the pivot row p among the unused rows
        int best = -1;
        int bi = B;
#pragma unroll
        for (int m = 0; m < MW; ++m) {
            const int r = tx + 32 * m;
            if (r < B && !((used[m] >> tx) & 1u)) {
                const int v = piv_key(ck[r]);
                if (v > best) {
                    best = v;
                    bi = r;
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if (bi >= B) {
            // no comparable candidate (a non-finite column): the lowest unused row, so that
            // every index stays inside the block; the non-finite values propagate
#pragma unroll
            for (int m = MW - 1; m >= 0; --m) {
                const int nv = B - 32 * m < 32 ? B - 32 * m : 32;
                const unsigned fr = ~used[m] & (nv == 32 ? 0xffffffffu : ((1u << nv) - 1u));
                if (fr) bi = 32 * m + __ffs((int)fr) - 1;
            }
        }
        const int p = bi;
#pragma unroll
        for (int m = 0; m < MW; ++m)
            if (m == (p >> 5)) used[m] |= 1u << (p & 31);
        const float inv = 1.0f / ck[p];
        // (3) the warp that holds row p publishes it scaled (column k of it becomes 1/a_pk)
        if (ty == (p & 7)) {
            const int pi = p >> 3;
#pragma unroll
            for (int j = 0; j < CS; ++j) {
                float v = 0.0f;
#pragma unroll
                for (int i = 0; i < RS; ++i)
                    if (i == pi) v = a[i][j];
                const int c = tx + 32 * j;
                rk_s[c] = (c == k ? 1.0f : v) * inv;
            }
        }
        if (threadIdx.x == 0) perm[k] = p;
        __syncthreads();
        // (4) eliminate column k from every other row (padded rows have a zero column entry)
        float rk[CS];
#pragma unroll
        for (int j = 0; j < CS; ++j) rk[j] = rk_s[tx + 32 * j];
#pragma unroll
        for (int i = 0; i < RS; ++i) {
            if (ty + 8 * i == p) {
#pragma unroll
                for (int j = 0; j < CS; ++j) a[i][j] = rk[j];
            } else {
                const float f = ck[ty + 8 * i];
#pragma unroll
                for (int j = 0; j < CS; ++j) a[i][j] -= f * rk[j];
            }
        }
    }
    // Row r of the working matrix holds row invp[r] of the inverse, and its column k holds
    // column perm[k] (perm[k] = pivot row of step k, invp its inverse permutation).
    __syncthreads();
    for (int k = threadIdx.x; k < B; k += 256) invp[perm[k]] = k;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RS; ++i)
#pragma unroll
        for (int j = 0; j < CS; ++j) {
            const int r = ty + 8 * i, c = tx + 32 * j;
            if (r < B && c < B) tile[perm[c] * LD + invp[r]] = a[i][j];
        }
    __syncthreads();
    for (int t = threadIdx.x; t < B * B; t += 256) g[t] = tile[(t / B) * LD + (t % B)];
}

template <int B, int U>
cudaError_t gj_go(unsigned E, float* blk, cudaStream_t st) {
    const size_t sm = GjTile<B>::SMEM;
    cudaError_t e = cudaFuncSetAttribute(k_gj_tile<B, U>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_gj_tile<B, U><<<E, 256, sm, st>>>((int)E, blk);
    return cudaGetLastError();
}

#define EMG_GJ_TILE_INST(BB)                                                      \
    template cudaError_t gj_go<BB, 1>(unsigned, float*, cudaStream_t);            \
    template cudaError_t gj_go<BB, 4>(unsigned, float*, cudaStream_t);            \
    template cudaError_t gj_go<BB, 16>(unsigned, float*, cudaStream_t);
EMG_BSIZES(EMG_GJ_TILE_INST)
#undef EMG_GJ_TILE_INST
// the fully unrolled pivot loop (B <= 100)
template cudaError_t gj_go<15, 15>(unsigned, float*, cudaStream_t);
template cudaError_t gj_go<30, 30>(unsigned, float*, cudaStream_t);
template cudaError_t gj_go<50, 50>(unsigned, float*, cudaStream_t);
template cudaError_t gj_go<75, 75>(unsigned, float*, cudaStream_t);
template cudaError_t gj_go<20, 20>(unsigned, float*, cudaStream_t);
template cudaError_t gj_go<100, 100>(unsigned, float*, cudaStream_t);

}  // namespace emg
