// Launchers of the unblocked float32 Gauss-Jordan inverse variants (defined and explicitly
// instantiated for every block size in gj_tile.cu and gj_cols.cu, dispatched in gj.cu).
#pragma once

#include <cuda_runtime.h>

namespace emg {

template <int B, int U>
cudaError_t gj_go(unsigned E, float* blk, cudaStream_t st);
template <int B, int W>
cudaError_t gj_cols_go(unsigned E, float* blk, cudaStream_t st);
template <int B, int W>
cudaError_t gj_rot_go(unsigned E, float* blk, cudaStream_t st);

}  // namespace emg
