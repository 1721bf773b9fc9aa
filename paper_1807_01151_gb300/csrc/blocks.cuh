// Shared pieces of the block factorisations (LU of the FP64 form, Gauss-Jordan inverses of
// the float32 forms): the pivot key and the list of block sizes B = 5 N the levels use.
#pragma once

#include <cstdint>

namespace emg {

// Pivot magnitude as an ordered integer key: the IEEE bits of |x| order like its value for
// every finite or infinite x; a NaN gets -1, so it never wins against a number.  Comparing
// keys as integers keeps the pivot search deterministic and independent of how the compiler
// treats float comparisons with NaN (where every thread of a warp computes the pivot on its
// own, a disagreement would break the permutation).
__device__ __forceinline__ int piv_key(float x) {
    const unsigned b = __float_as_uint(x) & 0x7fffffffu;
    return b <= 0x7f800000u ? (int)b : -1;
}
__device__ __forceinline__ long long piv_key(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
    return b <= 0x7ff0000000000000ull ? (long long)b : -1ll;
}

// Two fused multiply-adds d_k <- a b_k + d_k (k = 0, 1) issued as one paired float32
// instruction; each component is rounded as by fmaf, so the results are bitwise those of two
// fmaf calls and only the instruction count changes.
__device__ __forceinline__ void fma2f(float a, float b0, float b1, float& d0, float& d1) {
    const float2 r = __ffma2_rn(make_float2(a, a), make_float2(b0, b1), make_float2(d0, d1));
    d0 = r.x;
    d1 = r.y;
}

// B = 5 N(p): 2-D p = 1..4, then 3-D p = 1..4 (B = 50 serves both dimensions).
#define EMG_BSIZES(X) X(15) X(30) X(50) X(75) X(20) X(100) X(175)

}  // namespace emg
