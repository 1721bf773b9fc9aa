// Pieces of the exact Jacobian blocks (Sec. 3.3) shared by the translation units that build
// them: jacobian.cu (SIMT assembly, p = 0 blocks, source term, launchers), jac_face.cu (face
// Jacobians by dual numbers) and jac_tc.cu (tensor-core assembly of the float32 forms).
#pragma once

#include "common.cuh"

namespace emg {

// A_k = dF_k/dU (closed form, Appendix Eq. dfdu with grad psi -> e_k and omega = 0).
__device__ __forceinline__ void flux_jac_k(const double U[5], double g, int k, double A[25]) {
    const double ir = 1.0 / U[0];
    const double v[3] = {U[1] * ir, U[2] * ir, U[3] * ir};
    const double q2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const double a0 = 0.5 * (g - 1.0) * q2;
    const double p = (g - 1.0) * (U[4] - 0.5 * U[0] * q2);
    const double H = (U[4] + p) * ir;
    const double vk = v[k];
#pragma unroll
    for (int t = 0; t < 25; ++t) A[t] = 0.0;
    A[1 + k] = 1.0;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        double* row = A + 5 * (1 + m);
        row[0] = (m == k ? a0 : 0.0) - v[m] * vk;
#pragma unroll
        for (int l = 0; l < 3; ++l)
            row[1 + l] = (l == k ? v[m] : 0.0) - (m == k ? (g - 1.0) * v[l] : 0.0) + (m == l ? vk : 0.0);
        row[4] = m == k ? (g - 1.0) : 0.0;
    }
    A[20] = (a0 - H) * vk;
#pragma unroll
    for (int l = 0; l < 3; ++l) A[21 + l] = (l == k ? H : 0.0) - (g - 1.0) * v[l] * vk;
    A[24] = g * vk;
}

// The same closed form in float for the FP32 block path.
__device__ __forceinline__ void flux_jac_k(const float U[5], float g, int k, float A[25]) {
    const float ir = 1.0f / U[0];
    const float v[3] = {U[1] * ir, U[2] * ir, U[3] * ir};
    const float q2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const float a0 = 0.5f * (g - 1.0f) * q2;
    const float p = (g - 1.0f) * (U[4] - 0.5f * U[0] * q2);
    const float H = (U[4] + p) * ir;
    const float vk = v[k];
#pragma unroll
    for (int t = 0; t < 25; ++t) A[t] = 0.0f;
    A[1 + k] = 1.0f;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        float* row = A + 5 * (1 + m);
        row[0] = (m == k ? a0 : 0.0f) - v[m] * vk;
#pragma unroll
        for (int l = 0; l < 3; ++l)
            row[1 + l] = (l == k ? v[m] : 0.0f) - (m == k ? (g - 1.0f) * v[l] : 0.0f) + (m == l ? vk : 0.0f);
        row[4] = m == k ? (g - 1.0f) : 0.0f;
    }
    A[20] = (a0 - H) * vk;
#pragma unroll
    for (int l = 0; l < 3; ++l) A[21 + l] = (l == k ? H : 0.0f) - (g - 1.0f) * v[l] * vk;
    A[24] = g * vk;
}

// Face Jacobians of level p in float32 (jac_face.cu); the FP64 ones are launch_face_jacobian.
emg_status launch_face_jacobian32(emg_ctx* c, int p, const double* u);

// Tensor-core assembly of the float32 forms at level p (jac_tc.cu): P_e (shifted) or D_e
// without the rotating frame's source term, which the caller adds.
emg_status launch_diag_blocks_tc(emg_ctx* c, int p, const double* u, const double* cfl_dev, int shifted,
                                 float* out);

}  // namespace emg
