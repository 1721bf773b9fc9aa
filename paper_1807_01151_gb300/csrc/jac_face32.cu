// Float32 face Jacobians of the float32 block forms, 2-D levels (3-D: jac_face32_3d.cu);
// kernels in jac_face.cuh.
#include "jac_face.cuh"
#include "jacobian.cuh"

namespace emg {

emg_status launch_face_jacobian32_3d(emg_ctx* c, int p, const double* u);

emg_status launch_face_jacobian32(emg_ctx* c, int p, const double* u) {
    if (c->dim == 3) return launch_face_jacobian32_3d(c, p, u);
    switch (c->dim * 8 + p) {
        case 16: face_jacobian32_go<2, 0>(c, u); break;
        case 17: face_jacobian32_go<2, 1>(c, u); break;
        case 18: face_jacobian32_go<2, 2>(c, u); break;
        case 19: face_jacobian32_go<2, 3>(c, u); break;
        case 20: face_jacobian32_go<2, 4>(c, u); break;
        default:
            c->err = "unsupported (dim, p)";
            return EMG_ERR_ARG;
    }
    EMG_CHECK_LAUNCH(c);
    return EMG_OK;
}

}  // namespace emg
