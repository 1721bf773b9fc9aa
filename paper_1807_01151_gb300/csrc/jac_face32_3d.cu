// Float32 face Jacobians of the float32 block forms, 3-D levels; kernels in jac_face.cuh.
#include "jac_face.cuh"
#include "jacobian.cuh"

namespace emg {

emg_status launch_face_jacobian32_3d(emg_ctx* c, int p, const double* u) {
    switch (p) {
        case 0: face_jacobian32_go<3, 0>(c, u); break;
        case 1: face_jacobian32_go<3, 1>(c, u); break;
        case 2: face_jacobian32_go<3, 2>(c, u); break;
        case 3: face_jacobian32_go<3, 3>(c, u); break;
        case 4: face_jacobian32_go<3, 4>(c, u); break;
        default:
            c->err = "unsupported (dim, p)";
            return EMG_ERR_ARG;
    }
    EMG_CHECK_LAUNCH(c);
    return EMG_OK;
}

}  // namespace emg
