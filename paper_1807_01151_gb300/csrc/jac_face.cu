// FP64 face Jacobians (the FP64 block form and the p = 0 Jacobian); kernels in jac_face.cuh.
#include "jac_face.cuh"
#include "jacobian.cuh"

namespace emg {

emg_status launch_face_jacobian(emg_ctx* c, int p, const double* u) {
    LevelDev& L = c->lv[p];
    const int F = (int)c->F, Fi = (int)c->F_int;
    U5 ui;
    for (int a = 0; a < 5; ++a) ui.v[a] = c->uinf[a];
#define EMG_FJ(DD, PP)                                                                                       \
    {                                                                                                        \
        const int64_t nf = (int64_t)F * Lv<DD, PP>::QF;                                                      \
        ProfScope _ps(c, PC_FACE_JAC);                                                                       \
        if (c->rot)                                                                                          \
            k_face_jac<DD, PP, double, true><<<(unsigned)((nf + 127) / 128), 128, 0, c->stream>>>(           \
                F, Fi, c->face_L, c->face_R, c->face_bc, L.fnrm, L.famag, L.fpsiL, L.fpsiR, L.fwn, u,          \
                c->prm.gamma, ui, L.fvr, L.fjl, L.fjr);                                                      \
        else                                                                                                 \
            k_face_jac<DD, PP, double, false><<<(unsigned)((nf + 127) / 128), 128, 0, c->stream>>>(          \
                F, Fi, c->face_L, c->face_R, c->face_bc, L.fnrm, L.famag, L.fpsiL, L.fpsiR, L.fwn, u,          \
                c->prm.gamma, ui, nullptr, L.fjl, L.fjr);                                                    \
        EMG_CHECK_LAUNCH(c);                                                                                 \
    }
    EMG_DISPATCH_DP(c->dim, p, EMG_FJ)
#undef EMG_FJ
    return EMG_OK;
}

}  // namespace emg
