// Shared definitions of the eMG CUDA library: compile-time level shapes, the context
// layout in device memory, and error plumbing.  Everything here is private to the
// library; the public surface is include/emg.h.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <functional>
#include <string>
#include <vector>

#include "../../include/emg.h"

namespace emg {

constexpr int NVAR = 5;
constexpr int MAX_P = 4;
constexpr int MAX_KRYLOV = 64;

// The float32 block forms (FP32 and BF16 blocks) share the float tables, the explicit
// inverse and the stage GEMV.
inline bool blocks_f32(int prec) { return prec == EMG_PREC_FP32_BLOCKS || prec == EMG_PREC_BF16_BLOCKS; }

// Which float32 block kernels a level uses (emg_params.block_kernels).  The default follows the
// per-cycle kernel times measured on the GB300 with both forms: the SIMT assembly was faster at
// every level (2-D p = 4: 1.69 vs 2.33 ms, 3-D p = 3: 3.72 vs 4.63 ms, 3-D p = 4: 11.8 vs
// 16.6 ms per cycle); the tensor-core inverse was faster at B = 100 (2.67 vs 3.47 ms) and
// slower at B = 75 and 175.  The BF16 form needs the tensor-core assembly.
inline bool use_tc_assembly(int dim, int p, int prec, int block_kernels) {
    (void)dim;
    (void)p;
    if (prec == EMG_PREC_BF16_BLOCKS || block_kernels == 1) return true;
    return false;
}
inline bool use_tc_inverse(int B, int block_kernels) {
    const bool built = B == 75 || B == 100 || B == 175;
    if (!built || block_kernels >= 2) return false;
    if (block_kernels == 1) return true;
    return B == 100;
}

__host__ __device__ constexpr int n_modes(int D, int P) {
    return D == 2 ? (P + 1) * (P + 2) / 2 : (P + 1) * (P + 2) * (P + 3) / 6;
}
__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

// Shapes of level p in dimension D: N modes, q = p + 2 Gauss points per direction,
// Q volume points, QF points per face, NF faces per element, B = 5N block size.
template <int D_, int P_>
struct Lv {
    static constexpr int D = D_;
    static constexpr int P = P_;
    static constexpr int N = n_modes(D_, P_);
    static constexpr int q = P_ + 2;
    static constexpr int Q = ipow(P_ + 2, D_);
    static constexpr int QF = ipow(P_ + 2, D_ - 1);
    static constexpr int NF = 2 * D_;
    static constexpr int B = 5 * n_modes(D_, P_);
    static constexpr int NODES = 1 << D_;
};

// Device arrays of one multigrid level (p >= 0).
struct LevelDev {
    int p = 0, N = 0, q = 0, Q = 0, QF = 0, B = 0;
    // quadrature tables (per element / per face)
    double* vpsi = nullptr;    // [E][Q][N]      psi_i(x_q)
    double* vgw = nullptr;     // [E][D][Q][N]   W_q d_k psi_i(x_q)
    double* fnrm = nullptr;    // [F][QF][3]     unit outward normal of the L element
    double* famag = nullptr;   // [F][QF]        w |n dS|
    double* fpsiL = nullptr;   // [F][QF][N]     psi^L_i at the face points
    double* fpsiR = nullptr;   // [F_int][QF][N] psi^R_i at the face points
    double* fwn = nullptr;     // [F-F_int][QF][3] slip-wall reflection normal (body normal)
    double* vvr = nullptr;     // [E][Q][3]      frame velocity omega x x (rotating frame only)
    double* fvr = nullptr;     // [F][QF][3]     the same at the face points
    // states and work vectors, [E][5][N]
    double* v = nullptr;       // current approximation
    double* v0 = nullptr;      // restricted state (levels below p_max)
    double* tau = nullptr;     // FAS forcing (levels below p_max)
    double* un = nullptr;      // u^n of the PRK step
    double* r = nullptr;       // residual work
    double* r2 = nullptr;      // second residual buffer
    double* fhat = nullptr;    // [F][QF][5]     w|n dS| F~ at the face points
    double* fjl = nullptr;     // [F][QF][25]    w|n dS| dF~/dU_L (boundary: total derivative)
    double* fjr = nullptr;     // [F_int][QF][25] w|n dS| dF~/dU_R
    double* blk = nullptr;     // [E][B][B]      P_e, then its LU factors (column-major)
    int* piv = nullptr;        // [E][B]
    // FP32 block path (EMG_PREC_FP32_BLOCKS): float copies of the tables and blocks
    float* vpsi32 = nullptr;
    float* vgw32 = nullptr;
    float* fpsiL32 = nullptr;
    float* fpsiR32 = nullptr;
    float* blk32 = nullptr;    // [E][B][B]
    float* fjl32 = nullptr;    // [F][QF][25]  face Jacobians for the FP32 blocks
    float* fjr32 = nullptr;    // [F_int][QF][25]
    int gj_variant = 0;        // tuned variant of the FP32 Gauss-Jordan kernel
    bool tc_asm = false;       // float32 block assembly on the tensor cores
    bool tc_gj = false;        // float32 block inverse on the tensor cores
};

// Small device-side scalars of the cycle (no host round trip inside a V-cycle).
struct DevScalars {
    double cfl;
    double res;          // ||R(rho)|| at cycle entry
    double res5[5];
    double res_ref;      // ||R(rho_1)|| (<= 0: unset)
    double beta;         // ||N|| of the Krylov start vector
    double hsub;         // h_{j+1,j} of the current Arnoldi step
    double w0;           // ||A v_j|| before orthogonalisation
    int m_used;          // Arnoldi steps taken
    int broken;          // happy breakdown seen
    int nonfinite;       // non-finite residual seen
    int pad;             // non-positive density or pressure seen
    int timeout;         // a bounded device-side wait gave up
    int bad_index;       // an input index out of range (no-allocation EXP1 step)
    long long cycle;     // V-cycle index n of Eq. cfl (advanced on the device by every cycle body)
};

// Kernel classes of the event profiler (emg_profile_*).
enum ProfClass {
    PC_RES_FACE = 0, PC_RES_VOL, PC_FACE_JAC, PC_DIAG, PC_LU, PC_STAGE, PC_BSR0, PC_ARNOLDI, PC_PHI,
    PC_COMBINE, PC_TRANSFER, PC_CONTROL, PC_SETUP, PC_COUNT
};

struct Prof {
    bool on = false;
    std::vector<cudaEvent_t> ev;     // pool
    std::vector<int> pair_cls;       // class of pair k (events 2k, 2k+1)
    int used = 0;                    // events used
    double ms[PC_COUNT] = {};
    int64_t cnt[PC_COUNT] = {};
};

}  // namespace emg

struct emg_ctx {
    emg_params prm{};
    int dim = 0;
    int p_max = 0;
    int64_t E = 0, F = 0, F_int = 0, n_nodes = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t stream2 = nullptr;  // side stream: residuals that overlap a level's block build
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool side_pending = false;       // side work enqueued, not yet joined
    int device = 0;
    std::string err;
    int64_t bytes = 0;
    std::vector<void*> allocs;
    // mesh (device)
    int* face_L = nullptr;       // [F]
    int* face_fL = nullptr;      // [F]
    int* face_R = nullptr;       // [F] (-1 on boundary faces)
    int* face_bc = nullptr;      // [F]
    int* elem_face = nullptr;    // [E][2D]  (face id << 1) | side (0 = L, 1 = R)
    int* elem_nbr = nullptr;     // [E][2D]  neighbour or -1
    double* elem_x = nullptr;    // [E][2^D][D]
    double* elem_wn = nullptr;   // [E][2^D][D] body normals at the nodes (wall_normal input)
    int has_wn = 0;
    bool rot = false;              // rotating frame (omega != 0, Eq. euler)
    double* xc = nullptr;        // [E][3]
    double* Lh = nullptr;        // [E][3]
    double* vol = nullptr;       // [E]
    double* surf = nullptr;      // [E]
    double* h = nullptr;         // [E]
    double* C = nullptr;         // [E][Nmax][Nmax]
    double* psic = nullptr;      // [E][Nmax] psi_i(x_c)
    double* gl = nullptr;        // [8][2][8] Gauss-Legendre nodes/weights, q = 1..7
    double domain_volume = 0.0;
    double uinf[5] = {0, 0, 0, 0, 0};
    emg::LevelDev lv[emg::MAX_P + 1];
    // EXP1 / Krylov
    double* dt = nullptr;        // [E] EXP1 steps
    double* bsr = nullptr;       // [E][1+2D][25]
    double* V = nullptr;         // [(m+1)][K0]
    double* w = nullptr;         // [K0]
    double* H = nullptr;         // [(m+1)][m] row-major
    double* hcol = nullptr;      // [m+1] current Hessenberg column
    double* y = nullptr;         // [m]
    double* partial = nullptr;   // 3 x [red_blocks][MAX_KRYLOV+8] reduction partials
    unsigned int* bar = nullptr; // grid barrier state of the persistent Arnoldi kernel
    int red_blocks = 0;
    emg::DevScalars* sc = nullptr;
    emg::DevScalars* sc_host = nullptr;   // pinned
    double* stage_in = nullptr;  // staging for component calls, [E][5][Nmax]
    double* stage_in2 = nullptr;
    double* stage_out = nullptr; // output staging of the component calls, grown on demand
    int64_t stage_out_n = 0;
    double* stage_small = nullptr; // [E] (dt input)
    int64_t cycle_n = 1;
    double res_ref = 0.0;
    emg::Prof prof;
    int64_t launches = 0;            // kernels launched by this context
    cudaGraphExec_t body_exec = nullptr;  // captured V-cycle body up to the Arnoldi kernel
    cudaGraphExec_t body_exec_frozen = nullptr;  // the same with the block factors reused (jac_freeze)
    int64_t body_kernels_frozen = 0;
    int64_t up_kernels = 0;          // kernels of the captured part from the Arnoldi kernel on
    bool frozen = false;             // the cycle being issued reuses the stored block factors
    bool blocks_valid = false;       // the stored factors of every level come from a V-cycle
    cudaGraphExec_t krylov_exec = nullptr; // the rest of the body, from the Arnoldi kernel on
    int64_t body_kernels = 0;        // kernels in both
    bool capturing = false;          // a graph capture is in progress on the stream
    std::string tuning;              // variants chosen by the tuner, with their times
    bool graph_failed = false;       // capture or instantiation failed: launch kernel by kernel
};

namespace emg {
void prof_flush(emg_ctx* c);
// Brackets one kernel launch with events on the context's stream when profiling is on,
// and counts the launch.
struct ProfScope {
    emg_ctx* c;
    int cls;
    int b = -1;
    ProfScope(emg_ctx* c_, int cls_) : c(c_), cls(cls_) {
        c->launches++;
        if (!c->prof.on) return;
        if (c->prof.used + 2 > (int)c->prof.ev.size()) prof_flush(c);
        b = c->prof.used;
        cudaEventRecord(c->prof.ev[b], c->stream);
        c->prof.used += 2;
        c->prof.pair_cls[b / 2] = cls;
    }
    ~ProfScope() {
        if (b >= 0) cudaEventRecord(c->prof.ev[b + 1], c->stream);
    }
};
}  // namespace emg

#define EMG_CUDA_TRY(ctx, call)                                                           \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e_);              \
            return EMG_ERR_CUDA;                                                          \
        }                                                                                 \
    } while (0)

#define EMG_CHECK_LAUNCH(ctx) EMG_CUDA_TRY(ctx, cudaGetLastError())

// Launch helpers implemented in the .cu files (host side).
namespace emg {
emg_status setup_device_mesh(emg_ctx* c, const emg_mesh_desc* m);
emg_status launch_residual(emg_ctx* c, int p, const double* u, const double* tau, double* R);
emg_status launch_face_jacobian(emg_ctx* c, int p, const double* u);
emg_status launch_diag_blocks(emg_ctx* c, int p, const double* u, const double* cfl_dev, int shifted,
                              double* out);
emg_status launch_lu(emg_ctx* c, int p);
emg_status launch_stage(emg_ctx* c, int p, const double* r, const double* un, double beta, double* out);
emg_status launch_diag_blocks32(emg_ctx* c, int p, const double* u, const double* cfl_dev, int shifted, float* out);
emg_status launch_lu32(emg_ctx* c, int p);
emg_status launch_stage32(emg_ctx* c, int p, const double* r, const double* un, double beta, double* out);
emg_status build_float_tables(emg_ctx* c);
emg_status tune_gj(emg_ctx* c);
emg_status selftest_barrier_timeout(emg_ctx* c, int* timed_out);
emg_status launch_bsr0(emg_ctx* c);
emg_status launch_exp1(emg_ctx* c, const double* u0, const double* tau0, const double* dt, double* out);
emg_status launch_exp1_prepare(emg_ctx* c, const double* u0, const double* tau0);
emg_status launch_exp1_krylov(emg_ctx* c, const double* u0, const double* dt, double* out);
emg_status coop_ordered(int device, cudaStream_t st, const std::function<cudaError_t()>& launch, std::string* err);
emg_status launch_restrict(emg_ctx* c, int p_fine, const double* fine, double* coarse);
emg_status launch_tau(emg_ctx* c, int p_coarse, const double* rfine, const double* rcoarse, double* tau);
emg_status launch_prolong(emg_ctx* c, int p_fine, double* fine, const double* vc, const double* v0c);
emg_status launch_norm_cfl(emg_ctx* c, const double* R, int update_cfl);
emg_status launch_dtau(emg_ctx* c, int p, const double* u, const double* cfl_dev, double factor, double* dt);
emg_status launch_dt_global(emg_ctx* c, double* dt);
emg_status launch_axpby(emg_ctx* c, int64_t n, double a, const double* x, double b, const double* y, double* out);
emg_status launch_check_state(emg_ctx* c, const double* u, int64_t n);
// V-cycle pieces (api.cu), shared with the request loop (server.cu)
emg_status vcycle_entry(emg_ctx* c);
emg_status vcycle_body_down(emg_ctx* c);
emg_status vcycle_body_up(emg_ctx* c);
emg_status vcycle_body(emg_ctx* c);
emg_status run_body(emg_ctx* c);
emg_status check_flags(emg_ctx* c);
int64_t estimate_bytes(int dim, int64_t E, int64_t F, int64_t F_int, int p_max, int m, int prec, bool rot);
DevScalars* pinned_scalars_acquire();
void pinned_scalars_release(DevScalars* p);
}  // namespace emg
