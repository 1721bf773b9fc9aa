// C ABI (include/emg.h): context life cycle, state I/O, the FAS V-cycle of Sec. 2.3 and
// the component entry points.  All arithmetic runs in the kernels of the other files; this
// file only sequences launches on the context's stream.
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "common.cuh"

using namespace emg;

namespace {

emg_status fail(emg_ctx* c, emg_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

emg_status sync(emg_ctx* c) {
    EMG_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return EMG_OK;
}

emg_status read_scalars(emg_ctx* c) {
    EMG_CUDA_TRY(c, cudaMemcpyAsync(c->sc_host, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream));
    return sync(c);
}

emg_status copy_in(emg_ctx* c, double* dst, const double* src, int64_t n, int on_device) {
    EMG_CUDA_TRY(c, cudaMemcpyAsync(dst, src, n * sizeof(double),
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    return EMG_OK;
}

// Output staging of the component calls, grown on demand (a full set of FP64 blocks of the
// top level is only needed by emg_jacobian_diag with host output).
emg_status stage_out(emg_ctx* c, int64_t n, double** out) {
    if (c->stage_out_n < n) {
        if (c->stage_out) EMG_CUDA_TRY(c, cudaFreeAsync(c->stage_out, c->stream));
        c->stage_out = nullptr;
        c->stage_out_n = 0;
        EMG_CUDA_TRY(c, cudaMallocAsync((void**)&c->stage_out, (size_t)n * sizeof(double), c->stream));
        c->stage_out_n = n;
    }
    *out = c->stage_out;
    return EMG_OK;
}

emg_status copy_out(emg_ctx* c, double* dst, const double* src, int64_t n, int on_device) {
    EMG_CUDA_TRY(c, cudaMemcpyAsync(dst, src, n * sizeof(double),
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (!on_device) return sync(c);
    return EMG_OK;
}

}  // namespace

namespace emg {

__global__ void k_set_freestream(int64_t E, int N, const double* __restrict__ vol, double u0, double u1, double u2,
                                 double u3, double u4, double* __restrict__ v) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= E * 5 * N) return;
    const int i = (int)(idx % N);
    const int a = (int)((idx / N) % 5);
    const int64_t e = idx / (5 * N);
    const double U[5] = {u0, u1, u2, u3, u4};
    v[idx] = i == 0 ? U[a] * sqrt(vol[e]) : 0.0;
}

// float32 blocks widened to float64 row-major (colmajor: the source is column-major)
__global__ void k_widen_blocks(int64_t E, int B, const float* __restrict__ src, int colmajor,
                               double* __restrict__ dst) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t BB = (int64_t)B * B;
    if (t >= E * BB) return;
    const int64_t e = t / BB;
    const int rc = (int)(t % BB);
    const int r = rc / B, cc = rc % B;
    dst[t] = (double)src[e * BB + (colmajor ? (int64_t)cc * B + r : (int64_t)r * B + cc)];
}

__global__ void k_set_cfl(DevScalars* sc, double cfl) { sc->cfl = cfl; }
__global__ void k_set_ref(DevScalars* sc, double ref) { sc->res_ref = ref; }
__global__ void k_set_cycle(DevScalars* sc, long long n) { sc->cycle = n; }
__global__ void k_advance_cycle(DevScalars* sc) { sc->cycle += 1; }

// Work that does not depend on a level's block build (residuals) runs on the side stream
// while the main stream assembles and factors the blocks: fork_side enqueues `side` on the
// side stream after everything already on the main stream, join_side makes the main stream
// wait for it.  Inside a graph capture the two branches become parallel branches of the
// graph.  With the event profiler on (it times one stream) the side work runs in order.
static emg_status fork_side(emg_ctx* c, const std::function<emg_status(emg_ctx*)>& side) {
    if (c->prof.on || !c->stream2) return side(c);
    EMG_CUDA_TRY(c, cudaEventRecord(c->ev_fork, c->stream));
    EMG_CUDA_TRY(c, cudaStreamWaitEvent(c->stream2, c->ev_fork, 0));
    std::swap(c->stream, c->stream2);
    const emg_status st = side(c);
    std::swap(c->stream, c->stream2);
    if (st != EMG_OK) return st;
    EMG_CUDA_TRY(c, cudaEventRecord(c->ev_join, c->stream2));
    c->side_pending = true;
    return EMG_OK;
}
static emg_status join_side(emg_ctx* c) {
    if (!c->side_pending) return EMG_OK;
    c->side_pending = false;
    EMG_CUDA_TRY(c, cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    return EMG_OK;
}

// One PRK step (Eq. prk_scalar) on level p: u^n = L.v on entry, result in L.v.
// r_first: R~_p(u^n) if already available; side: work to run on the side stream during the
// block build that leaves R~_p(u^n) in r_first (else R~_p(u^n) itself is computed there when
// the blocks are built, and in order otherwise).  reuse_blocks: apply the factors of the
// previous step of this level instead of P(u^n) (lagged preconditioner).
static emg_status prk_step(emg_ctx* c, int p, const double* tau, const double* r_first, bool reuse_blocks = false,
                           const std::function<emg_status(emg_ctx*)>& side = nullptr) {
    LevelDev& L = c->lv[p];
    const int64_t S = c->E * L.B;
    EMG_CUDA_TRY(c, cudaMemcpyAsync(L.un, L.v, S * 8, cudaMemcpyDeviceToDevice, c->stream));
    const bool f32 = blocks_f32(c->prm.prec);
    emg_status st = EMG_OK;
    if (!reuse_blocks) {
        if (side) {
            st = fork_side(c, side);
        } else if (!r_first) {
            st = fork_side(c, [p, tau](emg_ctx* cc) { return launch_residual(cc, p, cc->lv[p].v, tau, cc->lv[p].r); });
            r_first = L.r;
        }
        if (st != EMG_OK) return st;
        st = f32 ? launch_diag_blocks32(c, p, L.un, &c->sc->cfl, 1, L.blk32)
                 : launch_diag_blocks(c, p, L.un, &c->sc->cfl, 1, L.blk);
        if (st == EMG_OK) st = f32 ? launch_lu32(c, p) : launch_lu(c, p);
        // joined on every path: a fork left open would also invalidate a graph capture
        const emg_status sj = join_side(c);
        if (st != EMG_OK) return st;
        if (sj != EMG_OK) return sj;
    } else if (side) {
        st = side(c);
        if (st != EMG_OK) return st;
    }
    const int s = c->prm.rk_stages;
    for (int k = 1; k <= s; ++k) {
        const double beta = 1.0 / (double)(s - k + 1);
        const double* r = nullptr;
        if (k == 1 && r_first) {
            r = r_first;
        } else {
            st = launch_residual(c, p, L.v, tau, L.r);
            if (st != EMG_OK) return st;
            r = L.r;
        }
        st = f32 ? launch_stage32(c, p, r, L.un, beta, L.v) : launch_stage(c, p, r, L.un, beta, L.v);
        if (st != EMG_OK) return st;
    }
    return EMG_OK;
}

// Entry of V-cycle n (n kept on the device): R_pmax(v), ||R(rho)|| and CFL_n.
emg_status vcycle_entry(emg_ctx* c) {
    LevelDev& T = c->lv[c->p_max];
    emg_status st = launch_residual(c, c->p_max, T.v, nullptr, T.r);
    if (st != EMG_OK) return st;
    return launch_norm_cfl(c, T.r, 1);
}

// First part of the cycle body: the down leg (PRK smoothing, restriction and FAS forcing on
// every level p >= 1, Sec. 2.3 steps 1-4) and the EXP1 inputs on p = 0.
emg_status vcycle_body_down(emg_ctx* c) {
    const int P = c->p_max;
    const double fac = c->prm.exp_dt_factor > 0.0 ? c->prm.exp_dt_factor : (double)(P + 1);
    emg_status st = launch_dtau(c, P, c->lv[P].v, &c->sc->cfl, fac, c->dt);
    if (st != EMG_OK) return st;
    if (c->prm.exp_dt_global) {
        st = launch_dt_global(c, c->dt);
        if (st != EMG_OK) return st;
    }
    // forcing of the level below (steps 2-3): R~_p(v_p) and R_{p-1}(v0_{p-1}) give tau_{p-1}, and
    // R~_{p-1}(v0_{p-1}) = R_{p-1}(v0_{p-1}) + tau_{p-1} is the first PRK stage's residual there.
    // It needs only the restricted state, so it runs on the side stream while the level below
    // assembles and factors its blocks.
    auto forcing = [](int p) {
        return [p](emg_ctx* cc) -> emg_status {
            LevelDev& Lp = cc->lv[p];
            LevelDev& Lq = cc->lv[p - 1];
            emg_status s2 = launch_residual(cc, p, Lp.v, p == cc->p_max ? nullptr : Lp.tau, Lp.r);
            if (s2 != EMG_OK) return s2;
            s2 = launch_residual(cc, p - 1, Lq.v0, nullptr, Lq.r2);
            if (s2 != EMG_OK) return s2;
            s2 = launch_tau(cc, p - 1, Lp.r, Lq.r2, Lq.tau);
            if (s2 != EMG_OK) return s2;
            if (p - 1 >= 1) s2 = launch_axpby(cc, cc->E * Lq.B, 1.0, Lq.r2, 1.0, Lq.tau, Lq.r);
            return s2;
        };
    };
    for (int p = P; p >= 1; --p) {
        LevelDev& L = c->lv[p];
        LevelDev& Lc = c->lv[p - 1];
        const double* tau = p == P ? nullptr : L.tau;
        for (int sm = 0; sm < c->prm.pre_smooth; ++sm) {
            const bool reuse = c->frozen || (c->prm.lag_blocks != 0 && sm > 0);
            if (sm == 0 && p == P)
                st = prk_step(c, p, tau, L.r, reuse);   // R_pmax(v) from the cycle entry
            else if (sm == 0)
                st = prk_step(c, p, tau, L.r, reuse, forcing(p + 1));   // R~_p(v0_p), from the forcing
            else
                st = prk_step(c, p, tau, nullptr, reuse);
            if (st != EMG_OK) return st;
        }
        // restriction of the smoothed state (its residual and the forcing follow, above)
        st = launch_restrict(c, p, L.v, Lc.v0);
        if (st != EMG_OK) return st;
        EMG_CUDA_TRY(c, cudaMemcpyAsync(Lc.v, Lc.v0, c->E * Lc.B * 8, cudaMemcpyDeviceToDevice, c->stream));
        if (p == 1) {   // p = 0 has no blocks to overlap with
            st = forcing(1)(c);
            if (st != EMG_OK) return st;
        }
    }
    LevelDev& L0 = c->lv[0];
    if (P == 0) EMG_CUDA_TRY(c, cudaMemcpyAsync(L0.v0, L0.v, c->E * 5 * 8, cudaMemcpyDeviceToDevice, c->stream));
    return launch_exp1_prepare(c, L0.v0, P == 0 ? nullptr : L0.tau);
}

// Second part of the cycle body: the EXP1 Krylov step on p = 0, then prolongation and
// correction up to p_max (Sec. 2.3 steps 5-6), and the cycle counter.
emg_status vcycle_body_up(emg_ctx* c) {
    const int P = c->p_max;
    LevelDev& L0 = c->lv[0];
    emg_status st = launch_exp1_krylov(c, L0.v0, c->dt, L0.v);
    if (st != EMG_OK) return st;
    for (int p = 1; p <= P; ++p) {
        st = launch_prolong(c, p, c->lv[p].v, c->lv[p - 1].v, c->lv[p - 1].v0);
        if (st != EMG_OK) return st;
    }
    { ProfScope _ps(c, PC_CONTROL); k_advance_cycle<<<1, 1, 0, c->stream>>>(c->sc); }
    EMG_CHECK_LAUNCH(c);
    return EMG_OK;
}

emg_status vcycle_body(emg_ctx* c) {
    emg_status st = vcycle_body_down(c);
    if (st != EMG_OK) return st;
    return vcycle_body_up(c);
}

// Capture one part of the body into an executable graph (nothing runs during a capture).
static emg_status capture(emg_ctx* c, emg_status (*part)(emg_ctx*), cudaGraphExec_t* exec, int64_t* kernels) {
    const int64_t l0 = c->launches;
    EMG_CUDA_TRY(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    c->capturing = true;
    const emg_status st = part(c);
    c->capturing = false;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    cudaError_t ei = cudaErrorUnknown;
    if (st == EMG_OK && e == cudaSuccess && g) ei = cudaGraphInstantiate(exec, g, 0);
    if (g) cudaGraphDestroy(g);
    *kernels = c->launches - l0;   // kernels recorded, none launched yet
    c->launches = l0;
    if (ei != cudaSuccess) {
        cudaGetLastError();
        *exec = nullptr;
        return EMG_ERR_CUDA;
    }
    return EMG_OK;
}

// The cycle body as two CUDA graphs, captured on first use and then replayed (the host
// sequence has no data-dependent branch: every decision of the cycle is on the device).
// The split sits before the cooperative Arnoldi kernel, whose replay is ordered with the
// cooperative launches of other contexts.
// With jac_freeze = k > 1, cycles n with (n - 1) mod k != 0 reuse the block factors of every
// level (once factors from a V-cycle exist), through a second captured down leg.
static emg_status run_body_impl(emg_ctx* c) {
    if (!c->prm.use_graph || c->graph_failed || c->prof.on) return vcycle_body(c);
    if (!c->body_exec || !c->krylov_exec) {
        int64_t k1 = 0, k2 = 0;
        const bool fz = c->frozen;
        c->frozen = false;
        if (capture(c, vcycle_body_down, &c->body_exec, &k1) != EMG_OK ||
            capture(c, vcycle_body_up, &c->krylov_exec, &k2) != EMG_OK) {
            if (c->body_exec) cudaGraphExecDestroy(c->body_exec);
            if (c->krylov_exec) cudaGraphExecDestroy(c->krylov_exec);
            c->body_exec = c->krylov_exec = nullptr;
            c->graph_failed = true;   // run kernel by kernel from now on (same kernels)
            c->frozen = fz;
            return vcycle_body(c);
        }
        c->frozen = fz;
        c->body_kernels = k1 + k2;
        c->up_kernels = k2;
    }
    cudaGraphExec_t down = c->body_exec;
    int64_t nk = c->body_kernels;
    if (c->frozen) {
        if (!c->body_exec_frozen) {
            int64_t k1 = 0;
            if (capture(c, vcycle_body_down, &c->body_exec_frozen, &k1) != EMG_OK) {
                c->body_exec_frozen = nullptr;
                return vcycle_body(c);
            }
            c->body_kernels_frozen = k1;
        }
        down = c->body_exec_frozen;
        nk = c->body_kernels_frozen + c->up_kernels;
    }
    EMG_CUDA_TRY(c, cudaGraphLaunch(down, c->stream));
    cudaGraphExec_t kx = c->krylov_exec;
    if (c->prm.coop_krylov) {
        emg_status st = coop_ordered(c->device, c->stream, [kx, c]() { return cudaGraphLaunch(kx, c->stream); }, &c->err);
        if (st != EMG_OK) return st;
    } else {
        EMG_CUDA_TRY(c, cudaGraphLaunch(kx, c->stream));
    }
    c->launches += nk;
    return EMG_OK;
}

emg_status run_body(emg_ctx* c) {
    const int k = c->prm.jac_freeze;
    c->frozen = k > 1 && c->blocks_valid && ((c->cycle_n - 1) % k) != 0;
    const emg_status st = run_body_impl(c);
    if (st == EMG_OK && !c->frozen) c->blocks_valid = true;
    c->frozen = false;
    return st;
}

// Page-locked host slots for the per-context device scalars, taken from chunks that live
// as long as the process: creating and destroying contexts then never frees page-locked
// memory, which would wait for the whole device.
namespace {
std::mutex g_pin_mu;
std::vector<DevScalars*> g_pin_free;
}  // namespace

DevScalars* pinned_scalars_acquire() {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    if (g_pin_free.empty()) {
        constexpr int kChunk = 64;
        DevScalars* chunk = nullptr;
        if (cudaMallocHost(&chunk, kChunk * sizeof(DevScalars)) != cudaSuccess) return nullptr;
        for (int i = kChunk - 1; i >= 0; --i) g_pin_free.push_back(chunk + i);
    }
    DevScalars* p = g_pin_free.back();
    g_pin_free.pop_back();
    std::memset(p, 0, sizeof(DevScalars));
    return p;
}

void pinned_scalars_release(DevScalars* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free.push_back(p);
}

void prof_flush(emg_ctx* c) {
    if (c->prof.used == 0) return;
    cudaStreamSynchronize(c->stream);
    for (int k = 0; k < c->prof.used / 2; ++k) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, c->prof.ev[2 * k], c->prof.ev[2 * k + 1]) == cudaSuccess) {
            c->prof.ms[c->prof.pair_cls[k]] += ms;
            c->prof.cnt[c->prof.pair_cls[k]] += 1;
        }
    }
    c->prof.used = 0;
}

emg_status check_flags(emg_ctx* c) {
    if (c->sc_host->timeout) return fail(c, EMG_ERR_TIMEOUT, "a grid barrier wait in the Arnoldi kernel timed out");
    if (c->sc_host->nonfinite) return fail(c, EMG_ERR_NONFINITE, "non-finite residual or Krylov quantity");
    if (c->sc_host->pad) return fail(c, EMG_ERR_UNPHYSICAL, "non-positive density or pressure at a cell centre");
    return EMG_OK;
}

}  // namespace emg

extern "C" {

void emg_default_params(emg_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->gamma = 1.4;
    p->mach = 0.3;
    p->alpha_deg = 0.0;
    p->p_max = 2;
    p->rk_stages = 4;
    p->krylov_m = 30;
    p->cfl_max = 100.0;
    p->exp_dt_factor = 0.0;
    p->pre_smooth = 2;
    p->prec = EMG_PREC_FP64;
    p->cuda_stream = nullptr;
    p->use_graph = 1;
    p->autotune = 1;
    p->coop_krylov = 1;
    p->krylov_tol = 0.0;
    p->exp_dt_global = 0;
    p->jac_freeze = 1;
    p->quad_extra = 2;
    p->omega[0] = p->omega[1] = p->omega[2] = 0.0;
    p->block_kernels = 0;
    p->krylov_f32 = -1;
}

const char* emg_build_info(void) {
    return "emg sm_103a: FP64 residual (face Roe + element volume), AD face Jacobians, block assembly; "
           "FP64 blocks: shared-memory LU + warp substitution; FP32 blocks: tuned Gauss-Jordan inverse + GEMV; "
           "CGS2 Arnoldi (persistent cooperative or barrier-free), Pade-13 phi_1; graph-captured V-cycle; "
           "continuous-batching request loop";
}

emg_status emg_create_mesh(const emg_mesh_desc* m, const emg_params* prm, emg_ctx** out) {
    if (!out) return EMG_ERR_ARG;
    *out = nullptr;
    if (!m || !prm) return EMG_ERR_ARG;
    emg_ctx* c = new (std::nothrow) emg_ctx();
    if (!c) return EMG_ERR_OOM;
    *out = c;
    c->prm = *prm;
    if (m->dim != 2 && m->dim != 3) return fail(c, EMG_ERR_ARG, "dim must be 2 or 3");
    if (m->n_elems <= 0 || m->n_nodes <= 0 || !m->xyz || !m->elem_nodes || !m->face_bc)
        return fail(c, EMG_ERR_ARG, "empty or incomplete mesh");
    if (m->n_elems > (int64_t)1 << 30) return fail(c, EMG_ERR_ARG, "too many elements");
    if (prm->p_max < 0 || prm->p_max > MAX_P) return fail(c, EMG_ERR_ARG, "p_max must be in 0..4");
    if (prm->rk_stages < 1 || prm->rk_stages > 16) return fail(c, EMG_ERR_ARG, "rk_stages must be in 1..16");
    if (prm->krylov_m < 1 || prm->krylov_m > 40) return fail(c, EMG_ERR_ARG, "krylov_m must be in 1..40");
    if (!(prm->cfl_max > 0.0)) return fail(c, EMG_ERR_ARG, "cfl_max must be positive");
    if (prm->pre_smooth < 1) return fail(c, EMG_ERR_ARG, "pre_smooth must be >= 1");
    if (!(prm->gamma > 1.0) || !(prm->mach >= 0.0)) return fail(c, EMG_ERR_ARG, "bad gamma or mach");
    if (prm->prec != EMG_PREC_FP64 && prm->prec != EMG_PREC_FP32_BLOCKS && prm->prec != EMG_PREC_BF16_BLOCKS)
        return fail(c, EMG_ERR_ARG, "prec must be EMG_PREC_FP64, EMG_PREC_FP32_BLOCKS or EMG_PREC_BF16_BLOCKS");
    if (!(prm->krylov_tol >= 0.0)) return fail(c, EMG_ERR_ARG, "krylov_tol must be >= 0");
    if (prm->exp_dt_global != 0 && prm->exp_dt_global != 1) return fail(c, EMG_ERR_ARG, "exp_dt_global must be 0 or 1");
    if (prm->jac_freeze < 0) return fail(c, EMG_ERR_ARG, "jac_freeze must be >= 1");
    if (prm->quad_extra != 0 && prm->quad_extra != 2)
        return fail(c, EMG_ERR_ARG, "only the rule q = p + 2 is built (quad_extra 2)");
    if (prm->block_kernels < 0 || prm->block_kernels > 3)
        return fail(c, EMG_ERR_ARG, "block_kernels must be 0, 1, 2 or 3");
    if (prm->krylov_f32 < -1 || prm->krylov_f32 > 1) return fail(c, EMG_ERR_ARG, "krylov_f32 must be -1, 0 or 1");
    if (c->prm.krylov_f32 < 0) c->prm.krylov_f32 = blocks_f32(prm->prec) ? 1 : 0;
    if (!std::isfinite(prm->omega[0]) || !std::isfinite(prm->omega[1]) || !std::isfinite(prm->omega[2]))
        return fail(c, EMG_ERR_ARG, "omega must be finite");
    if (m->dim == 2 && (prm->omega[0] != 0.0 || prm->omega[1] != 0.0))
        return fail(c, EMG_ERR_ARG, "in 2-D the rotation axis must be z (omega = (0, 0, w))");
    c->rot = prm->omega[0] != 0.0 || prm->omega[1] != 0.0 || prm->omega[2] != 0.0;
    c->p_max = prm->p_max;
    if (c->prm.jac_freeze < 1) c->prm.jac_freeze = 1;
    EMG_CUDA_TRY(c, cudaGetDevice(&c->device));
    if (prm->cuda_stream) {
        c->stream = (cudaStream_t)prm->cuda_stream;
    } else {
        EMG_CUDA_TRY(c, cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    EMG_CUDA_TRY(c, cudaStreamCreateWithFlags(&c->stream2, cudaStreamNonBlocking));
    EMG_CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    EMG_CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    const double g = prm->gamma;
    const double a = prm->alpha_deg * M_PI / 180.0;
    const double vx = prm->mach * std::cos(a), vy = prm->mach * std::sin(a);
    c->uinf[0] = 1.0;
    c->uinf[1] = vx;
    c->uinf[2] = vy;
    c->uinf[3] = 0.0;
    c->uinf[4] = (1.0 / g) / (g - 1.0) + 0.5 * (vx * vx + vy * vy);
    emg_status st = setup_device_mesh(c, m);
    if (st != EMG_OK) return st;
    return emg_set_state(c, nullptr, 0);
}

emg_status emg_destroy(emg_ctx* c) {
    if (!c) return EMG_OK;
    if (c->body_exec) cudaGraphExecDestroy(c->body_exec);
    if (c->body_exec_frozen) cudaGraphExecDestroy(c->body_exec_frozen);
    if (c->krylov_exec) cudaGraphExecDestroy(c->krylov_exec);
    for (void* p : c->allocs) cudaFreeAsync(p, c->stream);
    if (c->stage_out) cudaFreeAsync(c->stage_out, c->stream);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto& e : c->prof.ev) cudaEventDestroy(e);
    pinned_scalars_release(c->sc_host);
    if (c->stream2) {
        cudaStreamSynchronize(c->stream2);
        cudaStreamDestroy(c->stream2);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return EMG_OK;
}

const char* emg_last_error(const emg_ctx* c) { return c ? c->err.c_str() : "null context"; }

int64_t emg_device_bytes(const emg_ctx* c) { return c ? c->bytes : 0; }

emg_status emg_set_state(emg_ctx* c, const double* U, int32_t on_device) {
    if (!c || !c->sc) return EMG_ERR_ARG;
    LevelDev& T = c->lv[c->p_max];
    const int64_t n = c->E * T.B;
    if (U) {
        emg_status st = copy_in(c, T.v, U, n, on_device);
        if (st != EMG_OK) return st;
    } else {
        { ProfScope _ps(c, PC_SETUP); k_set_freestream<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(
            c->E, T.N, c->vol, c->uinf[0], c->uinf[1], c->uinf[2], c->uinf[3], c->uinf[4], T.v); }
        EMG_CHECK_LAUNCH(c);
    }
    EMG_CUDA_TRY(c, cudaMemsetAsync(c->sc, 0, sizeof(DevScalars), c->stream));
    { ProfScope _ps(c, PC_CONTROL); k_set_cycle<<<1, 1, 0, c->stream>>>(c->sc, 1); }
    EMG_CHECK_LAUNCH(c);
    emg_status st = launch_check_state(c, T.v, n);
    if (st != EMG_OK) return st;
    st = read_scalars(c);
    if (st != EMG_OK) return st;
    if (c->sc_host->nonfinite) return fail(c, EMG_ERR_NONFINITE, "state contains NaN or Inf");
    c->cycle_n = 1;
    c->res_ref = 0.0;
    c->blocks_valid = false;
    return EMG_OK;
}

emg_status emg_get_state(emg_ctx* c, double* U, int32_t on_device) {
    if (!c || !U) return EMG_ERR_ARG;
    LevelDev& T = c->lv[c->p_max];
    return copy_out(c, U, T.v, c->E * T.B, on_device);
}

emg_status emg_set_cycle(emg_ctx* c, int64_t n, double res_ref) {
    if (!c || n < 1) return EMG_ERR_ARG;
    c->cycle_n = n;
    { ProfScope _ps(c, PC_CONTROL); k_set_ref<<<1, 1, 0, c->stream>>>(c->sc, res_ref > 0.0 ? res_ref : 0.0); }
    EMG_CHECK_LAUNCH(c);
    { ProfScope _ps(c, PC_CONTROL); k_set_cycle<<<1, 1, 0, c->stream>>>(c->sc, (long long)n); }
    EMG_CHECK_LAUNCH(c);
    return EMG_OK;
}

emg_status emg_get_cycle(emg_ctx* c, int64_t* n, double* res_ref) {
    if (!c) return EMG_ERR_ARG;
    emg_status st = read_scalars(c);
    if (st != EMG_OK) return st;
    if (n) *n = c->cycle_n;
    if (res_ref) *res_ref = c->sc_host->res_ref;
    return EMG_OK;
}

emg_status emg_vcycle(emg_ctx* c, emg_cycle_info* info) {
    if (!c) return EMG_ERR_ARG;
    const int64_t n = c->cycle_n;
    emg_status st = vcycle_entry(c);
    if (st != EMG_OK) return st;
    st = run_body(c);
    if (st != EMG_OK) return st;
    c->cycle_n = n + 1;
    if (info) {
        st = read_scalars(c);
        if (st != EMG_OK) return st;
        info->n = n;
        info->res_rho = c->sc_host->res;
        for (int a = 0; a < 5; ++a) info->res[a] = c->sc_host->res5[a];
        info->cfl = c->sc_host->cfl;
        info->krylov_dim = c->sc_host->m_used;
        return check_flags(c);
    }
    return EMG_OK;
}

emg_status emg_solve_steady(emg_ctx* c, double drop, int64_t max_cycles, emg_solve_report* rep) {
    if (!c || !(drop > 0.0) || max_cycles < 0) return EMG_ERR_ARG;
    double r0 = -1.0, res = 0.0;
    int64_t done = 0;
    for (int64_t k = 0; k <= max_cycles; ++k) {
        const int64_t n = c->cycle_n;
        emg_status st = vcycle_entry(c);
        if (st != EMG_OK) return st;
        st = read_scalars(c);
        if (st != EMG_OK) return st;
        st = check_flags(c);
        if (st != EMG_OK) return st;
        res = c->sc_host->res;
        if (r0 < 0.0) r0 = res;
        if (res <= drop * r0 || k == max_cycles) break;
        st = run_body(c);
        if (st != EMG_OK) return st;
        c->cycle_n = n + 1;
        ++done;
    }
    if (rep) {
        rep->cycles = done;
        rep->res0 = r0;
        rep->res_final = res;
        rep->converged = res <= drop * r0 ? 1 : 0;
    }
    if (!(res <= drop * r0)) return fail(c, EMG_ERR_NOT_CONVERGED, "max_cycles reached");
    return EMG_OK;
}

emg_status emg_residual_norm(emg_ctx* c, double* res_rho, double* res5) {
    if (!c) return EMG_ERR_ARG;
    LevelDev& T = c->lv[c->p_max];
    emg_status st = launch_residual(c, c->p_max, T.v, nullptr, T.r2);
    if (st != EMG_OK) return st;
    st = launch_norm_cfl(c, T.r2, 0);
    if (st != EMG_OK) return st;
    st = read_scalars(c);
    if (st != EMG_OK) return st;
    if (res_rho) *res_rho = c->sc_host->res;
    if (res5)
        for (int a = 0; a < 5; ++a) res5[a] = c->sc_host->res5[a];
    return c->sc_host->nonfinite ? fail(c, EMG_ERR_NONFINITE, "non-finite residual") : EMG_OK;
}

emg_status emg_residual(emg_ctx* c, int32_t p, const double* u, double* R, int32_t on_device) {
    if (!c || !u || !R || p < 0 || p > c->p_max) return EMG_ERR_ARG;
    const int64_t n = c->E * c->lv[p].B;
    const double* ud = u;
    double* Rd = R;
    if (!on_device) {
        emg_status st = copy_in(c, c->stage_in, u, n, 0);
        if (st != EMG_OK) return st;
        ud = c->stage_in;
        st = stage_out(c, n, &Rd);
        if (st != EMG_OK) return st;
    }
    emg_status st = launch_residual(c, p, ud, nullptr, Rd);
    if (st != EMG_OK) return st;
    if (!on_device) return copy_out(c, R, Rd, n, 0);
    return EMG_OK;
}

emg_status emg_jacobian_diag(emg_ctx* c, int32_t p, const double* u, double* D, int32_t on_device) {
    if (!c || !u || !D || p < 0 || p > c->p_max) return EMG_ERR_ARG;
    const int B = c->lv[p].B;
    const int64_t n = c->E * B;
    const double* ud = u;
    double* Dd = D;
    if (!on_device) {
        emg_status st = copy_in(c, c->stage_in, u, n, 0);
        if (st != EMG_OK) return st;
        ud = c->stage_in;
        st = stage_out(c, n * B, &Dd);
        if (st != EMG_OK) return st;
    }
    emg_status st = launch_diag_blocks(c, p, ud, &c->sc->cfl, 0, Dd);
    if (st != EMG_OK) return st;
    if (!on_device) return copy_out(c, D, Dd, n * B, 0);
    return EMG_OK;
}

emg_status emg_prk_step(emg_ctx* c, int32_t p, const double* u, const double* tau, double cfl, double* u_out,
                        int32_t on_device) {
    if (!c || !u || !u_out || p < 1 || p > c->p_max || !(cfl > 0.0)) return EMG_ERR_ARG;
    LevelDev& L = c->lv[p];
    const int64_t n = c->E * L.B;
    emg_status st = copy_in(c, L.v, u, n, on_device);
    if (st != EMG_OK) return st;
    if (tau) {
        st = copy_in(c, L.tau, tau, n, on_device);
        if (st != EMG_OK) return st;
    }
    { ProfScope _ps(c, PC_CONTROL); k_set_cfl<<<1, 1, 0, c->stream>>>(c->sc, cfl); }
    EMG_CHECK_LAUNCH(c);
    c->blocks_valid = false;   // the level's stored factors are replaced
    st = prk_step(c, p, tau ? L.tau : nullptr, nullptr);
    if (st != EMG_OK) return st;
    return copy_out(c, u_out, L.v, n, on_device);
}

emg_status emg_block_operator(emg_ctx* c, int32_t p, const double* u, double cfl, int32_t which, double* out,
                              int32_t on_device) {
    if (!c || !u || !out || p < 1 || p > c->p_max || !(cfl > 0.0) || (which != 0 && which != 1)) return EMG_ERR_ARG;
    const bool f32 = blocks_f32(c->prm.prec);
    if (which == 1 && !f32) return fail(c, EMG_ERR_ARG, "the FP64 form keeps LU factors, not an explicit inverse");
    LevelDev& L = c->lv[p];
    const int B = L.B;
    const int64_t n = c->E * B;
    emg_status st = copy_in(c, L.un, u, n, on_device);
    if (st != EMG_OK) return st;
    { ProfScope _ps(c, PC_CONTROL); k_set_cfl<<<1, 1, 0, c->stream>>>(c->sc, cfl); }
    EMG_CHECK_LAUNCH(c);
    c->blocks_valid = false;   // the level's stored factors are replaced
    double* Dd = out;
    if (!on_device) {
        st = stage_out(c, n * B, &Dd);
        if (st != EMG_OK) return st;
    }
    if (f32) {
        st = launch_diag_blocks32(c, p, L.un, &c->sc->cfl, 1, L.blk32);
        if (st != EMG_OK) return st;
        if (which == 1) {
            st = launch_lu32(c, p);
            if (st != EMG_OK) return st;
        }
        const int64_t tot = n * B;
        { ProfScope _ps(c, PC_CONTROL); k_widen_blocks<<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(
            c->E, B, L.blk32, which, Dd); }
        EMG_CHECK_LAUNCH(c);
    } else {
        st = launch_diag_blocks(c, p, L.un, &c->sc->cfl, 1, L.blk);
        if (st != EMG_OK) return st;
        EMG_CUDA_TRY(c, cudaMemcpyAsync(Dd, L.blk, (size_t)n * B * 8, cudaMemcpyDeviceToDevice, c->stream));
    }
    if (!on_device) return copy_out(c, out, Dd, n * B, 0);
    return EMG_OK;
}

emg_status emg_jacobian_p0(emg_ctx* c, const double* u0, double* diag, double* off, int64_t* nbr, int32_t on_device) {
    if (!c || !u0) return EMG_ERR_ARG;
    const int NF = 2 * c->dim;
    const int64_t n = c->E * 5;
    const double* ud = u0;
    if (!on_device) {
        emg_status st = copy_in(c, c->stage_in, u0, n, 0);
        if (st != EMG_OK) return st;
        ud = c->stage_in;
    }
    emg_status st = launch_face_jacobian(c, 0, ud);
    if (st != EMG_OK) return st;
    st = launch_bsr0(c);
    if (st != EMG_OK) return st;
    std::vector<double> hb((size_t)c->E * (1 + NF) * 25);
    EMG_CUDA_TRY(c, cudaMemcpyAsync(hb.data(), c->bsr, hb.size() * 8, cudaMemcpyDeviceToHost, c->stream));
    std::vector<int> hn((size_t)c->E * NF);
    EMG_CUDA_TRY(c, cudaMemcpyAsync(hn.data(), c->elem_nbr, hn.size() * 4, cudaMemcpyDeviceToHost, c->stream));
    st = sync(c);
    if (st != EMG_OK) return st;
    // unpacking is layout conversion only
    std::vector<double> hd((size_t)c->E * 25), ho((size_t)c->E * NF * 25);
    for (int64_t e = 0; e < c->E; ++e) {
        std::memcpy(&hd[e * 25], &hb[e * (1 + NF) * 25], 25 * 8);
        std::memcpy(&ho[e * NF * 25], &hb[e * (1 + NF) * 25 + 25], NF * 25 * 8);
    }
    if (diag) {
        if (on_device)
            EMG_CUDA_TRY(c, cudaMemcpy(diag, hd.data(), hd.size() * 8, cudaMemcpyHostToDevice));
        else
            std::memcpy(diag, hd.data(), hd.size() * 8);
    }
    if (off) {
        if (on_device)
            EMG_CUDA_TRY(c, cudaMemcpy(off, ho.data(), ho.size() * 8, cudaMemcpyHostToDevice));
        else
            std::memcpy(off, ho.data(), ho.size() * 8);
    }
    if (nbr)
        for (size_t i = 0; i < hn.size(); ++i) nbr[i] = hn[i];
    return EMG_OK;
}

emg_status emg_exp1_step(emg_ctx* c, const double* u0, const double* tau0, const double* dt, double* u_out,
                         int32_t* krylov_dim, int32_t on_device) {
    if (!c || !u0 || !dt || !u_out) return EMG_ERR_ARG;
    LevelDev& L = c->lv[0];
    const int64_t n = c->E * 5;
    emg_status st = copy_in(c, c->stage_in, u0, n, on_device);
    if (st != EMG_OK) return st;
    if (tau0) {
        st = copy_in(c, c->stage_in2, tau0, n, on_device);
        if (st != EMG_OK) return st;
    }
    st = copy_in(c, c->stage_small, dt, c->E, on_device);
    if (st != EMG_OK) return st;
    double* so = nullptr;
    st = stage_out(c, n, &so);
    if (st != EMG_OK) return st;
    st = launch_exp1(c, c->stage_in, tau0 ? c->stage_in2 : nullptr, c->stage_small, so);
    if (st != EMG_OK) return st;
    (void)L;
    st = copy_out(c, u_out, so, n, on_device);
    if (st != EMG_OK) return st;
    st = read_scalars(c);
    if (st != EMG_OK) return st;
    if (krylov_dim) *krylov_dim = c->sc_host->m_used;
    return check_flags(c);
}

static const char* kClassNames[PC_COUNT] = {"residual_face_flux", "residual_volume", "face_jacobian",
                                            "diag_block_assembly", "block_lu", "prk_stage_solve", "p0_bsr",
                                            "arnoldi", "phi1_pade", "krylov_combine", "level_transfer",
                                            "norm_cfl_dtau", "setup"};

emg_status emg_profile_enable(emg_ctx* c, int32_t on) {
    if (!c) return EMG_ERR_ARG;
    prof_flush(c);
    if (on && c->prof.ev.empty()) {
        c->prof.ev.resize(16384);
        c->prof.pair_cls.resize(8192);
        for (auto& e : c->prof.ev) EMG_CUDA_TRY(c, cudaEventCreate(&e));
    }
    for (int k = 0; k < PC_COUNT; ++k) {
        c->prof.ms[k] = 0.0;
        c->prof.cnt[k] = 0;
    }
    c->prof.on = on != 0;
    return EMG_OK;
}

emg_status emg_profile_read(emg_ctx* c, int32_t cls, double* total_ms, int64_t* launches) {
    if (!c || cls < 0 || cls >= PC_COUNT) return EMG_ERR_ARG;
    prof_flush(c);
    if (total_ms) *total_ms = c->prof.ms[cls];
    if (launches) *launches = c->prof.cnt[cls];
    return EMG_OK;
}

const char* emg_profile_class_name(int32_t cls) {
    return (cls >= 0 && cls < PC_COUNT) ? kClassNames[cls] : nullptr;
}

int64_t emg_launch_count(const emg_ctx* c) { return c ? c->launches : 0; }

const char* emg_tuning(const emg_ctx* c) { return c ? c->tuning.c_str() : ""; }

int64_t emg_graph_kernels(const emg_ctx* c) { return c && c->body_exec ? c->body_kernels : 0; }

emg_status emg_selftest_wait_timeout(emg_ctx* c) {
    if (!c) return EMG_ERR_ARG;
    int flag = 0;
    emg_status st = selftest_barrier_timeout(c, &flag);
    if (st != EMG_OK) return st;
    if (!flag) return fail(c, EMG_ERR_CUDA, "bounded wait did not report its timeout");
    return fail(c, EMG_ERR_TIMEOUT, "bounded wait gave up as designed");
}

emg_status emg_element_geometry(emg_ctx* c, double* vol, double* h) {
    if (!c) return EMG_ERR_ARG;
    if (vol) EMG_CUDA_TRY(c, cudaMemcpyAsync(vol, c->vol, c->E * 8, cudaMemcpyDeviceToHost, c->stream));
    if (h) EMG_CUDA_TRY(c, cudaMemcpyAsync(h, c->h, c->E * 8, cudaMemcpyDeviceToHost, c->stream));
    return sync(c);
}

}  // extern "C"
