/*
 * emg.h -- C ABI of the GB300 exponential p-multigrid (eMG) solver for the steady
 * compressible Euler equations with a modal discontinuous Galerkin discretisation
 * (Li, "Efficient p-multigrid method based on an exponential time discretization
 * for compressible steady flows", arXiv:1807.01151).
 *
 * Conventions for every call:
 *   - Plain C types only; no exceptions cross the boundary.  Every call returns an
 *     emg_status; on failure emg_last_error(ctx) holds a one-line message.
 *   - A context owns all device memory it allocates (freed by emg_destroy).  Caller
 *     arrays are only read/written during the call.
 *   - `on_device` = 0: the pointer is host memory (pageable or pinned); the call
 *     copies through the context's stream and returns after the data is in place.
 *     `on_device` = 1: the pointer is device memory on the context's device; work is
 *     enqueued on the context's stream and the call returns without synchronising,
 *     except where a host-visible scalar output (emg_cycle_info, norms, Krylov
 *     dimension) is requested, which synchronises the stream.
 *   - Within a call the context may fork work onto a second stream it owns (residual
 *     evaluations that run beside a level's block build) and joins it back before the
 *     call's next dependent step, so that seen from the caller every call stays ordered
 *     on the context's stream (in the V-cycle graphs the context captures itself, the
 *     fork and the join are graph edges).
 *   - Modal states use the canonical layout [n_elems][5][N_p] (float64), variables
 *     (rho, rho u, rho v, rho w, rho E) (rho w is kept, and stays 0, in 2-D), modes
 *     in the basis order: total degree 0..p, within a degree x exponent descending,
 *     then y (then z).  N_p = (p+1)(p+2)/2 in 2-D, (p+1)(p+2)(p+3)/6 in 3-D.
 *   - A context is not thread-safe; distinct contexts may be used concurrently.
 */
#ifndef EMG_H
#define EMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct emg_ctx emg_ctx;

typedef enum {
    EMG_OK = 0,
    EMG_ERR_ARG = 1,           /* invalid argument or unsupported configuration      */
    EMG_ERR_OOM = 2,           /* admission: the context does not fit in free memory */
    EMG_ERR_CUDA = 3,          /* a CUDA runtime call failed                         */
    EMG_ERR_NONFINITE = 4,     /* NaN/Inf in a state or residual                      */
    EMG_ERR_UNPHYSICAL = 5,    /* non-positive density or pressure at a cell centre  */
    EMG_ERR_NOT_CONVERGED = 6, /* emg_solve_steady reached max_cycles                 */
    EMG_ERR_TIMEOUT = 7,       /* a bounded device-side wait gave up                  */
    EMG_CANCELLED = 8          /* a served request withdrawn by emg_server_cancel     */
} emg_status;

/* Boundary codes of emg_mesh_desc.face_bc. */
#define EMG_BC_INTERIOR (-1)
#define EMG_BC_WALL 1      /* inviscid slip wall: ghost with mirrored normal velocity (Sec. 3.3) */
#define EMG_BC_FARFIELD 2  /* characteristic far field from 1-D Riemann invariants (Sec. 5)     */
#define EMG_BC_SYMMETRY 3  /* symmetry plane of the sphere case (Sec. 5): ghost state with the
                              velocity mirrored about the (flat) face normal                   */

typedef enum {
    EMG_PREC_FP64 = 0,        /* every step in float64                                   */
    EMG_PREC_FP32_BLOCKS = 1, /* PRK block assembly, LU and solves in float32; residual,
                                 Arnoldi and phi_1 in float64                             */
    EMG_PREC_BF16_BLOCKS = 2  /* as EMG_PREC_FP32_BLOCKS, but the block assembly multiplies
                                 bfloat16 operands (float32 accumulation)                 */
} emg_prec;

/* Mesh of straight-sided bilinear quadrilaterals (dim 2) or trilinear hexahedra (dim 3).
 * xyz: [dim][n_nodes] (structure of arrays).  elem_nodes: [n_elems][2^dim], reference
 * node order (-1,-1),(1,-1),(1,1),(-1,1) (quads); the same at zeta=-1 then zeta=+1
 * (hexes); the map must have a positive Jacobian determinant.  face_bc: [n_elems][2*dim],
 * local face f = 2*axis + (side > 0) (xi-, xi+, eta-, eta+, zeta-, zeta+); -1 marks an
 * interior face whose neighbour is found by matching its nodes.
 * wall_normal: optional [dim][n_nodes] unit normal of the true (curved) body at the
 * nodes of wall faces (other entries are ignored), or NULL.  The paper's meshes are
 * curved (Sec. 5); on straight-sided elements the slip-wall ghost state mirrors the
 * velocity about the body normal interpolated from these node normals (normalised
 * multilinear interpolation along the face), while fluxes are integrated on the flat
 * faces.  NULL mirrors about the flat face normal. */
typedef struct {
    int32_t dim;
    int64_t n_nodes;
    const double* xyz;
    int64_t n_elems;
    const int64_t* elem_nodes;
    const int32_t* face_bc;
    const double* wall_normal;
} emg_mesh_desc;

typedef struct {
    double gamma;          /* ratio of specific heats (7/5, Sec. 3)                         */
    double mach;           /* free-stream Mach number; rho = 1, p = 1/gamma                  */
    double alpha_deg;      /* free-stream angle in the x-y plane                              */
    int32_t p_max;         /* finest DG degree, 0..4                                          */
    int32_t rk_stages;     /* s of Eq. prk_scalar (paper: 4)                                  */
    int32_t krylov_m;      /* Krylov dimension of the EXP1 step (paper: 30), 1..40             */
    double cfl_max;        /* CFL_max of Eq. cfl (paper: 100 for eMG)                         */
    double exp_dt_factor;  /* EXP1 step = factor * dtau(p_max); <= 0 selects p_max + 1 (Sec. 4) */
    int32_t pre_smooth;    /* PRK steps per level on the down leg (default 2)                 */
    int32_t prec;          /* emg_prec                                                         */
    void* cuda_stream;     /* cudaStream_t to run on; NULL = a stream owned by the context     */
    int32_t lag_blocks;    /* 1: factor P_e once per level per V-cycle and reuse it for every
                              PRK step of that level (a lagged preconditioner; the fixed point
                              R = 0 is unchanged); 0 (default): P(u^n) at every step         */
    int32_t use_graph;     /* 1 (default): the V-cycle body (every level's smoother, transfers,
                              EXP1) is captured once into a CUDA graph and replayed each cycle;
                              0: launched kernel by kernel.  The same kernels run either way and
                              give bitwise the same result.  The event profiler, when on, uses
                              the kernel-by-kernel path. */
    int32_t autotune;      /* 1 (default): at creation, time the variants of the tuned kernels
                              (FP32 Gauss-Jordan: warps per block) per block size on this
                              device and use the fastest (cached per process); 0: the first
                              variant.  Variants compute identically: results do not change. */
    int32_t coop_krylov;   /* 1 (default): the Arnoldi process of the EXP1 step is one persistent
                              cooperative kernel with bounded grid barriers; 0: the same process
                              as 2 + 3m plain kernels with no grid barrier (bitwise the same
                              result), for contexts that share the device with other work, where
                              the blocks of a persistent kernel may not all be resident at once
                              (the request loop uses 0). */
    double krylov_tol;     /* 0 (default): the Arnoldi process takes krylov_m steps (or stops at
                              happy breakdown).  > 0: the Krylov tolerance of Sec. 5 (paper:
                              1e-5); step j ends the process when the leading term of the phi_1
                              error series, beta h_{j+1,j} |(phi_2(H_j) e_1)_j|, is at most
                              krylov_tol * beta ||phi_1(H_j) e_1|| (phi_1 and phi_2 from one
                              exponential of the (j+2)-augmented Hessenberg matrix). */
    int32_t exp_dt_global; /* 0 (default): local EXP1 steps dt_e = factor * dtau_e (p = p_max);
                              1: one step for the whole mesh, min_e dt_e (Eq. EXP1 as written) */
    int32_t jac_freeze;    /* k >= 1: the PRK block factors of every level are assembled and
                              factored in V-cycles n with (n - 1) mod k = 0 only and reused by the
                              other cycles (a frozen preconditioner; the fixed point R = 0 is
                              unchanged).  1 (default): every cycle. */
    int32_t quad_extra;    /* q = p + quad_extra Gauss points per direction and level; only the
                              rule q = p + 2 is built (2, the default; 0 is read as 2) */
    double omega[3];       /* angular velocity of the rotating frame (Eq. euler), (0, 0, 0)
                              by default (an absolute frame).  Otherwise the state keeps the
                              absolute velocity v; mass and momentum are carried by the velocity
                              relative to the frame, v - v_r with v_r = omega x x; the energy
                              flux is rho E (v - v_r) + p v (what the Appendix's Jacobian
                              differentiates); the source -rho omega x v is added; walls are at
                              rest in the frame (the relative velocity is mirrored) and the far
                              field takes the free stream (absolute frame) through the same
                              characteristic condition in relative velocities.  In 2-D only a
                              rotation about z, omega = (0, 0, w), is accepted (else
                              EMG_ERR_ARG); non-finite values: EMG_ERR_ARG. */
    int32_t block_kernels; /* kernels of the float32 block forms' assembly and inverse:
                              0 (default): per level, the form measured faster on GB300;
                              1: the tensor-core forms (tcgen05: 3xTF32 assembly, blocked
                              Gauss-Jordan with rank-16 MMA updates for B = 75, 100, 175);
                              2: the SIMT (FMA) forms (blocked Gauss-Jordan with rank-8
                              updates where a thread's share fits 64 registers, else the
                              unblocked column-owner form); 3: the SIMT forms with the
                              unblocked Gauss-Jordan everywhere.  The forms differ only in
                              rounding; the BF16 form always assembles on the tensor cores. */
    int32_t krylov_f32;    /* precision of the Arnoldi process of the EXP1 step: 1: its basis,
                              products, dot products and reductions in float32 (the Hessenberg
                              matrix, phi_1 and the combination stay FP64; happy breakdown at
                              h_{j+1,j} <= 1e-5 ||A v_j||); 0: all FP64; -1 (default): float32
                              with the float32 block forms (EMG_PREC_FP32_BLOCKS,
                              EMG_PREC_BF16_BLOCKS), FP64 with EMG_PREC_FP64.  The EXP1 step only
                              corrects the coarse level, so the fixed point R = 0 is unchanged
                              (as with the float32 block factors).  Other values: EMG_ERR_ARG. */
} emg_params;

typedef struct {
    int64_t n;             /* index of the V-cycle just run (1-based)                         */
    double res_rho;        /* ||R(rho)|| of Eq. cfl at the state entering this cycle          */
    double res[5];         /* the same norm for each conservative variable                   */
    double cfl;            /* CFL_n used by this cycle                                        */
    int32_t krylov_dim;    /* Arnoldi steps taken by the EXP1 step                            */
} emg_cycle_info;

typedef struct {
    int64_t cycles;        /* V-cycles run                                                    */
    double res0;           /* ||R(rho)|| of the initial state                                 */
    double res_final;      /* ||R(rho)|| of the returned state                                */
    int32_t converged;     /* 1 if res_final <= drop * res0                                    */
} emg_solve_report;

/* Fill p with the paper's defaults (gamma 1.4, Ma 0.3, alpha 0, p_max 2, s = 4, m = 30,
 * CFL_max = 100, EXP1 factor p_max+1, 2 PRK steps per level, FP64, own stream). */
void emg_default_params(emg_params* p);

/* Build connectivity, geometry (|E|, x_c, half bounding box L, |dE|, h = 2d|E|/|dE|,
 * Eq. x3d), the orthonormal Cartesian basis of Eqs. basis2/basis by modified
 * Gram-Schmidt and the quadrature tables of every level (Gauss-Legendre, q = p + 2 per
 * direction), all on the device.  Admission: fails with EMG_ERR_OOM, allocating
 * nothing, when the estimated footprint exceeds the device's free memory.  The state is
 * initialised to the free stream. */
emg_status emg_create_mesh(const emg_mesh_desc* mesh, const emg_params* params, emg_ctx** out);
emg_status emg_destroy(emg_ctx* ctx);
const char* emg_last_error(const emg_ctx* ctx);

/* Bytes of device memory the context holds. */
int64_t emg_device_bytes(const emg_ctx* ctx);

/* Set / get the p_max state, [n_elems][5][N_pmax].  U = NULL in emg_set_state selects the
 * free stream.  emg_set_state restarts the CFL schedule of Eq. cfl (cycle counter 1,
 * reference residual unset) and rejects non-finite input (EMG_ERR_NONFINITE). */
emg_status emg_set_state(emg_ctx* ctx, const double* U, int32_t on_device);
emg_status emg_get_state(emg_ctx* ctx, double* U, int32_t on_device);

/* CFL schedule state (Eq. cfl): the index of the next V-cycle and the reference
 * residual ||R(rho_1)|| (<= 0: taken from the next cycle).  For checkpoint/resume. */
emg_status emg_set_cycle(emg_ctx* ctx, int64_t n, double res_ref);
emg_status emg_get_cycle(emg_ctx* ctx, int64_t* n, double* res_ref);

/* One FAS V-cycle p_max -> 0 -> p_max (Sec. 2.3): params.pre_smooth PRK steps (Eq.
 * prk_scalar; default 2) per level p >= 1 on the down leg, with exact element-diagonal
 * Jacobian blocks (Eq. jac1) and P = I/dtau - dR/du, restriction/forcing, one EXP1 step
 * (Eq. EXP1) with an Arnoldi phi_1 product (Eqs. vm, final) on p = 0, prolongation and
 * correction, no post-smoothing.  info may be NULL (then nothing is read back). */
emg_status emg_vcycle(emg_ctx* ctx, emg_cycle_info* info);

/* Run V-cycles until ||R(rho)|| <= drop * ||R(rho)|| of the entry state, or max_cycles.
 * Returns EMG_ERR_NOT_CONVERGED (report still filled) when the cap is reached. */
emg_status emg_solve_steady(emg_ctx* ctx, double drop, int64_t max_cycles, emg_solve_report* report);

/* ||R(rho)|| (Eq. cfl) and the per-variable norms of the current p_max state. */
emg_status emg_residual_norm(emg_ctx* ctx, double* res_rho, double* res5);

/* ---- component entry points (same kernels as emg_vcycle; used by parity tests) ---- */

/* R_p(u) of Eq. euler3, u and R [n_elems][5][N_p]. */
emg_status emg_residual(emg_ctx* ctx, int32_t p, const double* u, double* R, int32_t on_device);

/* Element-diagonal Jacobian blocks D_e = dR_{p,e}/du_e (Eq. jac1, with the boundary chain
 * rule of Sec. 3.3), [n_elems][5 N_p][5 N_p] row-major, row/column index var*N_p + mode. */
emg_status emg_jacobian_diag(emg_ctx* ctx, int32_t p, const double* u, double* D, int32_t on_device);

/* One PRK step (Eq. prk_scalar) at level p >= 1 from u with forcing tau (NULL = 0) at the
 * given CFL: P_e = I/dtau_e - D_e(u), dtau_e of Eq. x3d. */
emg_status emg_prk_step(emg_ctx* ctx, int32_t p, const double* u, const double* tau, double cfl,
                        double* u_out, int32_t on_device);

/* p = 0 Jacobian in block-sparse form (Eqs. jac1, jac2): diag [n_elems][5][5],
 * off [n_elems][2 dim][5][5] (dR_e/du_nb across local face f; zero on boundaries),
 * nbr [n_elems][2 dim] (neighbour index or -1). */
emg_status emg_jacobian_p0(emg_ctx* ctx, const double* u0, double* diag, double* off, int64_t* nbr,
                           int32_t on_device);

/* One EXP1 step on level 0 (Eq. EXP1): u0 + phi_1(DT J_0) DT (R_0(u0) + tau0), DT =
 * diag(dt_e); tau0 may be NULL.  krylov_dim receives the Arnoldi steps taken. */
emg_status emg_exp1_step(emg_ctx* ctx, const double* u0, const double* tau0, const double* dt,
                         double* u_out, int32_t* krylov_dim, int32_t on_device);

/* ---- EXP1 step that allocates nothing (the paper has no counterpart) ----
 * For callers that cannot allocate device memory once they are running: an application
 * whose device memory is handed out only by its own pool (a caching allocator that already
 * holds what the device has free, so a cudaMalloc would fail), or a loop that may not stall
 * on the implicit device-wide synchronisation a cudaMalloc/cudaFree can take.  The step is the same
 * as emg_exp1_step (u_out = u0 + phi_1(DT J_0) DT r0, m Arnoldi steps with happy
 * breakdown, Pade phi_1), but it takes the p = 0 Jacobian in the block form that
 * emg_jacobian_p0 returns and the residual r0 = R~_0(u0), and needs no context.
 * Its work memory is one file-scope device array of about 26 MB, which every GPU that
 * loads this library holds until the process exits; no call makes or frees an
 * allocation.  Limits: n_elems <= 8192, krylov_m <= 40, dim 2 or 3; larger requests fail
 * with EMG_ERR_ARG.
 * All array arguments are device pointers on the current device: diag [n_elems][5][5],
 * off [n_elems][2 dim][5][5], nbr [n_elems][2 dim] (neighbour or -1), r0 and u0 and
 * u_out [n_elems][5], dt [n_elems].  Work is enqueued on cuda_stream (NULL = the legacy
 * default stream); the call then reads the Krylov dimension and the status flags back
 * and synchronises that stream before it returns (krylov_dim may be NULL).
 * The first call on a device looks up the array's device address with that device
 * current (once per device, safe from several host threads); make that first call
 * before any stream capture.  Every neighbour index must be -1 or in [0, n_elems): the
 * packing kernel checks each one and the call returns EMG_ERR_ARG, without running the
 * Krylov step, if any is out of range.  Every call on a device
 * shares the one array and finds the previous call's contents in it (the call clears
 * what must start at zero), so calls whose work overlaps on the GPU, from several
 * streams or host threads, race and must be serialised by the caller.
 * Returns EMG_ERR_TIMEOUT or EMG_ERR_NONFINITE like emg_exp1_step, EMG_ERR_CUDA on a
 * runtime failure (no per-call message: there is no context). */
emg_status emg_exp1_step_noalloc(int32_t dim, int64_t n_elems, const double* diag, const double* off,
                                 const int64_t* nbr, const double* r0, const double* dt, const double* u0,
                                 int32_t krylov_m, void* cuda_stream, double* u_out, int32_t* krylov_dim);

/* The block operator the PRK stages of level p apply (Eq. prk_scalar), in the context's
 * precision form, for the state u [n_elems][5][N_p] at the given CFL:
 *   which = 0: P_e = I/dtau_e - D_e(u) as assembled (Eq. jac1 with dtau_e of Eq. x3d);
 *   which = 1: P_e^{-1} as the stages apply it (the float32 explicit inverse of the
 *              EMG_PREC_FP32_BLOCKS and EMG_PREC_BF16_BLOCKS forms; EMG_ERR_ARG for the
 *              FP64 form, which keeps LU factors instead).
 * out: [n_elems][5 N_p][5 N_p] float64, row-major, row/column index var*N_p + mode (float32
 * values widened exactly).  Uses (and overwrites) the level's block storage. */
emg_status emg_block_operator(emg_ctx* ctx, int32_t p, const double* u, double cfl, int32_t which,
                              double* out, int32_t on_device);

/* Element volumes |E| and length scales h = 2d|E|/|dE| (Eq. x3d), [n_elems] each. */
emg_status emg_element_geometry(emg_ctx* ctx, double* vol, double* h);

/* ---- tracing (no counterpart in the paper) ----
 * Event profiler: when enabled, every kernel launch of the context is bracketed by CUDA
 * events on the context's stream and its time accumulated per kernel class (class ids
 * 0..12, names from emg_profile_class_name).  Enabling or disabling resets the totals.
 * emg_profile_read synchronises the stream. */
emg_status emg_profile_enable(emg_ctx* ctx, int32_t on);
emg_status emg_profile_read(emg_ctx* ctx, int32_t cls, double* total_ms, int64_t* launches);
const char* emg_profile_class_name(int32_t cls);
/* Number of kernels the context has launched since creation (a graph replay counts the
 * kernels it holds). */
int64_t emg_launch_count(const emg_ctx* ctx);
/* The tuner's choices and timings for this context (empty when nothing was tuned). */
const char* emg_tuning(const emg_ctx* ctx);
/* Kernels in the captured V-cycle graph; 0 before the first cycle, with use_graph = 0, or
 * if the capture failed (then the body runs kernel by kernel). */
int64_t emg_graph_kernels(const emg_ctx* ctx);

/* ---- failure detection (no counterpart in the paper) ----
 * Every device-side wait (the grid barriers of the persistent Arnoldi kernel) gives up
 * after a bounded number of clock cycles, records the timeout and returns, and the call
 * reports EMG_ERR_TIMEOUT with the context still usable.  This self-test launches one
 * block at a barrier that expects two, so the wait runs out (~0.1 s); it returns
 * EMG_ERR_TIMEOUT when the bounded wait works and clears the flag afterwards. */
emg_status emg_selftest_wait_timeout(emg_ctx* ctx);

/* Device bytes emg_create_mesh would allocate for this mesh and these parameters (the
 * admission estimate; equal to emg_device_bytes of the context it creates).  Host only. */
emg_status emg_estimate_device_bytes(const emg_mesh_desc* mesh, const emg_params* params, int64_t* bytes);

/* ---- request loop with continuous batching (no counterpart in the paper) ----
 * A server runs many steady solves (emg_solve_steady semantics: V-cycles until
 * ||R(rho)|| <= drop * ||R(rho)|| of the first cycle) of different meshes, orders and
 * Mach numbers as they arrive.  Requests wait in submission order; the head request is
 * admitted when one of max_active slots is free and its footprint
 * (emg_estimate_device_bytes) fits in what the memory budget has left.  An admitted solve
 * owns a context (its own stream; state, blocks and Krylov arrays resident on the device
 * until it ends; its Arnoldi process runs as plain kernels, coop_krylov = 0, since no
 * kernel of a solve may wait for blocks that other solves' work keeps off the SMs) and
 * keeps one V-cycle in flight; emg_server_step only polls events and
 * enqueues the next cycle of every solve whose residual check has arrived, so the cycles
 * of different solves overlap on the device.  A solve ends converged (EMG_OK), at
 * max_cycles (EMG_ERR_NOT_CONVERGED), or with its own failure status; the others carry
 * on.  The arithmetic of a solve depends on nothing outside its context (fixed-order
 * reductions, no atomics), so its result is bitwise the same alone and in the mix.
 * The caller's arrays are copied by emg_server_submit.  One host thread drives a server
 * (not thread-safe); different servers are independent. */
typedef struct emg_server emg_server;

typedef struct {
    int64_t mem_budget;  /* device bytes the active solves may hold together; <= 0: 90 % of free memory */
    int32_t max_active;  /* slots: solves in flight at once, >= 1 */
    double drop;         /* relative drop of ||R(rho)|| that ends a solve (> 0), e.g. 1e-10 */
    int64_t max_cycles;  /* V-cycles per solve (>= 0) */
    int32_t keep_state;  /* 1: keep each converged state on the host for emg_server_take_state */
    int64_t stall_cycles; /* > 0: a solve whose ||R(rho)|| has set no new minimum for this many
                             cycles ends with EMG_ERR_NOT_CONVERGED; 0: only max_cycles ends it */
} emg_server_params;

typedef struct {
    int64_t id;           /* from emg_server_submit */
    emg_status status;    /* EMG_OK = converged; EMG_ERR_OOM = does not fit the budget; ... */
    int64_t cycles;       /* V-cycles done */
    double res0;          /* ||R(rho)|| at the first cycle */
    double res_final;     /* ||R(rho)|| at the last check */
    double t_submit;      /* seconds on the server clock (emg_server_clock) */
    double t_admit;
    double t_done;
    int64_t device_bytes; /* the admission estimate */
} emg_request_result;

emg_status emg_server_create(const emg_server_params* params, emg_server** out);
/* Waits for and frees the active solves; queued requests are dropped. */
emg_status emg_server_destroy(emg_server* srv);
const char* emg_server_last_error(const emg_server* srv);
/* Seconds since the server's creation (host steady clock). */
double emg_server_clock(const emg_server* srv);
/* Queue one solve.  mesh and params as for emg_create_mesh (params->cuda_stream is
 * ignored: each solve gets its own stream); U0 [n_elems][5][N_pmax] on the host, or NULL
 * for the free stream.  id receives the request id (0, 1, 2, ... per server). */
emg_status emg_server_submit(emg_server* srv, const emg_mesh_desc* mesh, const emg_params* params,
                             const double* U0, int64_t* id);
/* One scheduling round, without waiting: advance every solve whose last residual check
 * has arrived, retire the finished ones, admit queued requests.  Returns the number of
 * active and queued requests. */
emg_status emg_server_step(emg_server* srv, int32_t* n_active, int32_t* n_queued);
/* Move up to capacity finished requests' results (in completion order) into out. */
emg_status emg_server_results(emg_server* srv, emg_request_result* out, int32_t capacity, int32_t* n_out);
/* Withdraw request id: a queued request is dropped; an active one ends before its next
 * cycle is enqueued (the cycle in flight completes first), its context and memory are
 * released.  Its result (status EMG_CANCELLED, the cycles done) is then reported by
 * emg_server_results.  EMG_ERR_ARG if id is unknown or has already finished. */
emg_status emg_server_cancel(emg_server* srv, int64_t id);
/* Copy the kept converged state of request id ([n_elems][5][N_pmax], n doubles) to host
 * memory and release it.  EMG_ERR_ARG if none is kept or n does not match. */
emg_status emg_server_take_state(emg_server* srv, int64_t id, double* U, int64_t n);

/* ---- arithmetic peaks of the current device (no counterpart in the paper) ----
 * Register-only multiply-add loops (every block of the grid resident, 8 independent
 * chains per thread, no memory traffic in the timed loop), timed with CUDA events:
 * float64 and float32 FMA throughput in TFLOP/s (2 flop per FMA).  These are the
 * denominators of the ALU rooflines of the FP64 residual and the FP32 block kernels.
 * sm_mhz receives the SM clock the device reports for the run (may be NULL). */
emg_status emg_probe_peaks(double* fp64_tflops, double* fp32_tflops, double* sm_mhz);

/* Build identification string (architecture and kernel variants). */
const char* emg_build_info(void);

#ifdef __cplusplus
}
#endif

#endif /* EMG_H */
