/*
 * bq.h -- C ABI of the GB300 solver for the mapped adjoint Lindblad equation
 * (Makinen et al., "Efficient classical simulation of open bosonic quantum systems").
 *
 * The library integrates the adjoint (Heisenberg-picture) master equation of a measured
 * operator A (Eq. 3) after the paper's mapping of A to generating functions (Eqs. 5-8):
 * every separable initial condition G^(p,q)(0) = x^p y^q (Eqs. 10, 13) is evolved as the
 * coupled system G = G_x G_y + R (Eqs. 9a-c, network form Eqs. 303a-c) with classical RK4,
 * one fused CUDA kernel per RK4 stage.  It also carries the "conventional" direct
 * number-basis integration of Eq. 3 for the paper's comparison.
 *
 * Conventions
 *   - Every function returns an int status: BQ_OK (0) or a negative BQ_E* code.  A
 *     human-readable detail of the last failure on the calling thread is returned by
 *     bq_last_error().  No function aborts the process.
 *   - Problems (bq_problem) and states (bq_state) are opaque, library-owned host handles.
 *   - Device memory is caller-owned: bq_map() carves everything it needs (tables,
 *     state, RK4 scratch) out of one caller-provided device buffer and never frees it.
 *   - Device work is enqueued asynchronously on the caller's CUDA stream (a
 *     cudaStream_t passed as void*, NULL = legacy default stream).  Functions that return
 *     host data synchronise that stream.
 *   - Operators are normal-ordered monomials prod_j (a_j^dag)^u_j a_j^v_j given by the
 *     power arrays u, v of length n_modes (Eq. 1 / Eq. S1, o1 = a^dag, o2 = a, r = 1).
 *   - Time is in ns, angular frequencies in rad/ns.
 *   - There is no CPU fallback: every step of the path runs in this library's kernels.
 */
#ifndef BQ_H_
#define BQ_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------- */
#define BQ_OK 0
#define BQ_EINVAL (-1)        /* bad argument (sizes, indices, non-Hermitian H, ...)   */
#define BQ_EUNSTABLE_DT (-2)  /* dt above the RK4 imaginary-axis stability bound        */
#define BQ_ENOMEM (-3)        /* caller's device buffer too small                      */
#define BQ_ECUDA (-4)         /* a CUDA runtime call failed (detail in bq_last_error)  */
#define BQ_ENONFINITE (-5)    /* NaN/Inf detected in a result                          */
#define BQ_ETIMEOUT (-6)      /* a bounded device wait gave up                         */
#define BQ_EUNSUPPORTED (-7)  /* valid request outside this build's limits             */

/* ---- enums ------------------------------------------------------------------------ */
/* Channel (drive envelope) kinds, Eq. 301's time dependence.  Parameters:
 *   CONST: (re, im)                      value re + i im
 *   GAUSS: (amp_re, amp_im, t0, sigma)   amp exp(-(t - t0)^2 / (2 sigma^2))
 *   PWC:   (t_start, seg_len, re_0, im_0, re_1, im_1, ...)  piecewise constant
 *   CEXP:  (amp_re, amp_im, omega)       amp exp(i omega t)
 * Smooth kinds are evaluated at every RK4 stage time; PWC at the midpoint of each step
 * (the Hamiltonian is held constant within a step).  With reverse_time the physical time
 * of integration time tau is t = horizon - tau (Heisenberg picture of a time-dependent
 * Hamiltonian); otherwise t = tau. */
enum { BQ_CH_CONST = 0, BQ_CH_GAUSS = 1, BQ_CH_PWC = 2, BQ_CH_CEXP = 3 };

enum { BQ_METHOD_MAPPED = 0, BQ_METHOD_DIRECT = 1 };
enum { BQ_F64 = 0, BQ_F32 = 1 };
enum { BQ_R_FULL = 0, BQ_R_OFF = 1, BQ_R_DIAG = 2 };
/* Storage basis of the coefficients: MONOMIAL stores g_{k,l} as in Eq. 6; NUMBER stores
 * sqrt(k! l!) g_{k,l} (a diagonal similarity, exact in exact arithmetic; keeps FP32 in
 * range for large truncations).  AUTO = MONOMIAL for F64 mapped, NUMBER otherwise. */
enum { BQ_BASIS_AUTO = 0, BQ_BASIS_MONOMIAL = 1, BQ_BASIS_NUMBER = 2 };
enum { BQ_C_EQ304 = 0, BQ_C_ZERO = 1 };
/* Separable initial conditions of the mapped method: MONOMIAL = one system x^p y^q per
 * non-zero element of A(0) (Eqs. 10 / 13, weight g_{p,q}(0), C of Eq. 304); SVD = one
 * system per singular value of g(0) seen as a (prod M) x (prod M) matrix above 1e-12 of the
 * largest, G_x(0) = s_i u_i, G_y(0) = conj(v_i), weight 1, C = 0 (at most prod M systems;
 * the summed result equals the monomial one up to the RK4 error of the different C). */
enum { BQ_IC_MONOMIAL = 0, BQ_IC_SVD = 1 };

#define BQ_MAX_MODES 4

typedef struct bq_problem bq_problem;
typedef struct bq_state bq_state;

typedef struct bq_map_opts {
  int method;        /* BQ_METHOD_*                                                     */
  int dtype;         /* BQ_F64 | BQ_F32: arithmetic and storage type of the state       */
  int r_layout;      /* BQ_R_FULL | BQ_R_OFF (R ~ 0 when kappa t << 1, main text after Eq. 9) |
                      * BQ_R_DIAG (R kept only where k = l, i.e. as a function of the products
                      * x_j y_j, the paper's observation with Fig. 2; Eq. 303c projected onto
                      * those entries: exact when the dynamics keep R diagonal, an
                      * approximation of order kappa t otherwise; mapped method, tiled stage
                      * kernel; bq_grad differentiates the projected system).  bq_read_system
                      * returns R expanded to n_g x n_g. */
  int basis;         /* BQ_BASIS_*                                                      */
  int c_mode;        /* BQ_C_EQ304 | BQ_C_ZERO: separation constant                     */
  int reverse_time;  /* 1: t = horizon - tau                                            */
  int grid[BQ_MAX_MODES]; /* coefficient truncation M per mode; 0 = the Fock truncation */
  double horizon;    /* T, physical end time                                            */
  double dt;         /* time step the state will be stepped with (stability check)      */
  int ic_mode;       /* BQ_IC_MONOMIAL | BQ_IC_SVD (mapped method; prod M <= 1024 for SVD) */
  int pad;
} bq_map_opts;

/* ---- problem construction (host only; Eqs. 1-3, S1-S2) ---------------------------- */

/* New problem with n_modes (1..BQ_MAX_MODES) modes, Fock truncation fock_trunc[j] >= 1. */
int bq_problem_create(bq_problem** out, int n_modes, const int* fock_trunc);
void bq_problem_destroy(bq_problem* p);

/* Adds a drive envelope (kinds above); *ch_out receives its index. */
int bq_problem_add_channel(bq_problem* p, int kind, const double* params, int n_params, int* ch_out);

/* Adds h * [param] * [channel(t) or conj(channel(t))] * prod (a^dag)^u a^v to H (Eq. 1).
 * channel = -1: static.  param = -1: no parameter, else the coefficient is multiplied by
 * the real parameter params[param] (bq_problem_set_params).  The caller adds Hermitian
 * conjugate terms explicitly; bq_map() rejects a non-Hermitian H with BQ_EINVAL. */
int bq_problem_add_h_term(bq_problem* p, double re, double im, const int* u, const int* v,
                          int channel, int conj, int param);

/* Sets the real parameter values referenced by H terms. */
int bq_problem_set_params(bq_problem* p, const double* values, int n);

/* Adds a Lindblad channel with rate kappa >= 0 and jump operator
 * L = sum_t (c_re[t] + i c_im[t]) prod (a^dag)^u[t] a^v[t]; u, v are n_terms x n_modes,
 * row-major (Eq. 3). */
int bq_problem_add_jump(bq_problem* p, double kappa, int n_terms, const double* c_re,
                        const double* c_im, const int* u, const int* v);

/* Adds the secular ("proper") dissipator of Eq. 203 / Eq. S9 to mode `mode`: rate kappa >= 0
 * and, for n = 0..n_nbar-1, the thermal occupation nbar[n] >= 0 of the bath at the n <-> n+1
 * transition frequency (Eq. S10; n >= n_nbar: 0; n_nbar = 0 is zero temperature).  In the
 * mapped representation it is a separable decay plus the projector term P of Eq. 302c /
 * Eq. S15, which acts only where the x and y indices of the mode agree (every stage,
 * persistent-solve and adjoint kernel restricts it there).  BQ_EINVAL for a bad mode, rate
 * or occupation. */
int bq_problem_add_secular(bq_problem* p, int mode, double kappa, int n_nbar, const double* nbar);

/* Measured operator A(0) by number-basis elements <k|A|l> = re + i im; k, l are n x n_modes
 * row-major.  Repeated (k, l) pairs add up. */
int bq_problem_set_measured(bq_problem* p, int n, const int* k, const int* l, const double* re,
                            const double* im);

/* Initial density matrix rho0 by elements <k|rho0|l> (default: vacuum |0><0|); used by
 * bq_evaluate for Tr(rho0 A(t)). */
int bq_problem_set_rho0(bq_problem* p, int n, const int* k, const int* l, const double* re,
                        const double* im);

/* ---- mapping (Eqs. 6, 10-13, 304) ---------------------------------------------------- */

/* Device bytes bq_map() needs for B problems mapped with the same options. */
int bq_required_bytes(const bq_problem* const* probs, int B, const bq_map_opts* opts, size_t* out);

/* Host-only view of the plan bq_map() would build (no device needed; no counterpart in the
 * paper: the work decomposition of the stage kernels).  n_work: CTAs of one stage launch of
 * the tiled kernel at the default schedule (single-mode states: one item per system, used by
 * the adjoint); work_cap: capacity of the work-item segment (the shortest tile); lanes: the
 * default lanes per point; smem_bytes / adj_smem_bytes: dynamic shared memory per CTA of the
 * tiled forward and adjoint stage kernels; stage_variant as bq_stage_variant. */
typedef struct bq_plan_info {
  int n_systems;
  int n_work;
  int work_cap;
  int lanes;
  int stage_variant;
  int smem_bytes;
  int adj_smem_bytes;
  int pad;
  int64_t total_elems;
} bq_plan_info;
int bq_plan(const bq_problem* const* probs, int B, const bq_map_opts* opts, bq_plan_info* out);

/* Maps B problems into one batched state inside [device_pool, device_pool + pool_bytes)
 * (256-byte aligned, caller-owned).  For the mapped method every non-negligible
 * g_{p,q}(0) = <p|A|q>/sqrt(p! q!) (Eq. 6 with Eq. 8's basis) becomes one separable
 * initial condition G_x = x^p, G_y = y^q, R = 0 with separation constant C (Eq. 304);
 * for the direct method the state is A(0) itself.  Returns BQ_EUNSTABLE_DT if
 * opts->dt exceeds the RK4 bound 2 sqrt(2) / rho, rho a Gershgorin bound of the generator. */
int bq_map(const bq_problem* const* probs, int B, const bq_map_opts* opts, void* device_pool,
           size_t pool_bytes, void* stream, bq_state** out);

/* ---- stepping (Eqs. 9a-c / 303a-c, classical RK4) ----------------------------------- */

/* Advances every system of the state by n_steps RK4 steps of size dt (the mapped value
 * of dt must not exceed the bound checked at bq_map).  Fused stage kernels: on the
 * pipelined single-mode path the four stages of a step run in one launch (bq_tune
 * pipe_fused), otherwise one launch per stage; replayed from a CUDA graph; asynchronous on
 * stream. */
int bq_step(bq_state* s, double dt, int64_t n_steps, void* stream);

/* Batched persistent solve (one launch for all steps of all systems of the batch; the
 * paper's independent initial conditions, main text after Eq. 13, processed as a work
 * queue): every CTA takes systems from an atomic queue, largest first, and keeps the
 * system on chip for all n_steps steps (the RK4 stage buffers, stage sums and compensation
 * in shared memory, the state in registers).  The same arithmetic as bq_step (classical
 * RK4, compensated state update) up to rounding order.  Where bq_autotune measured stepping
 * faster (bq_tune solve_kernel = BQ_SOLVE_STEP), bq_solve runs bq_step instead.  Applies to single-mode
 * states whose systems hold at most 1792 points (M <= 41 with the separable part) and at
 * most two stencil terms per side; other states are stepped with bq_step.  Asynchronous. */
int bq_solve(bq_state* s, double dt, int64_t n_steps, void* stream);

/* Which fused stage kernel bq_step launches for this state: 0 = generic (1-4 modes, tiles
 * with halo windows), 1 = single-mode one-CTA-per-system, 2 = single-mode pipelined
 * (persistent CTAs with 1-D bulk-copy prefetch of the next systems).  Diagnostic only. */
int bq_stage_variant(const bq_state* s, int* variant);

/* *eligible = 1 if bq_solve runs the persistent kernel for this state, 0 if it falls back. */
int bq_solve_eligible(const bq_state* s, int* eligible);

/* ---- schedule selection (autotuner) -------------------------------------------------- *
 * The paper leaves the parallel schedule open (independent initial conditions processed
 * "in an ideal fashion", main text after Eq. 13).  A state carries a schedule for bq_step
 * and one for bq_solve; bq_map picks defaults from occupancy, bq_autotune measures the
 * candidates on the state itself and keeps the fastest.  Changing a schedule never changes
 * the arithmetic: every candidate computes the same RK4 step in the same order per point. */
#define BQ_PATH_TILED 0    /* generic kernel, tiles of R with halo windows (any mode count) */
#define BQ_PATH_SYSTEM 1   /* single mode, one CTA per system */
#define BQ_PATH_PIPE 2     /* single mode, persistent CTAs with bulk-copy prefetch */
#define BQ_SOLVE_STEP (-1)  /* bq_solve steps with bq_step's schedule (where bq_autotune measured it
                             * faster than the persistent kernels, or no persistent kernel fits) */
#define BQ_SOLVE_PROGRAM 0 /* persistent solve, per-term stencil programs */
#define BQ_SOLVE_MERGED 1  /* persistent solve, merged per-row / per-column coefficients */

typedef struct bq_tune {
  int stage_path;        /* BQ_PATH_* used by bq_step */
  int pipe_slots;        /* BQ_PATH_PIPE: shared-memory slots per CTA (2..4) */
  int pipe_ctas_per_sm;  /* BQ_PATH_PIPE: resident CTAs per SM (0 = occupancy limit) */
  int solve_kernel;      /* BQ_SOLVE_* used by bq_solve (BQ_SOLVE_STEP: bq_solve runs bq_step) */
  int solve_ctas_per_sm; /* persistent solve: resident CTAs per SM (0 = occupancy limit) */
  int n_candidates;      /* bq_autotune: schedules measured */
  double step_us;        /* bq_autotune: device time of one RK4 step with bq_step's schedule */
  double solve_us;       /* bq_autotune: device time per RK4 step with bq_solve's schedule */
  int tile;              /* BQ_PATH_TILED: points per tile of a split system (0 = enough tiles
                          * for two CTAs per SM; >= 32); also the adjoint's tiles */
  int lanes;             /* lanes per point of the tiled stage kernel and of the adjoint stage
                          * kernel: 1, 2 or 4 (the terms of a point are split across them);
                          * 0 in bq_set_tune = by the state's size */
  int gread;             /* BQ_PATH_TILED: 1 = split tiles read R (and the adjoint its cotangent)
                          * from global memory instead of staging halo windows in shared
                          * memory; 0 = only where a halo does not fit */
  int grad_coop;         /* bq_grad on the tiled path: 1 = one cooperative launch per checkpoint
                          * segment and direction (all stages of the segment, separated by
                          * grid barriers whose waits are bounded), 0 = one launch per stage;
                          * ignored where the device has no cooperative launch */
  double grad_us;        /* bq_autotune_grad: device time of the trial gradient per RK4 step */
  int pipe_fused;        /* BQ_PATH_PIPE: 1 = the four stages of a step in one launch (every CTA
                          * runs its own systems' stages in order; no CTA waits for another),
                          * 0 = one launch per RK4 stage.  The arithmetic is the same. */
  int pad;
} bq_tune;

/* Current schedules of the state (step_us / solve_us: last bq_autotune result, else 0). */
int bq_get_tune(const bq_state* s, bq_tune* out);

/* Sets the schedules.  BQ_EUNSUPPORTED if a path or kernel is not available for this state
 * (BQ_PATH_PIPE / BQ_PATH_SYSTEM need a single-mode state; BQ_SOLVE_MERGED needs every
 * stencil shift in {-1, 0, 1}; pipe_slots and tiles must fit in shared memory).  A new tile
 * length rewrites the state's work items with a synchronous copy: call it while no step of
 * the state is in flight. */
int bq_set_tune(bq_state* s, const bq_tune* t);

/* Device bytes of the scratch buffer bq_autotune needs: a copy of the state and its
 * rounding compensation (2 x bq_state_bytes). */
int bq_autotune_scratch_bytes(const bq_state* s, size_t* out);

/* Measures every available schedule on the state itself: for bq_step the available paths x
 * slot counts x CTAs per SM (pipelined) or tile lengths (tiled), for bq_solve the available kernels x CTAs per SM, each over
 * trial_steps RK4 steps of size dt after one warm-up step (CUDA events on stream), and sets
 * the fastest.  The state, its compensation and its time are saved into the caller-owned
 * device buffer scratch (scratch_bytes >= bq_autotune_scratch_bytes) first and restored
 * after every trial, so the state is unchanged on return.  Synchronises stream.  out (may
 * be NULL) receives the chosen schedules and their times. */
int bq_autotune(bq_state* s, double dt, int trial_steps, void* scratch, size_t scratch_bytes, void* stream,
                bq_tune* out);

/* ---- gradients (discrete adjoint of the RK4 solve) ----------------------------------- */

/* Number of gradient slots of the state: for every problem b in order, its parameters
 * theta_0..theta_{P_b-1} (bq_problem_set_params), then (Re, Im) of every segment of every
 * piecewise-constant channel of b, channels in order. */
int bq_grad_size(const bq_state* s, int* n);

/* Device bytes of the gradient workspace for n_steps steps checkpointed every
 * checkpoint_every steps: ceil(n/k) checkpoints of the state and 2 x 4 k recorded stage
 * inputs (two segments), plus four cotangent arrays. */
int bq_grad_required_bytes(const bq_state* s, int64_t n_steps, int checkpoint_every, size_t* out);

/* Bytes of one segment's recorded stage inputs (4 checkpoint_every states) and the number of
 * segments.  A workspace larger than bq_grad_required_bytes holds
 * 2 + (work_bytes - required) / per_segment recordings: on the cooperative path (bq_tune
 * grad_coop) bq_grad records that many segments, the last ones, in its forward pass and does
 * not recompute them; with n_segments - 2 extra recordings nothing is recomputed. */
int bq_grad_record_bytes(const bq_state* s, int64_t n_steps, int checkpoint_every, size_t* per_segment,
                         int64_t* n_segments);

/* Loss l_b = Re Tr(rho0_b A_b(tau0 + n_steps dt)) of every problem (loss_out[B]) and the
 * gradient of sum_b l_b (grad_out[bq_grad_size]) with respect to every H parameter and every
 * piecewise-constant segment value, by the exact discrete adjoint of the RK4 solve: a forward
 * pass storing the state every checkpoint_every steps, then, segment by segment in reverse, a
 * recomputation recording the RK4 stage inputs and four adjoint stages per step (transposed
 * stencils, transposed separable source, per-term gradient reductions).  With grad_coop
 * (bq_tune; the default where the device allows cooperative launches) each segment's forward
 * and adjoint stages run in one cooperative launch each on `stream`, and segments recorded in
 * the forward pass (see bq_grad_record_bytes) are not recomputed; otherwise one launch per
 * stage, the recomputation of a segment on an internal stream concurrent with the adjoint of
 * the following segment on another, both ordered after the work already on `stream`.  A grid
 * barrier that waits longer than about 2 s sets the error word: BQ_ETIMEOUT.  The
 * separation constant's dependence on the parameters (Eq. 304) is included.  The state is left
 * as it was (content and tau).  work: caller-owned device buffer, 256-byte aligned.
 * Synchronises stream. */
int bq_grad(bq_state* s, double dt, int64_t n_steps, int checkpoint_every, void* work, size_t work_bytes,
            double* loss_out, double* grad_out, void* stream);

/* Schedules for bq_grad chosen by measuring bq_grad itself (no counterpart in the paper: the
 * adjoint kernels' schedule): every available tiled schedule (tile length x lanes per point x
 * global-read tiles; lanes only for single-mode states) runs one gradient of trial_steps
 * steps of size dt checkpointed every checkpoint_every steps (after one warm-up gradient),
 * timed with CUDA events on stream, and the fastest is set.  The stepping path, pipelined and
 * persistent-solve schedules are kept.  work: as for bq_grad with (trial_steps,
 * checkpoint_every).  The state is unchanged on return (bq_grad leaves it as it was).
 * Synchronises stream.  out (may be NULL) receives the schedules and grad_us. */
int bq_autotune_grad(bq_state* s, double dt, int trial_steps, int checkpoint_every, void* work, size_t work_bytes,
                     void* stream, bq_tune* out);

/* bq_step without any memory allocation, for callers that cannot allocate device memory:
 * code whose device memory is all owned by another component's allocator (a framework that
 * reserves the GPU at start-up and hands out no raw cudaMalloc), embedded callers whose memory
 * budget is fixed at start-up, or loops that must not pay an allocation's latency or risk its
 * failure.  The paper has no counterpart: it is an alternative scratch placement of bq_step.
 *
 * The two RK4 stage buffers and the stage-sum buffer are taken from a fixed device array
 * compiled into this library (three buffers of 4 MiB each, i.e. states of up to 262 144
 * complex FP64 or 524 288 complex FP32 elements; larger states get BQ_EUNSUPPORTED and should
 * use bq_step).  Every GPU that loads the library holds that array until the process
 * exits.  The state's own scratch regions in its pool are not touched; its state arrays are
 * updated exactly as bq_step updates them (same kernels, same arithmetic).  Plain kernel
 * launches on stream (4 per step) after clearing the used part of the three buffers; no
 * allocation, no cudaFree, no allocating library routine.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 *     once per device, with that device current); make that first call before any stream
 *     capture is begun on the calling thread.
 *   - All calls share the one array, and it keeps the last call's contents.  Every element a
 *     stage reads was written earlier in the same step, except the padding between a system's
 *     arrays, which is read at the edges of a system with zero coefficients and never written;
 *     each call therefore clears the part of the three buffers its state uses (a memset on
 *     stream) before its first stage, so that stale values of another state or precision
 *     cannot enter as non-finite numbers.  Calls whose work overlaps on the GPU (different
 *     streams, or other threads) race on the array: serialise them.
 * Results equal bq_step's (same kernels; the stage buffers' placement does not enter the
 * arithmetic). */
int bq_step_fixed_scratch(bq_state* s, double dt, int64_t n_steps, void* stream);

/* Current integration time tau of the state (host copy, no synchronisation). */
int bq_time(const bq_state* s, double* tau);

/* ---- evaluation (Eqs. 7, 11) --------------------------------------------------------- */

/* out_host[2b], out_host[2b+1] = Re, Im of Tr(rho0_b A_b(tau)) for every problem b
 * (warp reductions over initial conditions and rho0's support).  Synchronises stream. */
int bq_evaluate(bq_state* s, double* out_host, void* stream);

/* The same values without synchronising: the computation and the copy into out are
 * enqueued on stream, and out holds them once the stream has reached that point.  out is
 * device memory or pinned host memory (2 * B doubles, owned by the caller; pageable host
 * memory also works but makes the copy synchronous for the host, as cudaMemcpyAsync does).
 * Neither the device error word nor finiteness is checked here: bq_evaluate, or any later
 * synchronising call, reports a bounded wait that gave up. */
int bq_evaluate_async(bq_state* s, double* out, void* stream);

/* Number-basis block <k|A_b(tau)|l> for every mode index < lo (the paper's epsilon_r
 * block uses lo = 3).  out_host holds B * D * D complex values (re, im interleaved),
 * D = prod_j min(lo, grid_j), row-major (k, l).  Synchronises stream. */
int bq_fock_block(bq_state* s, int lo, double* out_host, void* stream);

/* Shape of the state for bq_read_state: number of systems (initial conditions) in
 * total, and per system the element counts of G_x, G_y and R (0 if absent). */
int bq_state_info(const bq_state* s, int* n_systems, int64_t* total_elems);
int bq_system_info(const bq_state* s, int sys, int* problem, int* p_idx, int* q_idx,
                   int64_t* n_gx, int64_t* n_gy, int64_t* n_r, double* weight_re_im,
                   double* c_re_im);

/* Copies system sys's G_x, G_y, R (or A for the direct method, in R) to host as
 * complex FP64, converted to the monomial basis g_{k,l} of Eq. 6 (number-basis values
 * A_{k,l} for the direct method).  Buffers may be NULL to skip.  Synchronises stream. */
int bq_read_system(bq_state* s, int sys, double* gx, double* gy, double* r, void* stream);

/* Raw state snapshot (checkpoint / resume, host-resident inputs): the G_x, G_y, R arrays
 * of every system in storage layout, *nbytes = total_elems * complex element size.
 * bq_store_state copies device -> host, bq_load_state host -> device and clears the
 * state's rounding compensation (the integration time tau is part of neither;
 * bq_set_time sets it).  Host buffers may be pageable or
 * pinned; both calls are asynchronous on stream for pinned memory. */
int bq_state_bytes(const bq_state* s, size_t* nbytes);
int bq_store_state(bq_state* s, void* host, void* stream);
int bq_load_state(bq_state* s, const void* host, void* stream);
int bq_set_time(bq_state* s, double tau);

void bq_state_destroy(bq_state* s);

/* ---- diagnostics ---------------------------------------------------------------------- */
const char* bq_status_string(int status);
const char* bq_last_error(void);

/* Number of kernel launches this library has enqueued since load (graph replays count
 * every kernel node). */
int64_t bq_launch_count(void);

/* Measured arithmetic roof of the current GPU (no counterpart in the paper: the denominator
 * of the roofline fraction of kernels bound by FP64 or FP32 arithmetic instead of HBM).
 * Runs 16 independent dependent FMA chains per thread, 8 x iters FMAs each, on 4 CTAs of
 * 256 threads per SM after a one-iteration warm-up launch, timed with CUDA events on stream
 * at the GPU's current clocks (none is set).  dtype: BQ_F64 or BQ_F32.  *fma_per_s receives
 * thread-level FMA instructions per second (FLOP/s = 2 x).  BQ_EINVAL for a bad dtype,
 * iters < 1 or a NULL output; BQ_ECUDA if a launch fails.  Synchronises stream. */
int bq_fma_peak(int dtype, int64_t iters, double* fma_per_s, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* BQ_H_ */
