/*
 * dpf.h -- C ABI of the GB300 (sm_103a) Differentiable Power-Flow hot path.
 *
 * Differentiable Power-Flow (DPF) solves the AC power-flow problem of
 * Sec. 2.1 (Eq. powerbalance, Eq. pf_equation_full) by gradient descent on
 * the squared power mismatch (Eq. pf_optimization_problem, Sec. 4, Alg. 1):
 * each iteration forms S_calc = V (Y_bus V)^*, the mismatch
 * f = [dP(pv,pq), dQ(pq)], the loss L = (1/m)||f||^2 with m = |pv| + 2|pq|,
 * its gradient with respect to theta(pv,pq) and |V|(pq), and an Adam step
 * with a learning-rate scheduler.  This library runs that iteration for many
 * cases at once on one GPU, sharing one Y_bus (Sec. 4.2 batching; N-1 cases
 * as a per-case correction of the shared matrix).
 *
 * Conventions
 *   - All functions return an int status: DPF_OK (0) or a negative DPF_E_*.
 *     Nothing aborts or throws across the ABI; dpf_last_error() returns a
 *     human-readable message for the most recent failure on the calling
 *     thread.
 *   - Units: per unit (p.u.) and radians.  Injections are net
 *     (generation - load).
 *   - Layouts: per-case arrays are case-major, [n_case][n_bus] row-major
 *     (case k, bus i at k*n_bus + i).  Branch arrays are [n_branch].
 *   - Ownership: every pointer argument stays owned by the caller and is
 *     read or written only during the call (or, for device pointers, by work
 *     enqueued on `stream` by the call).  Handles (dpf_ybus, dpf_workspace)
 *     are owned by the library and released with their *_free function.
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *     default stream).  Work is enqueued on it; functions that return host
 *     values synchronise that stream (stated per function).
 *   - Device pointers must be 8-byte aligned (16 for double2-viewed data is
 *     not required: complex values are passed as separate re/im arrays).
 */
#ifndef DPF_H
#define DPF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
enum {
  DPF_OK = 0,
  DPF_E_INVALID = -1,     /* bad argument: NULL, size, index or bus type    */
  DPF_E_ISLANDED = -2,    /* an outage disconnects the grid                 */
  DPF_E_CUDA = -3,        /* a CUDA runtime call failed (message has detail) */
  DPF_E_OOM = -4,         /* device or host allocation failed               */
  DPF_E_UNSUPPORTED = -5, /* e.g. a phase-shifting transformer              */
  DPF_E_STATE = -6        /* call out of order (e.g. iterate before begin)  */
};

/* per-case outcome written to dpf_batch.status */
enum {
  DPF_CASE_CONVERGED = 0, /* FP64 max |f| <= tol                             */
  DPF_CASE_MAX_ITER = 1,  /* iteration budget spent above tol                */
  DPF_CASE_DIVERGED = 2   /* loss became NaN/Inf                             */
};

enum { DPF_PQ = 0, DPF_PV = 1, DPF_SLACK = 2 };            /* bus types (Sec. 2.1) */
/* iteration precision: DPF_FP32 -- FP32 iterations on an FP64-accurate
 * (double-float) master with the FP64 convergence test; DPF_FP64 -- FP64
 * throughout; DPF_MIXED (solves only) -- the forward pass (currents, S, the
 * mismatch and its weights) in FP64 over FP64 voltages, the adjoint and the
 * optimiser in FP32 on the double-float master: it resolves mismatches below
 * the FP32 current's error of a few |Y_ii| 2^-24 (~1e-5 p.u. with short
 * lines) at about the FP32 cost of the adjoint.
 * DPF_FP32R (solves only) -- refined FP32 iterations: every arithmetic step
 * of an iteration is FP32 as in DPF_FP32, but the forward pass evaluates the
 * mismatch as a correction to the FP64 residual of the case's most recent
 * convergence test, f = f_ref + dV conj(I_ref) + V conj(Y dV), where dV (the
 * change of V since that test, carried in FP32 and advanced from each
 * optimiser step) is small near convergence; the FP32 rounding error then
 * scales with dV instead of with |Y_ii| |V|, and the iterations reach
 * mismatches far below DPF_FP32's limit.  The FP64 test (every check_every
 * iterations, on the cases the gate admits, and on every active case at
 * the test of every refresh_every-th step, 100 by default -- or at every
 * test if check_every is larger) renews f_ref, I_ref and V_ref.  Until a case's first test its iterations
 * equal DPF_FP32 ones. */
enum { DPF_FP32 = 0, DPF_FP64 = 1, DPF_MIXED = 2, DPF_FP32R = 3 };
enum { DPF_SCHED_CONST = 0, DPF_SCHED_PLATEAU = 1, DPF_SCHED_STEP = 2 };
enum { DPF_OPT_ADAM = 0, DPF_OPT_SGD = 1, DPF_OPT_RMSPROP = 2 };    /* Sec. 5.3's optimisers */

/* ---- grid description (host arrays, caller-owned, read-only) -------------
 * The problem statement of Sec. 2.1 / Alg. 1 inputs: bus types with exactly
 * one slack per connected island (a block-diagonal batch of grids, Sec. 4.2,
 * is one grid with one island per member), specified P (pv, pq), Q (pq),
 * |V| (pv, slack), the slack angle (the same for every island),
 * and the branch table from which Y_bus is built with the pi-model (the
 * MATPOWER model the paper's Eq. powerbalance footnote refers to):
 *   y_s = 1/(r + jx); Y_ff += (y_s + j b_ch/2)/tap^2; Y_tt += y_s + j b_ch/2;
 *   Y_ft += -y_s/tap; Y_tf += -y_s/tap.
 * tap = 0 is read as 1 (no transformer).  shift may be NULL; a nonzero shift
 * is rejected with DPF_E_UNSUPPORTED.  Parallel branches are rejected with
 * DPF_E_UNSUPPORTED (each CSR off-diagonal entry maps to one branch). */
typedef struct {
  int32_t n_bus, n_branch;
  const uint8_t* bus_type;   /* [n_bus] DPF_PQ / DPF_PV / DPF_SLACK            */
  const double* p_spec;      /* [n_bus] net active injection                   */
  const double* q_spec;      /* [n_bus] net reactive injection (used at PQ)    */
  const double* vm_set;      /* [n_bus] |V| set-point (used at PV and slack)   */
  double va_slack;           /* slack angle                                    */
  const int32_t* f_bus;      /* [n_branch] 0-based from-bus (tap side)         */
  const int32_t* t_bus;      /* [n_branch] 0-based to-bus                      */
  const double *r, *x, *b_ch, *tap;  /* [n_branch]                              */
  const double* shift;       /* [n_branch] or NULL; must be 0                  */
} dpf_grid;

typedef struct dpf_ybus dpf_ybus;           /* Y_bus in CSR (host + device)   */
typedef struct dpf_workspace dpf_workspace; /* device state of one batch      */

/* Build Y_bus on the host (CSR, FP64, sorted columns, every diagonal
 * present) and validate the grid.  No CUDA call is made; a GPU is not needed.
 * Errors: DPF_E_INVALID (sizes, indices, an island without exactly one slack, f == t,
 * non-finite or zero impedance), DPF_E_UNSUPPORTED (shift, parallel branch). */
int dpf_build_ybus_host(const dpf_grid* g, dpf_ybus** out);

/* Copy a host-built Y_bus to the current device (FP32 and FP64 values, CSR
 * indices, branch data), enqueued on `stream`, which is then synchronised. */
int dpf_ybus_upload(dpf_ybus* y, void* stream);

/* dpf_build_ybus_host followed by dpf_ybus_upload. */
int dpf_build_ybus(const dpf_grid* g, void* stream, dpf_ybus** out);
int dpf_ybus_free(dpf_ybus* y);

/* Sizes of a built Y_bus (host values). */
int dpf_ybus_info(const dpf_ybus* y, int32_t* n_bus, int32_t* n_branch, int32_t* nnz);

/* Host copies of the FP64 CSR: row_ptr [n_bus+1], col [nnz], val_re/val_im
 * [nnz].  Any output may be NULL.  No CUDA call. */
int dpf_ybus_export(const dpf_ybus* y, int32_t* row_ptr, int32_t* col,
                    double* val_re, double* val_im);

/* bridge[l] = 1 if removing branch l disconnects the grid (Tarjan low-link on
 * the host).  N-1 outages of bridges are rejected with DPF_E_ISLANDED.
 * No CUDA call. */
int dpf_ybus_bridges(const dpf_ybus* y, uint8_t* bridge);

/* ---- batched solve ---------------------------------------------------------
 * One case = one power-flow problem on the shared grid, possibly with its own
 * injections / set-points (time series) and one branch outage (N-1).
 * All pointers are device pointers unless host_io = 1, in which case they are
 * host pointers (pinned memory gives the best transfer rate) and the library
 * copies them through its workspace inside the call, on `stream`. */
typedef struct {
  int32_t n_case;
  int32_t host_io;           /* 0: device pointers; 1: host pointers          */
  const double* p_spec;      /* [n_case][n_bus] or NULL = the grid's; p_spec  */
  const double* q_spec;      /* and q_spec are given together or not at all   */
  const double* vm_set;      /* [n_case][n_bus] or NULL = the grid's          */
  const int32_t* outage;     /* [n_case] branch index or -1, NULL = none      */
  double* va;                /* [n_case][n_bus] in: warm start (if flat_start
                                = 0); out: solution angles                   */
  double* vm;                /* [n_case][n_bus] in/out: magnitudes            */
  int32_t* iters;            /* [n_case] out: optimizer steps taken           */
  int32_t* status;           /* [n_case] out: DPF_CASE_*                      */
  double* max_mismatch;      /* [n_case] out: FP64 max |f| of the returned V  */
  double* loss;              /* [n_case] out: FP64 loss of the returned V     */
  const double* va_start;    /* [n_bus] or NULL: one warm start shared by    */
  const double* vm_start;    /* every case (given together; with flat_start =
                                0 they replace va/vm as the start, and va/vm
                                are outputs only) -- e.g. the base-case state
                                from which the cases of an N-1 batch start.
                                dpf_solve_* only (dpf_nr_solve: NULL)        */
} dpf_batch;

/* Iteration options.  Defaults (dpf_default_opts): Table 2 of the paper --
 * Adam betas (0.979, 0.963), eps 1e-8, ReduceLROnPlateau factor 0.547,
 * patience 41, threshold 0.0673 (relative), cooldown 97, max_iter 1000 --
 * with lr 1e-2, tol 1e-6 p.u., check_every 25, gate 1e-3, FP32 iterations. */
typedef struct {
  double lr, beta1, beta2, eps;   /* Adam (eps also RMSprop's)                 */
  int32_t optimizer;         /* DPF_OPT_* (PyTorch semantics: SGD without
                                dampening/Nesterov, RMSprop not centred)      */
  double momentum;           /* SGD momentum (0 = plain SGD)                   */
  double alpha;              /* RMSprop smoothing constant                     */
  int32_t sched;             /* DPF_SCHED_*                                    */
  double factor, threshold, min_lr;
  int32_t patience, cooldown;
  int32_t step_size;         /* StepLR                                         */
  double gamma;
  int32_t max_iter;          /* optimizer steps per case                       */
  int32_t check_every;       /* FP64 convergence test every k steps (>= 1)     */
  double tol;                /* stop when FP64 max |f| <= tol                  */
  double gate;               /* FP32 mode: the FP64 test examines only cases
                                whose FP32 max |f| from the latest forward pass
                                is <= gate (0 = every case).  It only skips
                                tests that cannot pass; a case is marked
                                converged by the FP64 test alone.             */
  int32_t flat_start;        /* 1: ignore va/vm inputs, start flat             */
  int32_t precision;         /* DPF_FP32 / DPF_FP64 / DPF_MIXED (see above)    */
  int32_t lanes;             /* cases per row group 1..32 (power of 2); 0=auto */
  int32_t warps;             /* warps per CTA (1..8); 0 = auto                 */
  int32_t row_blocks;        /* CTAs along the bus dimension; 0 = auto         */
  int32_t use_graph;         /* 1: replay iterations from a CUDA graph         */
  int32_t pair_cases;        /* FP32 batches of >= 64 cases at 32 lanes: bit 0
                                runs the forward pass, bit 1 the adjoint pass
                                with two cases per thread (16-byte accesses);
                                0: one case per thread                        */
  int32_t pdl;               /* 1: iteration kernels use programmatic dependent
                                launch (each may start while its predecessor
                                drains; it waits for it before touching the
                                state)                                         */
  int32_t stage_v;           /* 1: the forward pass first copies the rows of V
                                its row block references into shared memory
                                and gathers from there (lanes = 32 only)      */
  int32_t plain;             /* 1: the plain form of Alg. 1 -- one case at a
                                time, separate launches per iteration and a
                                host stop test (FP64 check + device-to-host
                                read) after every iteration; check_every is
                                taken as 1.  Used as the unbatched baseline. */
  int32_t dc_start;          /* 1 with flat_start: the angles start from the
                                DC approximation (dpf_dc_solve to dc_tol),
                                |V| from the flat start.
                                1 with a warm start (va/vm or va_start/
                                vm_start) and outages: a case whose branch
                                l = (f, t) is out starts from its start
                                angles plus the DC angle change of the
                                outage: dtheta solves B' dtheta =
                                b_l (theta_f - theta_t) (e_f - e_t), with B'
                                the DC matrix without l, b_l = 1/(x_l tau_l)
                                and theta the case's start angles -- the
                                branch's pre-outage DC flow put back at its
                                ends -- and dtheta = 0 at slack buses;
                                |V| as started.  Cases without an outage
                                keep their start.                           */
  int32_t stage_y;           /* single-case FP32 / FP32R solves (lanes = 1):
                                0 -- the passes read their Y_bus rows from
                                global memory, one wave of CTAs each owning
                                many rows (no reuse to stage for when every
                                entry serves one case); 1 -- stage each row
                                block's rows in shared memory like batches */
  double dc_tol;             /* dc_start: relative residual at which a case's
                                conjugate-gradient DC solve stops (> 0;
                                default 1e-10; >= 1e-5 runs it on FP32
                                vectors, as dpf_dc_solve)                   */
  int32_t dc_max_iter;       /* dc_start: CG iterations at most (>= 1; default
                                10000); a case still above dc_tol then
                                starts from its last CG iterate             */
  int32_t refresh_every;     /* DPF_FP32R with a gate: every active case is
                                tested, and its references renewed, when its
                                step count is a multiple of this (rounded
                                down to a multiple of check_every, at least
                                check_every); 0 = 100 (default).  The
                                refined mismatch's rounding grows with |dV|,
                                the distance moved since the last renewal. */
} dpf_solve_opts;

void dpf_default_opts(dpf_solve_opts* o);

/* Workspace: device buffers for up to `max_case` cases of one Y_bus.  All
 * device memory the solve needs is allocated here (and grown on demand by
 * dpf_solve_begin); nothing is allocated per iteration. */
int dpf_workspace_create(const dpf_ybus* y, int32_t max_case, dpf_workspace** out);
int dpf_workspace_free(dpf_workspace* ws);

/* Full solve (Alg. 1 for every case): dpf_solve_begin, iterations until every
 * case has converged, diverged or spent max_iter, dpf_solve_end.  Polls the
 * active-case count from the host every few check intervals (synchronises
 * `stream` at those points and at the end).  ws may be NULL (a temporary
 * workspace is created and freed inside the call). */
int dpf_solve_batch(const dpf_ybus* y, dpf_workspace* ws, const dpf_batch* b,
                    const dpf_solve_opts* o, void* stream);

/* Step-wise driving of the same solve.  begin: validate, copy inputs, set the
 * initial state (flat or warm start; fixed |V| and slack angle enforced),
 * compute the N-1 corrections.  iterate: n_iter DPF iterations of every
 * active case -- FP64 test (when due), forward SpMV + mismatch + loss, adjoint
 * SpMV + gradient + Adam, scheduler -- with no host synchronisation.  end:
 * final FP64 evaluation, statuses and solution written to the batch outputs
 * (synchronises `stream` when host_io = 1). */
int dpf_solve_begin(const dpf_ybus* y, dpf_workspace* ws, const dpf_batch* b,
                    const dpf_solve_opts* o, void* stream);
int dpf_solve_iterate(dpf_workspace* ws, int32_t n_iter, void* stream);
int dpf_solve_end(dpf_workspace* ws, const dpf_batch* b, void* stream);
/* Autotuner.  Times candidate launch shapes of the solve loop on this batch
 * -- cases per row group (`lanes`, i.e. rows per warp = 32/lanes), warps per
 * CTA, row blocks, the two-cases-per-thread variants and shared-memory V
 * staging -- for `iters`
 * iterations each (plus one warm-up check interval), and writes the fastest
 * into o->lanes, o->warps, o->row_blocks, o->pair_cases and o->stage_v.  The batch's
 * inputs are read (as in dpf_solve_begin) but no output is written; a later
 * dpf_solve_begin starts from scratch.  Results are cached in the workspace
 * per (n_case, precision, grid, outage/injection layout).  Synchronises
 * `stream`. */
int dpf_autotune(const dpf_ybus* y, dpf_workspace* ws, const dpf_batch* b, dpf_solve_opts* o,
                 int32_t iters, void* stream);

/* Number of cases still iterating (synchronises `stream`). */
int dpf_active_count(dpf_workspace* ws, int32_t* n_active, void* stream);
/* Steps taken so far by the batch (host counter, no synchronisation). */
int dpf_iterations_done(const dpf_workspace* ws, int32_t* n_iter);

/* ---- measurement ----------------------------------------------------------
 * dpf_profile_enable(ws, 1): from now on dpf_solve_iterate launches without a
 * CUDA graph and brackets every forward (k_fwd) and adjoint (k_adj) launch
 * with CUDA events on the caller's stream; 0 switches back to graph replay.
 * dpf_kernel_times: summed durations (ms) and launch counts of the
 * bracketed launches since the last enable (synchronises `stream`).
 * dpf_kernel_launches: number of kernels the workspace has enqueued since it
 * was created -- by the solve (begin, iterations, convergence tests, end, the
 * DC start), dpf_power, dpf_loss_backward and identification calls; graph
 * replays count their kernel nodes. */
int dpf_profile_enable(dpf_workspace* ws, int32_t on);
int dpf_kernel_times(dpf_workspace* ws, double* fwd_ms, double* adj_ms, int32_t* n_fwd, int32_t* n_adj,
                     void* stream);
int dpf_kernel_launches(const dpf_workspace* ws, int64_t* n);

/* Read-bandwidth probe (a measurement hook; the paper has no counterpart):
 * a plain kernel reads the caller's device buffer `buf` of `bytes` bytes
 * (16-byte aligned, bytes a multiple of 16) with 16-byte loads that bypass
 * L1 (ld.global.cg), grid = SMs x 8 CTAs of 256 threads; a launch reads the
 * buffer `passes` = min(64, max(1, 256 MB / bytes)) times; two untimed
 * launches, then `reps` launches between CUDA events on `stream`.
 * *gbs = bytes x passes x reps / elapsed time (GB/s).  A buffer far below
 * the L2's 129 MB measures the L2 read bandwidth, one far above it the HBM
 * read bandwidth.  Synchronises `stream`.  Errors: DPF_E_INVALID (NULL,
 * alignment, size, reps < 1), DPF_E_CUDA. */
int dpf_read_bandwidth(const void* buf, int64_t bytes, int32_t reps, double* gbs, void* stream);

/* Grid-barrier probe (a measurement hook; the paper has no counterpart): the
 * cost of one grid-wide barrier in a persistent (cooperative) launch of
 * num_SMs x ctas_per_sm CTAs of 256 threads -- the synchronisation a single
 * persistent kernel would need between the forward and adjoint passes of an
 * iteration.  Times a cooperative launch with `reps` barriers and one with
 * none (CUDA events on `stream`); *us_per_barrier = their difference / reps.
 * Synchronises `stream`.  Errors: DPF_E_INVALID (bad argument, or more CTAs
 * per SM than can be resident), DPF_E_CUDA. */
int dpf_grid_barrier_cost(int32_t ctas_per_sm, int32_t reps, double* us_per_barrier, void* stream);

/* ---- forward evaluation (Eq. powerbalance) --------------------------------
 * The evaluation entry points take (va, vm) verbatim, set-points included.
 * S_calc = V (Y V)^* for n_case voltage vectors (case-major device arrays),
 * optional per-case outage (NULL = none).  precision selects the FP32 or
 * FP64 kernels; outputs are FP64 either way. */
int dpf_power(const dpf_ybus* y, dpf_workspace* ws, int32_t n_case,
              const double* va, const double* vm, const int32_t* outage,
              int32_t precision, double* p_calc, double* q_calc, void* stream);

/* ---- forward evaluation without device allocation ---------------------------
 * No counterpart in the paper: a deployment variant of dpf_power for callers
 * that cannot allocate device memory -- code running inside an application
 * that owns the whole device memory budget through its own pool (a raw
 * cudaMalloc there fails or bypasses the application's accounting) and
 * latency-critical loops that cannot afford the implicit synchronisation of
 * cudaMalloc/cudaFree.  Same result as dpf_power with precision DPF_FP64
 * (va, vm taken verbatim; no outages), but it needs no workspace and calls
 * no allocating routine.  Its scratch is a fixed array inside the library of
 * DPF_NOALLOC_MAX_ELEMS complex values (4 MiB), which every GPU that loads
 * the library holds until the process exits; n_case * n_bus above that limit
 * is rejected with DPF_E_INVALID.  The first call on a device looks up the
 * array's device address (once per device, with that device current); make
 * that first call before any stream capture.  The address is kept for the
 * life of the process: do not use this entry point on a device after a
 * cudaDeviceReset (the reset destroys the context it belongs to).  All calls share the one array,
 * so calls whose work overlaps on the GPU (different streams, or host threads
 * without ordering) race: serialise them, e.g. on one stream.  The scratch
 * is fully rewritten by each call before it is read.  Inputs va, vm
 * [n_case][n_bus] and outputs p_calc, q_calc (either may be NULL) are
 * caller-owned device arrays. */
#define DPF_NOALLOC_MAX_ELEMS (1 << 18)
int dpf_power_noalloc(const dpf_ybus* y, int32_t n_case, const double* va, const double* vm,
                      double* p_calc, double* q_calc, void* stream);

/* ---- loss and its adjoint (Sec. 4.1: dL/dx = J^T F, scaled by the MSE) ----
 * For n_case states (va, vm) and specified injections (p_spec/q_spec, NULL =
 * the grid's; case-major device arrays) computes the FP64 loss per case and,
 * through the hand-written adjoint kernels in `precision`:
 *   d_va, d_vm [n_case][n_bus]  dL/dtheta (0 off pv,pq), dL/d|V| (0 off pq);
 *   d_p, d_q   [n_case][n_bus]  dL/dP_spec, dL/dQ_spec;
 *   d_g, d_b, d_bch [n_branch]  dL/d(series g), dL/d(series b), dL/d(b_ch),
 *                               summed over the cases (parameter
 *                               identification over operating points).
 * g_series / b_series ([n_branch] device, FP64) replace the branches' series
 * admittance g + jb (NULL = as built); charging and taps stay as built.
 * Any output pointer may be NULL to skip it.  outage may be NULL. */
int dpf_loss_backward(const dpf_ybus* y, dpf_workspace* ws, int32_t n_case,
                      const double* va, const double* vm,
                      const double* p_spec, const double* q_spec,
                      const int32_t* outage,
                      const double* g_series, const double* b_series,
                      int32_t precision,
                      double* loss, double* d_va, double* d_vm,
                      double* d_p, double* d_q,
                      double* d_g, double* d_b, double* d_bch, void* stream);

/* ---- DC approximation ------------------------------------------------------
 * The linearised comparison model and optional initialisation (Sec. 2,
 * Alg. 2): angles solving B theta = P over the pv and pq buses, with
 * B = sum_l b_l (e_f - e_t)(e_f - e_t)^T, b_l = 1 / (x_l tau_l) (resistance,
 * charging and |V| ignored), slack angles fixed at the grid's va_slack (one
 * slack per island).  For n_case cases: p_spec [n_case][n_bus] FP64 device
 * (NULL = the grid's), outage [n_case] device (-1 = none; NULL = none; a
 * bridge is DPF_E_ISLANDED) as for dpf_solve_batch.  Conjugate gradients
 * with the Jacobi preconditioner on the GPU, per case until |r| <= tol |r0|
 * or max_iter iterations; the vectors are double-float pairs (~48 bits)
 * for tol < 1e-5 and FP32 for tol >= 1e-5, the per-case scalars FP64.  Outputs (caller-owned device
 * arrays): va [n_case][n_bus] (required), iters [n_case] and rel_residual
 * [n_case] (|r| / |r0| at the stop; either may be NULL).  Uses (and
 * resets) the workspace like the other calls. */
int dpf_dc_solve(const dpf_ybus* y, dpf_workspace* ws, int32_t n_case,
                 const double* p_spec, const int32_t* outage, double tol,
                 int32_t max_iter, double* va, int32_t* iters,
                 double* rel_residual, void* stream);

/* ---- Newton-Raphson (Alg. 2) on the GPU ------------------------------------
 * The ground-truth solver of the paper (Alg. 2) for the same batches as
 * dpf_solve_batch, and the second stage of a hybrid in which Alg. 1 supplies
 * the start (its solution passed as va/vm with flat_start = 0).  Each Newton
 * step solves J_f dx = -f with J_f the Jacobian of Alg. 2 (rows P at pv and
 * pq buses, Q at pq buses; unknowns theta at pv and pq, |V| at pq), written
 * per bus as 2x2 blocks on the pattern of Y_bus (left-out rows and columns
 * become identity rows and columns), factorised by block LU without pivoting
 * outside the 2x2 diagonal blocks in a minimum-degree order found on the host.
 *
 * dpf_nr_create: host analysis of Y_bus (order, filled pattern, elimination
 * tree, update lists) and the device buffers for up to max_case cases (the
 * factor takes n_pos * 32 bytes per case).  y must be uploaded
 * (DPF_E_STATE otherwise) and outlive the handle.  Synchronous.
 * Errors: DPF_E_INVALID, DPF_E_OOM, DPF_E_UNSUPPORTED (update lists above
 * 2^28 block products or factor storage above 2^40 bytes).
 *
 * dpf_nr_solve: every case of the batch (device pointers only: host_io must
 * be 0; p_spec/q_spec/vm_set/outage as for dpf_solve_batch) from the flat
 * start (o->flat_start = 1) or from va/vm (fixed |V| and the slack angle
 * enforced), Newton steps until FP64 max |f| <= o->tol or o->max_iter steps.
 * o->precision: DPF_FP64 factorises and solves in FP64; DPF_FP32 in FP32 (the
 * mismatch, the stop test and the state stay FP64; convergence turns linear
 * at about cond(J) 2^-24 per step near the solution).  Outputs: va, vm
 * (solution), iters (Newton steps), status (DPF_CASE_CONVERGED, _MAX_ITER,
 * or _DIVERGED: a non-finite mismatch or a singular diagonal block),
 * max_mismatch and loss of the returned state (any of the last four may be
 * NULL).  Reads the number of unconverged cases from the device after every
 * step (synchronises `stream`).  Errors: DPF_E_INVALID (sizes, pointers,
 * outage index, options), DPF_E_ISLANDED (an outage of a bridge).
 *
 * dpf_nr_stats: positions of the filled pattern, block products of one
 * factorisation, tree levels, kernels enqueued so far (any output may be NULL).
 * dpf_nr_analyze / dpf_nr_pattern: the host analysis alone, no CUDA call:
 * sizes, and the elimination order (user bus indices, [n_bus]), the filled
 * pattern in that order (row_ptr [n_bus + 1], col [n_pos]) and the tree
 * level of every step ([n_bus]); any array may be NULL. */
typedef struct dpf_nr dpf_nr;
typedef struct {
  int32_t precision;         /* DPF_FP64 or DPF_FP32: the factor and the solves */
  double tol;                /* stop when FP64 max |f| <= tol                   */
  int32_t max_iter;          /* Newton steps per case                           */
  int32_t flat_start;        /* 1: ignore va/vm inputs, start flat              */
  int32_t lanes;             /* cases per CTA of the factor and solve kernels
                                (power of 2 up to 32; 0 = auto)               */
  int32_t fallback;          /* 1 (with flat_start = 0): a case Newton does not
                                converge keeps the start passed in va/vm and
                                reports the start's max |f| and loss (its
                                status still says Newton failed): a DPF
                                solution given as the start is the fallback  */
} dpf_nr_opts;
/* Defaults: DPF_FP64, tol 1e-10, max_iter 20, flat start, lanes auto, no fallback. */
void dpf_nr_default_opts(dpf_nr_opts* o);
int dpf_nr_create(const dpf_ybus* y, int32_t max_case, dpf_nr** out);
int dpf_nr_free(dpf_nr* h);
int dpf_nr_solve(dpf_nr* h, const dpf_batch* b, const dpf_nr_opts* o, void* stream);
int dpf_nr_stats(const dpf_nr* h, int64_t* n_pos, int64_t* n_pairs, int32_t* n_levels, int64_t* launches);
int dpf_nr_analyze(const dpf_ybus* y, int64_t* n_pos, int64_t* n_pairs, int32_t* n_levels);
int dpf_nr_pattern(const dpf_ybus* y, int32_t* order, int32_t* row_ptr, int32_t* col, int32_t* level);

/* ---- parameter identification over measured operating points -------------
 * The gradient of the loss to the branch parameters (Sec. 1 / abstract:
 * gradients to the simulation parameters, which lets them be identified)
 * for an iterative identification loop.
 * dpf_paramid_begin stages n_case measured operating points in the
 * workspace once: va, vm, p_spec, q_spec are [n_case][n_bus] FP64 device
 * arrays (caller-owned; p_spec/q_spec NULL = the grid's); precision as in
 * dpf_loss_backward.  dpf_paramid_step then evaluates, at those points and
 * for the series admittances g_series + j b_series ([n_branch] FP64 device,
 * required; charging and taps as built): the Y values, the forward pass and
 * the branch adjoint -- the same quantities as dpf_loss_backward with these
 * inputs and d_va = d_vm = d_p = d_q = NULL, without restaging the points.
 * d_g, d_b, d_bch [n_branch] (summed over the points) and loss [n_case]
 * (FP64; an extra FP64 pass) are device outputs, each may be NULL.
 * Any other call on the workspace (a solve, an evaluation) discards the
 * staged points: a later step returns DPF_E_STATE.  Errors as elsewhere. */
int dpf_paramid_begin(const dpf_ybus* y, dpf_workspace* ws, int32_t n_case,
                      const double* va, const double* vm,
                      const double* p_spec, const double* q_spec,
                      int32_t precision, void* stream);
int dpf_paramid_step(const dpf_ybus* y, dpf_workspace* ws,
                     const double* g_series, const double* b_series,
                     double* d_g, double* d_b, double* d_bch, double* loss,
                     void* stream);

/* ---- Adam on a parameter vector -------------------------------------------
 * One Adam step (the optimiser of Sec. 5.3, Kingma & Ba with bias correction)
 * on n FP64 parameters, e.g. the branch admittances g, b of parameter
 * identification driven by dpf_loss_backward's d_g, d_b.  All arrays are
 * device [n]: x (updated in place), grad, and the caller-owned moments m, v
 * (zero before step 1).  t is the 1-based step number.  lr_scale (or NULL)
 * gives a per-entry learning-rate factor (step_i = lr * lr_scale[i]), e.g.
 * the parameters' magnitudes for relative steps. */
int dpf_adam_update(int32_t n, double* x, const double* grad, double* m, double* v, const double* lr_scale,
                    int32_t t, double lr, double beta1, double beta2, double eps, void* stream);

/* Message of the most recent failure on this thread ("" if none). */
const char* dpf_last_error(void);
/* Static description of a status code. */
const char* dpf_status_str(int status);

#ifdef __cplusplus
}
#endif
#endif /* DPF_H */
