/*
 * ucn -- GPU-native sequential convex programming with a consensus-ADMM
 * inner solver (arXiv 2603.10711), for NVIDIA GB300 (sm_103a).
 *
 * C ABI.  Every pointer argument is either a HOST pointer (suffix none,
 * only in ucn_problem_desc) or a DEVICE pointer (suffix _d) owned by the
 * caller; sizes are element counts.  All device buffers are packed per
 * node across the batch:
 *
 *   states   x[total_x][nx], total_x = sum_b (N_b + 1); instance b owns rows
 *            xoff_b .. xoff_b + N_b with xoff_b = sum_{b'<b} (N_b' + 1)
 *   controls u[total_u][nu], total_u = sum_b N_b, uoff_b = sum_{b'<b} N_b'
 *   A[total_u][nx][nx], B[total_u][nx][nu], d[total_u][nx]  (row-major)
 *
 * Calls are asynchronous on the given CUDA stream (a cudaStream_t passed
 * as void*; NULL = legacy default stream).  They return validation and
 * launch errors synchronously; numerical outcomes are reported per
 * instance in the stats records.  No call allocates device memory except
 * ucn_problem_create (which allocates the whole workspace); no exception
 * crosses the ABI.  ucn_last_error() returns a thread-local message for
 * the last failing call on the calling thread.
 *
 * Equations cited are those of the paper:
 *   Eq. (1)   the discrete nonlinear optimal control problem
 *   Eq. (2)   the convex QP subproblem at SCP iterate k
 *   Eq. (3)   the augmented Lagrangian of the temporal splitting
 *   Eq. (4)   the per-node KKT Hessian H_i (Sec. III-B, Step 1)
 *   Eq. (5)   the dynamic consensus update (Step 2)
 *   Eq. (6)-(7) projections (Step 3);  Eq. (8) dual ascent (Step 4)
 */
#ifndef UCN_H
#define UCN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  UCN_OK = 0,
  UCN_EINVAL = 1,     /* invalid argument or descriptor */
  UCN_ENOMEM = 2,     /* device allocation failed (ucn_problem_create only) */
  UCN_ECUDA = 3,      /* a CUDA runtime call failed */
  UCN_ENUMERIC = 4,   /* per instance: NaN/Inf or a non-positive Cholesky pivot */
  UCN_ENOTCONV = 5,   /* per instance: final defect above defect_tol */
  UCN_ETIMEOUT = 6,   /* per instance: the device time budget ran out */
  UCN_EBUSY = 7       /* serving: no free slot / ring full */
} ucn_status;

typedef enum { UCN_MODEL_QUAD12 = 1, UCN_MODEL_MARS7 = 2, UCN_MODEL_QUAT13 = 3, UCN_MODEL_MARS14 = 4 } ucn_model;

/* Set parameters per instance in ucn_problem_desc.sets. */
#define UCN_SET_PARAMS 8
typedef enum { UCN_PREC_FP64 = 0, UCN_PREC_FP32_REFINE = 1 } ucn_precision;

/*
 * Problem batch (host memory; copied to the device by ucn_problem_create).
 * The OCP of Eq. (1):  min phi(x_N) + sum_i l(x_i,u_i)  s.t.  x_{i+1} = RK4(x_i,u_i,dt),
 * x_0 = x_init, S x_N = x_target (S = term_mask), x_i in X_i, u_i in U_i.
 *
 *  model         UCN_MODEL_QUAD12 (nx=12: p, v, ZYX Euler angles, body rates;
 *                nu=4 rotor thrusts), UCN_MODEL_QUAT13 (nx=13: p, v, unit
 *                quaternion body-to-world scalar first, body rates; nu=4 total
 *                thrust along body z and body torques; Sec. IV-A1) or
 *                UCN_MODEL_MARS7 (nx=7: r Up-East-North, v, mass; nu=3 thrust
 *                vector; non-dimensional units)
 *  horizon[b]    N_b >= 1;  dt[b] RK4 step
 *  model_params  [batch][8]: quadrotors (m, Jx, Jy, Jz, arm, km, drag, g; arm
 *                and km unused by QUAT13); Mars (g, alpha = mass flow per unit
 *                thrust, 0...)
 *  cost          l = 1/2 |x - x_ref|^2_Q + 1/2 |u - u_ref|^2_R (diagonal Q, R),
 *                phi = 1/2 |x_N - x_ref|^2_QN + qN^T x_N       [batch][nx|nu]
 *  boxes         x_lo/x_hi [batch][nx], u_lo/u_hi [batch][nu] (+-inf allowed)
 *  obstacles     quadrotors only: n_obs[b] <= max_obs spheres obs_c [batch][max_obs][3],
 *                obs_r [batch][max_obs]; linearised about the nominal
 *  sets          Mars only [batch][UCN_SET_PARAMS]: thrust_min (linearised |T| >= Tmin),
 *                thrust_max (ball |T| <= Tmax), tan of the glide-slope cone
 *                half-angle; a value <= 0 switches the set off
 *  rho_*         ADMM penalties of Eq. (3); rho_final > 0 selects the geometric
 *                schedule rho_k = rho * (rho_final/rho_geo)^(k/(scp_iters-1))
 *  scp_iters     SCP iteration cap; admm_iters ADMM iterations per SCP iteration
 *  stop          1: stop an instance once an accepted candidate has max defect
 *                <= defect_tol and step <= step_tol (0: run every iteration)
 *  tr_*          l_inf trust region (initial, floor, cap) of Eq. (2c)
 *  w_d           weight of the l1 defect in the acceptance merit
 *  vc_weight     virtual control weight; must be 0 (virtual control is off)
 *  precision     UCN_PREC_FP64: every step in FP64.  UCN_PREC_FP32_REFINE:
 *                Jacobians, factorisation and ADMM in FP32 with one
 *                iterative-refinement step per KKT solve; the nominal
 *                trajectory, RK4 rollout, defects, costs and merits in
 *                double-float (float pairs, ~48 bits; see ucn_df_check),
 *                the acceptance test and the results in FP64
 *  timeout_s     device time budget per ucn_scp_solve launch (0: 60 s)
 *  group         scenarios per group for robust MPC (Sec. IV-A); 0 or 1:
 *                independent instances.  With group = K in [2, UCN_MAX_GROUP] the
 *                instances gK .. gK+K-1 are scenarios of one problem that share
 *                the first control u_0: ucn_scp_solve runs each group's ADMM
 *                iterations in lockstep, setting the first control copy of every
 *                scenario to the average of their Step-3 arguments clamped to the
 *                intersection of their boxes, and accepts, resizes the trust
 *                region and stops per group (sums of the merits, maxima of
 *                defect and step).  The scenarios exchange their contributions
 *                through global memory (release/acquire counters, bounded
 *                waits); a group is launched as one thread-block cluster of K
 *                CTAs when K <= 16, else as K / c clusters of c CTAs (c the
 *                largest divisor of K up to 16), which must be resident
 *                together (ucn_scp_solve returns UCN_EINVAL when they cannot
 *                be).  Requires the
 *                quadrotor model, batch % K == 0 and records that fit in
 *                shared memory; ucn_admm_solve and ucn_problem_set_order
 *                reject grouped problems
 */
/* Largest scenario group (ucn_problem_desc.group). */
#define UCN_MAX_GROUP 1024

typedef struct {
  int model, nx, nu, batch;
  const int* horizon;
  const double* dt;
  const double* model_params;
  const double *Q_diag, *x_ref, *R_diag, *u_ref, *QN_diag, *qN;
  const double *x_lo, *x_hi, *u_lo, *u_hi;
  const double *x_init, *x_target;
  const unsigned char* term_mask;
  int max_obs;
  const int* n_obs;
  const double *obs_c, *obs_r;
  const double* sets;
  double rho_eq, rho_dyn, rho_geo, rho_final;
  int scp_iters, admm_iters, stop;
  double tr_init, tr_min, tr_max, w_d, defect_tol, step_tol, vc_weight;
  int precision;
  double timeout_s;
  int group;
} ucn_problem_desc;

/* Per-instance result of ucn_scp_solve (device memory, 128 bytes). */
typedef struct {
  double defect;        /* max_i |RK4(x_i,u_i) - x_{i+1}|_inf of the returned trajectory, by FP64
                           RK4 steps on the returned doubles on both paths (the status's
                           defect_tol test uses it) */
  double cost;          /* phi(x_N) + sum l(x_i,u_i) of the returned trajectory */
  double merit;         /* cost + w_d * sum_i |defect_i|_1 */
  double primal_res;    /* ADMM primal residual of the last ADMM iteration (Sec. III-B, Step 4) */
  double dual_res;      /* ADMM dual residual of the last ADMM iteration; both norms are sums of
                           squared iterate differences accumulated in FP64 (FP64 path) or in
                           double-float (FP32 path: exact differences of the FP32 iterates,
                           relative error of the sums below 1e-11; see ucn_df_check) */
  double tr_radius;     /* trust-region radius at exit */
  double step;          /* |candidate - nominal|_inf of the last SCP iteration */
  int scp_iters;        /* SCP iterations run */
  int accepted;         /* candidates accepted */
  unsigned long long accept_mask;   /* bit k: iteration k accepted (k < 64) */
  int status;           /* ucn_status: OK, ENUMERIC, ENOTCONV or ETIMEOUT */
  int reserved;
  unsigned long long t_start_ns, t_end_ns;   /* device globaltimer at instance start / end */
  double pad[4];
} ucn_scp_stats;

typedef struct ucn_problem ucn_problem;

/* Validate `desc`, copy it to the device and allocate every workspace the
 * calls below need (the only allocating call).  Blocks until the copies are
 * done.  Errors: UCN_EINVAL (bad sizes, model, pointers, vc_weight != 0,
 * horizon too long), UCN_ENOMEM, UCN_ECUDA.  Eq. (1) and (2) define the data. */
ucn_status ucn_problem_create(const ucn_problem_desc* desc, ucn_problem** out);

/* Free everything ucn_problem_create allocated (synchronises the device). */
void ucn_problem_destroy(ucn_problem* prob);

/* Order in which the fused solve takes the instances (host array, a permutation
 * of 0..batch-1; NULL = instance order).  The default, set by
 * ucn_problem_create, is largest estimated work first, so that the long solves
 * of an uneven batch start in the first wave.  Results do not depend on it.
 * Synchronous (copies the permutation).  Errors: UCN_EINVAL, UCN_ECUDA. */
ucn_status ucn_problem_set_order(ucn_problem* prob, const int* order);

/* Threads per time node of ucn_scp_solve (a scheduling choice; results agree
 * to rounding).  1: one thread per node.  4 (the default for quadrotor problems
 * of at most 128 nodes): the node's 16 rows split over 4 lanes of a warp that
 * exchange vectors by shuffles -- 4x the resident warps and a quarter of the
 * per-thread dependent chain.  UCN_EINVAL for other values, or 4 on a Mars or
 * longer problem.  ucn_problem_lanes returns the current choice (-1: NULL). */
ucn_status ucn_problem_set_lanes(ucn_problem* prob, int lanes_per_node);
int ucn_problem_lanes(const ucn_problem* prob);

/* Kernel launches made by the last ucn_scp_solve / ucn_scp_solve_warm /
 * ucn_admm_solve call on this problem: 1, or 2 when the fused
 * solve ran a first round on its three-CTAs-per-SM variant (see
 * ucn_scp_solve); 0 before the first call, -1 for NULL.  (Not in the paper;
 * for launch accounting.) */
int ucn_problem_last_launches(const ucn_problem* prob);

/* Number of elements of the packed state / trajectory buffers. */
long long ucn_total_x(const ucn_problem* prob);
long long ucn_total_u(const ucn_problem* prob);
/* Doubles written by ucn_state_export (sum over instances of the flat ADMM state). */
long long ucn_state_size(const ucn_problem* prob);

/* Linearisation (Sec. III-A, Eq. (2b)): for every node i < N_b of every
 * instance, A_i = dRK4/dx, B_i = dRK4/du at (xbar_i, ubar_i) and
 * d_i = RK4(xbar_i, ubar_i) - A_i xbar_i - B_i ubar_i.  Forward-mode
 * differentiation through the four RK4 stages, in FP64 (precision FP64)
 * or FP32 for A, B with d in FP64 (precision FP32_REFINE).
 * In: xbar_d [total_x][nx], ubar_d [total_u][nu].  Out: A_d, B_d, d_d. */
ucn_status ucn_linearize(ucn_problem* prob, const double* xbar_d, const double* ubar_d,
                         double* A_d, double* B_d, double* d_d, void* stream);

/* One ADMM call (Sec. III-B, Steps 1-4, `iters` iterations) on each
 * instance's QP of Eq. (2) built at the nominal (xbar, ubar) with the given
 * linearisation (A, B, d), trust radius radius_d[b] and the problem's costs,
 * boxes and sets.  H_i of Eq. (4) is assembled and Cholesky-factored once per
 * call.  warm = 0 starts from x = x-hat = z = nominal, zero duals; warm = 1
 * continues from the state left by the previous ucn_admm_solve on this
 * problem.  Out: xhat_d [total_x][nx], uhat_d [total_u][nu] (the mirror
 * trajectory), res_d [batch][2] (primal, dual residual), status_d [batch]. */
ucn_status ucn_admm_solve(ucn_problem* prob, const double* xbar_d, const double* ubar_d,
                          const double* A_d, const double* B_d, const double* d_d,
                          const double* radius_d, int iters, int warm,
                          double* xhat_d, double* uhat_d, double* res_d, int* status_d,
                          void* stream);

/* Copy the ADMM state left by the last ucn_admm_solve / ucn_scp_solve, in
 * absolute FP64 coordinates, to state_d [ucn_state_size].  Per instance, in
 * order: x (N+1)nx, u N nu, z (N+1)nx (z_0 = 0), lambda (N+1)nx, mu (N+1)nx,
 * x-hat (N+1)nx, u-hat N nu, nu_x (N+1)nx, nu_u N nu, mirrors s (N+1) mb 3 and
 * their duals (N+1) mb 3, where mb = max_obs (quad) or 3 (Mars: glide cone,
 * thrust ball, thrust lower bound). */
ucn_status ucn_state_export(ucn_problem* prob, double* state_d, void* stream);

/* Full SCP solve (Sec. III-A with the ADMM of Sec. III-B) of every
 * instance by persistent kernel launches that each run whole solves: per SCP
 * iteration the RK4 linearisation, assembly + factorisation, admm_iters ADMM
 * iterations, and the rollout / defect / trust-region acceptance test, all on
 * the device, one CTA per instance.  One launch; for batches of the 3-DOF Mars
 * model in FP32 that are not a whole number of resident rounds, a first launch
 * runs one round on a three-CTAs-per-SM variant of the same kernel and a second
 * the rest (same results per instance).  In: initial guesses x0_d, u0_d.  Out:
 * x_out_d, u_out_d (the last accepted trajectory), stats_d [batch], status_d
 * [batch] (== stats.status).  An instance whose data or guesses hold a NaN (or an
 * infinity outside the bounds and set parameters) ends UCN_ENUMERIC after its
 * first factorisation; the other instances are not affected. */
ucn_status ucn_scp_solve(ucn_problem* prob, const double* x0_d, const double* u0_d,
                         double* x_out_d, double* u_out_d, ucn_scp_stats* stats_d,
                         int* status_d, void* stream);

/* ucn_scp_solve started from a kept ADMM state instead of the cold start
 * (Sec. III-B: the inner ADMM solves are warm-started; here across solves, as
 * a server or a receding-horizon loop keeps the state of a finished solve).
 * state_d [ucn_state_size]: the absolute FP64 layout of ucn_state_export (for
 * instance b, the state of a solve of the same horizon -- typically exported
 * by an earlier solve of this or a nearby problem); each instance's variables
 * are taken relative to its guess (x0_d, u0_d), its mirror sets are
 * re-projected with the first SCP iteration's sets, as every later iteration
 * does, and with a penalty schedule (rho_final > 0) every SCP iteration uses
 * the schedule's final penalties, at which the kept state was computed.
 * Asynchronous on `stream`: state_d is copied into the problem's state buffer
 * first (it may be that buffer, as after ucn_state_export into it).
 * Errors: UCN_EINVAL (null pointer, scenario groups), UCN_ECUDA. */
ucn_status ucn_scp_solve_warm(ucn_problem* prob, const double* x0_d, const double* u0_d, const double* state_d,
                              double* x_out_d, double* u_out_d, ucn_scp_stats* stats_d, int* status_d,
                              void* stream);

/* Receding-horizon step for MPC (Sec. IV-A: the common first control is
 * executed after each solve and the next solve starts from the previous tube
 * moved one step ahead).
 * From the solution (x_d, u_d) of ucn_scp_solve:
 *   plant    each group's first instance (each instance when group <= 1) is
 *            the plant: x_init <- RK4(x_init, u_0, dt) with its own model
 *            parameters and first control, and every instance of the group
 *            takes that state as its new x_init (the problem's device copy is
 *            updated in place)
 *   shift    xg_d, ug_d, packed like the guesses: xg_0 = the new x_init,
 *            xg_i = x_{i+1} (0 < i < N), xg_N = x_N; ug_i = u_{i+1} (i < N-1),
 *            ug_{N-1} = u_{N-1}
 * Device pointers, asynchronous on `stream`; the outputs may not alias the
 * inputs.  Errors: UCN_EINVAL (null or aliased pointer), UCN_ECUDA. */
ucn_status ucn_mpc_shift(ucn_problem* prob, const double* x_d, const double* u_d, double* xg_d, double* ug_d,
                         void* stream);

/* ---------------------------------------------------------------- double-float check
 * The FP32 path carries its nominal trajectory and does its per-SCP-iteration
 * rollout, defects and merits in double-float arithmetic (a value is hi + lo,
 * two floats, ~48 significant bits) instead of FP64, whose rate on this GPU is
 * 1/64 of FP32.  This entry point runs that arithmetic on given inputs so that
 * it can be checked against FP64 (not in the paper; a diagnostic).
 *   op  UCN_DF_ADD, _SUB, _MUL, _DIV: out[k] = a[k] op b[k];
 *       UCN_DF_SQRT: out[k] = sqrt(a[k]); UCN_DF_ROUND: out[k] = a[k] through
 *       double-float and back;
 *       UCN_DF_SQDIFF_SUM: out[0] = sum_k (float(a[k]) - float(b[k]))^2 and
 *       UCN_DF_SQ_SUM: out[0] = sum_k float(a[k])^2, accumulated in order by the
 *       arithmetic that sums the FP32 path's ADMM residual norms (exact
 *       differences of the float values, double-float sums; one thread);
 *       UCN_DF_RK4 + model: one RK4 step of the model (Eq. (1b)) per row,
 *       a = x [n][nx], b = u [n][nu], prm = model_params [8], step h;
 *       out = [n][nx].
 * Inputs are rounded to double-float first, results returned as doubles.
 * Device pointers, asynchronous on `stream`.  Errors: UCN_EINVAL (unknown op
 * or model, null pointer, n < 0), UCN_ECUDA. */
#define UCN_DF_ADD 0
#define UCN_DF_SUB 1
#define UCN_DF_MUL 2
#define UCN_DF_DIV 3
#define UCN_DF_SQRT 4
#define UCN_DF_ROUND 5
#define UCN_DF_SQDIFF_SUM 6
#define UCN_DF_SQ_SUM 7
#define UCN_DF_RK4 100
ucn_status ucn_df_check(int op, const double* a_d, const double* b_d, const double* prm_d, double h, long long n,
                        double* out_d, void* stream);

/* Scratch held by ucn_scp_solve_noalloc on every GPU that loads the library. */
#define UCN_NOALLOC_SCRATCH_BYTES (64ull << 20)

/* ucn_scp_solve without any device allocation, for callers that cannot call
 * cudaMalloc (a real-time loop that must not allocate or wait on the device,
 * an application whose memory pool owns the GPU, a runtime that only hands out
 * pre-registered buffers).  The paper has no counterpart; this is a
 * deployment variant of the same fused kernel.
 *
 * desc: a host struct as for ucn_problem_create, except that `horizon` is a
 *   HOST array and every other array field is a DEVICE pointer (same layouts;
 *   owned by the caller, read during the kernel).  Device-side contents are
 *   not validated: dt[b] must be > 0; obstacle counts n_obs[b] are clamped to
 *   [0, max_obs] where the kernel reads them.  Quadrotor problems need n_obs
 *   even when max_obs = 0.
 * Buffers: as ucn_scp_solve.  The kernel's scratch -- per-instance index
 *   tables, the penalty schedule and the final ADMM state -- lives in one
 *   static device array of UCN_NOALLOC_SCRATCH_BYTES (64 MiB) per GPU, held
 *   until the process exits.  The tables reach the device as by-value
 *   parameters of small set-up kernels on `stream`: the call copies nothing
 *   from host memory, allocates nothing (device or host) and does not wait for
 *   the stream.
 * Errors: UCN_EINVAL when the batch needs more scratch than that, or when
 *   an instance does not fit in shared memory (there is no global workspace
 *   here), plus the descriptor checks of ucn_problem_create; UCN_ECUDA.
 * The first call on a device looks up the array's device address (once, with
 *   that device current); make that first call before any stream capture.
 * Every call shares the array: calls whose kernels overlap on the GPU race,
 *   so serialise them (one stream, or events).  The array keeps the last
 *   call's contents; nothing in it needs to start at zero (each call writes
 *   every table entry and exported state entry its kernels read). */
ucn_status ucn_scp_solve_noalloc(const ucn_problem_desc* desc, const double* x0_d, const double* u0_d,
                                 double* x_out_d, double* u_out_d, ucn_scp_stats* stats_d,
                                 int* status_d, void* stream);

/* ---------------------------------------------------------------- serving
 * Continuous batching of solves over a preallocated slot pool (not in the
 * paper; the serving layer around the method).  ucn_serve_create allocates
 * everything for `max_slots` instances of up to `max_horizon` nodes of one
 * model and precision, plus `lanes` CUDA streams and a ring of `kept`
 * finished results (0: 2 * max_slots) -- trajectory and final ADMM state --
 * for warm starts.  A request is admitted into a free slot while the sum of
 * admitted footprints stays within hbm_budget_bytes (0: no budget beyond the
 * slots); each pump launches the fused SCP kernel (one CTA per instance) over
 * the slots admitted since the last pump (at most 128) on the next free lane,
 * while earlier launches keep running: the requests' data go up in one copy
 * and a scatter kernel places them.  Each CTA writes its request's result into
 * mapped host memory the moment its solve ends, so a result is ready when its
 * own solve is done, and polls read host memory only.  Every slot has the same
 * CTA size and layout, so a result does not depend on what it was batched with.
 * Solver settings have the meaning they have in ucn_problem_desc. */
typedef struct {
  int model, precision, max_slots, max_horizon, max_obs, lanes, kept;
  double hbm_budget_bytes;
  double rho_eq, rho_dyn, rho_geo, rho_final;
  int scp_iters, admm_iters, stop;
  double tr_init, tr_min, tr_max, w_d, defect_tol, step_tol, timeout_s;
} ucn_serve_config;

/* One solve request (host memory, copied at submit).  Arrays as one instance
 * of ucn_problem_desc (model_params [8], sets [UCN_SET_PARAMS], obs_c [n_obs][3]).  The
 * initial guess is x_guess [(horizon+1)][nx], u_guess [horizon][nu]; if either
 * is NULL the request starts from the kept result of the request `warm_ticket`
 * (same horizon; launched, finished or not): its trajectory as the guess and its
 * final ADMM state as the start of the inner solves, as ucn_scp_solve_warm does
 * (copied on the device; the launch waits for that request's launch). */
typedef struct {
  int horizon, n_obs;
  double dt;
  const double* model_params;
  const double *Q_diag, *x_ref, *R_diag, *u_ref, *QN_diag, *qN;
  const double *x_lo, *x_hi, *u_lo, *u_hi, *x_init, *x_target;
  const unsigned char* term_mask;
  const double *obs_c, *obs_r, *sets;
  const double *x_guess, *u_guess;
  unsigned long long warm_ticket;
} ucn_request;

/* A finished request.  x, u: caller host buffers ((horizon+1)*nx, horizon*nu
 * doubles) filled by ucn_serve_poll when not NULL. */
typedef struct {
  ucn_scp_stats stats;
  double *x, *u;
  unsigned long long ticket;
  int horizon, reserved;
} ucn_result;

typedef struct ucn_server ucn_server;

/* Allocates the server.  Errors: UCN_EINVAL, UCN_ENOMEM, UCN_ECUDA. */
ucn_status ucn_serve_create(const ucn_serve_config* cfg, ucn_server** out);
/* Ends a running request loop, synchronises the device and frees everything. */
void ucn_serve_destroy(ucn_server* srv);
/* Admits a request into a free slot: UCN_OK and a ticket; UCN_EBUSY when no
 * slot is free or its footprint exceeds the HBM budget; UCN_EINVAL. */
ucn_status ucn_serve_submit(ucn_server* srv, const ucn_request* req, unsigned long long* ticket);
/* Launches every admitted slot on a free lane (stream); *launched = their
 * count (0 when nothing was admitted).  UCN_EBUSY when every lane is busy. */
ucn_status ucn_serve_pump(ucn_server* srv, int* launched);
/* Non-blocking (reads host memory; no CUDA call unless the request is still
 * running): UCN_OK and the result (the slot is freed, for reuse once its
 * launch has ended; the result stays kept for warm starts until the ring
 * reuses its entry), UCN_EBUSY while the request
 * is queued or running, UCN_EINVAL for an unknown ticket, UCN_ECUDA if its
 * launch failed. */
ucn_status ucn_serve_poll(ucn_server* srv, unsigned long long ticket, ucn_result* res);
/* Non-blocking: UCN_OK and the result of some finished request (res->ticket
 * says which; res->x, res->u, when not NULL, must hold max_horizon nodes),
 * UCN_EBUSY when none has finished, UCN_ECUDA if a launch failed. */
ucn_status ucn_serve_poll_any(ucn_server* srv, ucn_result* res);
/* Free slots right now (-1 for a NULL server). */
int ucn_serve_free_slots(ucn_server* srv);

/* Device-resident request loop (not in the paper; the serving layer around the
 * method).  ucn_serve_loop_start
 * launches one persistent kernel of `ctas` CTAs (0: as many as can be
 * resident at once) on the server's own stream.  From then on ucn_serve_submit
 * publishes each admitted request at once -- its record into mapped host
 * memory, the slot into a queue, then the queue head -- and a CTA of the
 * running kernel that is free claims it (in submission order), copies its data
 * into the slot, runs the same fused SCP solve as a pump launch (Secs. III-A,
 * III-B: the same kernel body on the same slot layout), keeps its result in the
 * ring and delivers it to host memory; there is no pump and no launch per
 * request.  Requests admitted and not pumped when the loop starts go to it
 * first.  Every wait of the kernel is bounded: once no request has been
 * published to the server for `idle_s` seconds (0 < idle_s <= 60) its CTAs
 * end (each CTA's idle clock restarts whenever a request is published, so the
 * loop keeps all its CTAs while requests arrive), and the next submit, pump,
 * poll or poll_any relaunches the loop if requests wait.  While the loop is on,
 * ucn_serve_pump only does that relaunch (*launched = 0), and a warm start must
 * name a result that has been delivered (UCN_EBUSY until then).  Errors:
 * UCN_EINVAL (bad arguments, loop already on), UCN_ECUDA. */
ucn_status ucn_serve_loop_start(ucn_server* srv, int ctas, double idle_s);
/* Serves every published request, ends the loop kernel (blocks until it has)
 * and returns the server to pump launches; UCN_OK when no loop is on.
 * Results stay in their slots until polled.  UCN_ECUDA if the loop failed (a
 * launch error or a device fault): requests it had not delivered cannot
 * complete, so destroy the server. */
ucn_status ucn_serve_loop_stop(ucn_server* srv);
/* Launches of the loop kernel so far (the first one and every relaunch after
 * an idle end); -1 for a NULL server. */
int ucn_serve_loop_launches(ucn_server* srv);
/* How many CTAs of this server's loop kernel can be resident at once on the
 * current device (the `ctas` that 0 stands for); -1 for a NULL server.  Several servers whose loops run at the same time
 * share the device: CTAs beyond what fits start only when others end, so give
 * each loop a share of its capacity. */
int ucn_serve_loop_capacity(ucn_server* srv);

/* Thread-local description of the last error on this thread ("" if none). */
const char* ucn_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* UCN_H */
