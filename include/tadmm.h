/*
 * tadmm — batched ADMM for densely coupled multi-agent trajectory QPs on GB300
 * (sm_103a).  C ABI of the library libtadmm.so.
 *
 * The method (TurboADMM, arXiv 2602.15838) solves the centralized QP of
 * Eq. (1) (Sec. III.A) with the collision constraints linearized to halfspaces
 *     a_ijt' (p_it - p_jt) >= d_min,   i < j,  t = 1..T,
 * by ADMM (Sec. III.B): each iteration solves one box-constrained LQ problem
 * per agent (the local QP of Sec. IV.A, a Riccati-factorized primal active set
 * that is warm-started from the affine LQR solution of Sec. IV.B on the first
 * iteration and hot-started from the previous working set and factors
 * afterwards, Sec. IV.C), then projects the per-pair consensus copies onto the
 * halfspace, updates the scaled duals (Sec. IV.A consensus and dual updates)
 * and reduces the primal and dual residuals (Sec. V.A convergence criteria).
 *
 * Model conventions: state x = [p; v] with the position p in the first dp
 * components (C = [I_dp 0]); objective exactly as Eq. (1) (no factor 1/2):
 * sum_t ||x_t - x_ref||^2_Q + ||u_t||^2_R over t < T plus ||x_T - x_ref||^2_Qf,
 * diagonal Q, R, Qf; input box umin <= u_t <= umax; no state bounds.
 * Supported dimensions: (nx, nu, dp) = (4, 2, 2) and (6, 3, 3).
 *
 * Errors: every call returns TADMM_OK (0) or a negative TADMM_E* code and
 * never aborts; tadmm_last_error() describes the last failure of the calling
 * thread.  Per-scenario outcomes are reported in a status array.
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream); work is
 * enqueued asynchronously unless stated.
 */
#ifndef TADMM_H
#define TADMM_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define TADMM_OK 0
#define TADMM_EINVAL (-1) /* bad argument or unsupported dimensions */
#define TADMM_ENOMEM (-2) /* device or host allocation failed */
#define TADMM_ECUDA (-3)  /* a CUDA runtime call failed */
#define TADMM_ESTATE (-4) /* call out of order (e.g. backward before solve) */

/* per-scenario status */
#define TADMM_CONVERGED 0     /* r <= tol and s <= tol */
#define TADMM_NOT_CONVERGED 1 /* max_iter reached */
#define TADMM_QP_FAIL 2       /* an agent QP hit the active-set iteration cap */
#define TADMM_NUMERIC 3       /* non-finite residual or non-positive pivot */
#define TADMM_INVALID_INPUT 4 /* tadmm_solve_noalloc: an input value breaks the rules that
                                 tadmm_create checks on the host; nothing was solved */

/* start modes of the per-agent QP (the paper's ablation variants, Sec. V.B) */
#define TADMM_START_COLD 0  /* BaseADMM: u = clip(0), empty working set, every iteration */
#define TADMM_START_HOT 1   /* HotstartADMM: cold first iteration, then previous (u, W, factors) */
#define TADMM_START_TURBO 2 /* TurboADMM: clipped affine-LQR warm start, then hot start */
#define TADMM_START_HOMOTOPY 3 /* turbo warm start, then a parametric (homotopy) hot start in the manner of
                                  qpOASES, which the paper's hot start names: the optimum is followed from
                                  the previous x-update's linear term to the new one, one direction solve
                                  per working-set change, then confirmed by the primal active set; plain
                                  and graph modes only (EINVAL in the batched mode) */

/* execution modes */
#define TADMM_MODE_BATCHED 0 /* all scenarios, all iterations in one persistent, graph-captured launch */
#define TADMM_MODE_PLAIN 1   /* one scenario at a time, one launch per phase and a host
                                read of the residuals after every iteration */
#define TADMM_MODE_GRAPH 2   /* grid-wide phase kernels over all scenarios repeated by a CUDA
                                graph conditional WHILE node (for scenarios too large for one CTA) */

/* A batch of independent scenarios sharing (nx, nu, dp), the dynamics (A, B)
 * and the input box.  All pointers are HOST pointers, row-major float64, read
 * only during the call that receives them.  Arrays are packed scenario after
 * scenario in this order (P_s = N_s (N_s - 1) / 2):
 *   per agent  (sum N_s rows):          Qd, Qfd, x_init, x_ref [nx]; Rd [nu]
 *   per pair-step (sum P_s T_s rows):   a [dp], pairs in pair order, then t = 1..T
 *   per agent-step (sum N_s T_s rows):  w0 [dp], agents, then t = 1..T          */
typedef struct {
  int32_t n_scen;
  int32_t nx, nu, dp;
  const int32_t* N;      /* [n_scen] agents per scenario, 1..32767 */
  const int32_t* T;      /* [n_scen] horizon per scenario, 1..100000; with N also
                            (T + 1) * N * 87 < 2^31 (the per-stage arrays of one
                            scenario are indexed in 32 bits), else EINVAL */
  const double* A;       /* [nx*nx] dynamics x_{t+1} = A x_t + B u_t */
  const double* B;       /* [nx*nu] */
  const double* umin;    /* [nu] */
  const double* umax;    /* [nu] */
  const double* Qd;      /* diag Q per agent */
  const double* Rd;      /* diag R per agent */
  const double* Qfd;     /* diag Q_T per agent */
  const double* x_init;  /* initial state per agent */
  const double* x_ref;   /* goal state per agent (constant over t) */
  const double* a;       /* unit halfspace normal per pair-step */
  const double* w0;      /* initial consensus position per agent-step (the guess) */
  const double* d_min;   /* [n_scen] */
  const double* rho;     /* [n_scen] ADMM penalty */
  /* Coupled pairs (an extension: the paper couples all pairs).  NULL: every
   * pair (i < j) of each scenario in lexicographic order, P_s = N_s(N_s-1)/2.
   * Otherwise pair_count[s] = P_s pairs listed in pair_ij [sum P_s][2] (i < j,
   * each pair at most once), scenario after scenario, in the order of the rows
   * of `a`; agent i's number of consensus copies n_c is its number of pairs. */
  const int32_t* pair_count;
  const int32_t* pair_ij;
  /* Heterogeneous agents (an extension: the paper's agents share one model).
   * NULL (both): every agent has A, B above.  Otherwise per-agent dynamics
   * A_agent [sum N][nx][nx] and B_agent [sum N][nx][nu], row-major, agents in
   * scenario order; the input box stays shared.  The products are then the
   * dense ones; not with TADMM_FLAG_DOUBLE_FLOAT (EINVAL). */
  const double* A_agent;
  const double* B_agent;
} tadmm_batch;

typedef struct {
  int32_t precision;       /* 64 (float64 arithmetic) or 32 (float32) */
  int32_t start_mode;      /* TADMM_START_* (TADMM_START_HOMOTOPY: plain and graph modes) */
  int32_t as_max;          /* cap on active-set EQP solves per agent QP; 0 = 10*T*nu + 10 */
  double eps_rel;          /* multiplier drop tolerance scale; 0 = 1e-12 (fp64) / 1e-5 (fp32) */
  int32_t mode;            /* TADMM_MODE_* */
  int32_t threads_per_cta; /* batched mode: threads per scenario CTA; 0 = tuned/default */
  int32_t ctas_per_sm;     /* batched mode: resident CTAs per SM; 0 = tuned/default */
  int32_t kernel_variant;  /* batched mode: register-budget variant 0..2 of the persistent kernel
                              (0: no cap, small active-set rounds on lane groups; 1: 32 threads x
                              12 CTAs/SM; 2: 64 threads x 8 CTAs/SM); results are the same bits */
  int32_t flags;           /* TADMM_FLAG_* bits; 0 = all optimizations on */
  /* Residual balancing of the penalty (an extension: the paper keeps rho fixed;
   * Boyd et al. 2011, Sec. 3.4.1).  Every adapt_every iterations (0 = off), after
   * the residuals r, s of that iteration and if the scenario has not stopped:
   * rho *= adapt_tau when r > adapt_mu * s, rho /= adapt_tau when s > adapt_mu * r,
   * the scaled duals rescaled so that the unscaled multipliers are unchanged.
   * Batched mode only, scenarios of at most 32 agents; EINVAL otherwise. */
  int32_t adapt_every;
  double adapt_mu;         /* > 1 */
  double adapt_tau;        /* > 1 */
  /* Over-relaxation (an extension: the paper's ADMM is unrelaxed; Boyd et al.
   * 2011, Sec. 3.4.3): the consensus projection and the scaled-dual update take
   * alpha p + (1 - alpha) w^k in place of the new positions p; the residuals
   * keep p.  0 or 1: off; otherwise 0 < alpha < 2.  Batched mode only, on the
   * group path (scenarios of at most 32 agents); EINVAL otherwise. */
  double relax_alpha;
} tadmm_options;

/* option flags (results are the same either way; for testing and measurement) */
#define TADMM_FLAG_NO_FUSED_PAIR_GATHER 1 /* separate pair and gather sweeps in the batched kernel */
#define TADMM_FLAG_NO_STRUCTURE 2         /* dense A, B products even for a double integrator */
#define TADMM_FLAG_NO_GROUPING 4          /* one scenario per CTA (no packing of small scenarios) */
#define TADMM_FLAG_DOUBLE_FLOAT 8         /* with precision 64 and the 2D model (4, 2, 2): arithmetic in
                                             double-float (pairs of floats, 48-bit significand) on the
                                             FP32 pipe instead of the FP64 pipe; results agree with
                                             float64 to about 1e-13 relative */
#define TADMM_FLAG_NO_LANE_GROUPS 16      /* stage refactorizations and EQP passes one lane per agent, never
                                             spread over a group of lanes (bitwise the same results) */
#define TADMM_FLAG_NO_COOP_REFACTOR TADMM_FLAG_NO_LANE_GROUPS

typedef struct tadmm_handle tadmm_handle;

/* Validates the batch and deep-copies it into library-owned device memory on
 * the current CUDA device (Sec. III problem data, already linearized).
 * `opt` may be NULL (defaults: fp64, turbo, batched).  On success *out owns
 * all device state until tadmm_destroy.  Synchronous. */
int tadmm_create(const tadmm_batch* batch, const tadmm_options* opt, tadmm_handle** out);

/* Re-uploads new problem data with the same shapes (N, T per scenario and the
 * dimensions must match the handle) from host memory, asynchronously on
 * `stream`; host arrays must stay valid until the stream reaches the copies.
 * With per-agent dynamics the call first synchronizes `stream` (the library
 * repacks the models in a host buffer that an earlier copy may still read). */
int tadmm_update(tadmm_handle* h, const tadmm_batch* batch, void* stream);

/* Replaces the per-agent cost data of Eq. (1) — diag Q, diag R, diag Q_T and the
 * goal state x_ref, each [sum N][nx] (R: [sum N][nu]) in the layouts of
 * tadmm_batch — from host or device memory (any pointer may be NULL: that array
 * is kept), e.g. the parameters of a differentiable layer that live on the GPU.
 * The values are checked on the device by tadmm_create's rules (finite, Q,
 * Q_T >= 0, R > 0); on a violation the call returns TADMM_EINVAL and the
 * handle's data is unchanged.  The other inputs (dynamics, x_init, normals,
 * guesses) and the last solve's results are kept.  Synchronizes `stream`
 * (to read the check). */
int tadmm_update_costs(tadmm_handle* h, const double* Qd, const double* Rd, const double* Qfd, const double* x_ref,
                       void* stream);

/* Runs ADMM from its initial point (consensus copies = w0, duals = 0) until
 * r <= tol and s <= tol or max_iter iterations, for every scenario.
 * r = max |p - w|_inf and s = rho * max |w^{k+1} - w^k|_inf over all pairs,
 * steps, sides and components (Sec. V.A criterion, absolute infinity norms).
 * Asynchronous on `stream`. */
int tadmm_solve(tadmm_handle* h, double tol, int32_t max_iter, void* stream);

/* Copies results into caller buffers (host or device pointers; any may be
 * NULL), converted to float64, then synchronizes `stream`:
 *   X [sum N][T_s+1][nx], U [sum N][T_s][nu], theta [sum P T] (pair-step order
 *   of `a`; the halfspace multiplier is rho * theta), W [sum N][T_s][nu] int8
 *   (0 free, 1 at lower bound, 2 at upper bound), status/iters [n_scen],
 *   res [n_scen][2] (final r, s). */
int tadmm_get_solution(tadmm_handle* h, double* X, double* U, double* theta, int8_t* W,
                       int32_t* status, int32_t* iters, double* res, void* stream);

/* Per-scenario work counters of the last solve (host buffers, synchronous):
 * eqp [n_scen] active-set EQP solves summed over agents and iterations,
 * fact [n_scen] Riccati stage factorizations, pairsteps processed. */
int tadmm_get_counters(tadmm_handle* h, int64_t* eqp, int64_t* fact, int64_t* pairsteps);

/* Outer linearize-and-solve step (the collision constraint |p_i - p_j| >= d_min
 * enters the QP as a halfspace linearized about a guess, Sec. III; repeating
 * the linearization at each solution gives a sequential-QP loop; this step is
 * an extension beyond the single linearized QP).  Replaces, on the device, every scenario's halfspace normals
 * by a_ijt = (p_it - p_jt) / |p_it - p_jt| at the final iterate of the last
 * solve (unchanged where the positions coincide; float64, correctly rounded
 * operations) and the initial consensus positions w0 by that iterate's
 * positions; the next tadmm_solve solves the re-linearized QP.  Asynchronous
 * on `stream`; ESTATE before the first solve.  tadmm_update restores the
 * caller's data. */
int tadmm_relinearize(tadmm_handle* h, void* stream);

/* Sequential-QP loop over the linearization (an extension beyond the single
 * linearized QP, with the termination rule of Sec. V.A: relative objective
 * change and collision-free at every time step).  Outer step m = 1, 2, ...
 * runs tadmm_solve(tol, max_iter) and then, per scenario, forms the objective
 * J_m of Eq. (1) at the solution (every term, t = 0 included) and the smallest
 * pair distance D_m = min |p_it - p_jt| over the coupled pairs and t = 1..T
 * (float64).  A scenario stops at step m when its solve converged, m >= 2,
 * |J_m - J_{m-1}| <= obj_rtol |J_{m-1}| and D_m >= d_min - dist_tol; the others
 * are re-linearized at their solution as tadmm_relinearize does, for at most
 * max_outer steps.  A scenario that stopped keeps its data, so its re-solves in
 * later steps reproduce its solution bit for bit (the work is repeated: every
 * solve runs all scenarios); afterwards tadmm_get_solution returns each
 * scenario's solution at the step where it stopped (or the last one).
 *   dist_tol < 0: 2 sqrt(dp) tol (a converged solve leaves each position within
 *               tol, per component, of consensus copies that satisfy the
 *               halfspace exactly)
 *   outer       [n_scen] outer steps taken (the stopping step)
 *   sqp_status  [n_scen] TADMM_CONVERGED when the rule was met, else
 *               TADMM_NOT_CONVERGED (max_outer reached)
 *   objective   [n_scen] J at the last step taken;  min_dist [n_scen] D there
 * Outputs are host buffers, any may be NULL.  Synchronizes `stream` after
 * every step (to read the measures).  tadmm_update restores the caller's data. */
int tadmm_sqp(tadmm_handle* h, double tol, int32_t max_iter, int32_t max_outer, double obj_rtol, double dist_tol,
              int32_t* outer, int32_t* sqp_status, double* objective, double* min_dist, void* stream);

/* Penalty of each scenario at the end of the last solve and the number of
 * times residual balancing changed it (host buffers, synchronous; either may
 * be NULL).  Without residual balancing: the input rho and 0. */
int tadmm_get_penalty(tadmm_handle* h, double* rho_final, int32_t* rho_changes);

/* Times the candidate launch shapes of the batched persistent kernel (threads
 * per CTA, resident CTAs per SM, register-budget variant) on this batch with
 * `probe_iter` ADMM iterations each, times the three fastest again over
 * 4 x probe_iter iterations and keeps the fastest of those.  Synchronous; the
 * probe solves overwrite the last solution.  Writes the choice to the non-NULL
 * outputs; on an error the previous shape is kept. */
int tadmm_autotune(tadmm_handle* h, int32_t probe_iter, void* stream, int32_t* threads_out,
                   int32_t* ctas_out, int32_t* variant_out);

/* Implicit-KKT gradients of a loss l(X) at the final active set of the last
 * solve (the paper differentiates nothing; this is an addition).  The
 * active set is the final bound working set of every agent plus the halfspaces
 * whose projection step exceeds theta_eps.  At that active set the
 * centralized QP of Eq. (1) (Sec. III.A) with linearized halfspaces is an
 * equality-constrained QP; its KKT system is solved exactly (the polished
 * solution) and differentiated implicitly: per-agent Riccati solves of the
 * block-tridiagonal LQ problems (Sec. IV.B) coupled through a dense Schur
 * complement over the active halfspaces.  Active rows may be linearly
 * dependent: the Schur complement is factored with diagonal pivoting up to its
 * numerical rank (pivots above 1e-12 (float64) or 1e-6 (float32) times its
 * largest diagonal entry), and the polished solution satisfies the active rows
 * with their right-hand side projected, in the least-squares sense, onto the
 * range of the rows (the rows themselves when they are consistent); the
 * gradient is that of this solution map.
 *   grad_X      dl/dX in the layout of X (host or device), entries at t = 0 are
 *               ignored (x_0 is data); NULL: only the polished solution, status
 *               and n_dependent are formed (the gradient outputs are not written)
 *   gQ, gQf     [sum N][nx] dl/d diag(Q_i) (stages t < T) and dl/d diag(Qf_i);
 *               for a tie Qf_i = c Q_i the total is gQ + c gQf
 *   gR          [sum N][nu] dl/d diag(R_i)
 *   gGoal       [sum N][nx] dl/d x_ref_i
 *   X_polished  polished states in the layout of X
 *   status      [n_scen] TADMM_CONVERGED, or TADMM_NUMERIC when a value is not
 *               finite
 *   n_dependent [n_scen] active halfspace rows found linearly dependent
 * Outputs may be host or device pointers, any may be NULL.  Horizons T <= 64.
 * Allocates its scratch on first use; synchronizes `stream`. */
int tadmm_backward(tadmm_handle* h, const double* grad_X, double theta_eps, double* gQ, double* gQf,
                   double* gR, double* gGoal, double* X_polished, int32_t* status, int32_t* n_dependent,
                   void* stream);

/* Active-set polishing of the last solve's result on the centralized QP (an
 * addition beyond the paper).  ADMM stopped at a tolerance leaves halfspaces
 * whose scaled dual theta has not yet decayed to zero, so the active set read
 * off its final iterate (inputs held at a bound by the last x-update,
 * halfspaces with theta > theta_eps) need not be the optimal one.  Each round
 * forms the polished point of the current set (as tadmm_backward does) and
 * checks the KKT conditions of Eq. (1) with the linearized halfspaces there:
 * active rows with a multiplier below -kkt_tol * max(1, largest multiplier)
 * leave the set, and inactive halfspaces violated by more than
 * kkt_tol * max(1, d_min), or inputs outside the box by more than
 * kkt_tol * max(1, |bound|), enter it (held at the violated bound).  Rounds
 * stop when no scenario's set changes or after max_rounds.  The refined set is
 * kept in the handle: tadmm_backward uses it (and ignores its theta_eps) until
 * the next tadmm_solve.
 *   kkt_tol     0 = 1e-9 (float64) / 1e-5 (float32)
 *   act         [sum P T] uint8 halfspace flags in the pair-step order of `a`
 *   W           [sum N][T][nu] int8 held inputs (0 free, 1 lower, 2 upper)
 *   status      [n_scen] TADMM_CONVERGED when the last round found the KKT
 *               conditions satisfied, TADMM_NOT_CONVERGED when max_rounds was
 *               reached first, TADMM_NUMERIC on a non-finite value
 *   rounds      rounds taken
 * act and W may be host or device pointers; status and rounds are host
 * pointers; any may be NULL.  Horizons T <= 64.  Allocates its scratch on
 * first use; synchronizes `stream` after every round. */
int tadmm_polish(tadmm_handle* h, double theta_eps, int32_t max_rounds, double kkt_tol, uint8_t* act, int8_t* W,
                 int32_t* status, int32_t* rounds, void* stream);

/* ---------------------------------------------------------------------------
 * Allocation-free single-scenario solve.
 *
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate device memory while they run, such as a real-time control loop
 * allowed to allocate only at start-up (cudaMalloc takes unpredictable time and
 * can synchronize the device) or a program whose device memory belongs to an
 * outside allocator.  It solves one scenario exactly like tadmm_create +
 * tadmm_solve + tadmm_get_solution in float64, but calls no allocating routine:
 * inputs and outputs are DEVICE buffers owned by the caller, in the layouts of
 * tadmm_batch for n_scen = 1, and all solver state lives in one fixed array of
 * TADMM_NOALLOC_SCRATCH_BYTES in device global memory that the library reserves
 * on every GPU that loads it and holds until the process exits.
 *
 * Limits and behaviour:
 *  - a scenario whose state does not fit (about 32 bytes per pair-step plus
 *    ~400 bytes per agent-step in 2D) is rejected with TADMM_EINVAL naming the
 *    required size; nothing is launched;
 *  - the array's device address is looked up with the device current, on
 *    every call made outside stream capture (a call during a capture reuses the
 *    last lookup on that device); with lazy module loading (the CUDA default)
 *    the first call on each device also loads the library's module there,
 *    which the driver allocates for: make one warm-up call per device (and per
 *    (nx, nu, dp), whose kernels load on first use) at start-up, before any
 *    stream capture; later calls allocate nothing;
 *  - every call shares the array and re-initializes all state it reads; calls
 *    whose GPU work overlaps (other streams or host threads on the same device)
 *    race on it and must be serialized by the caller;
 *  - input values are checked on the device by the rules tadmm_create applies
 *    on the host (finite data, umin <= umax, Q, Qf >= 0, R > 0); a scenario
 *    that breaks one gets status TADMM_INVALID_INPUT with iterations 0 and
 *    residuals NaN, is not solved, and its X, U, theta are left unspecified;
 *    pointers, sizes, rho, d_min, tol and max_iter are checked on the host
 *    (TADMM_EINVAL);
 *  - asynchronous on `stream`; outputs: X [N][T+1][nx], U [N][T][nu],
 *    theta [P*T] (may be NULL), status_iters [2] = {status, iterations},
 *    res [2] = {r, s}; any output pointer may be NULL.                        */
#define TADMM_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)

typedef struct {
  int32_t nx, nu, dp;    /* (4, 2, 2) or (6, 3, 3) */
  int32_t N, T;          /* agents (1..32767) and horizon (>= 1) */
  const double *A, *B, *umin, *umax;              /* device pointers */
  const double *Qd, *Rd, *Qfd, *x_init, *x_ref;   /* device pointers, per agent */
  const double *a;       /* device, [P*T][dp]; may be NULL when N == 1 */
  const double *w0;      /* device, [N*T][dp] */
  double d_min, rho;
} tadmm_scenario_dev;

int tadmm_solve_noalloc(const tadmm_scenario_dev* scenario, int32_t start_mode, double tol, int32_t max_iter,
                        double* X, double* U, double* theta, int32_t* status_iters, double* res, void* stream);

/* Arithmetic roof probe (measurement helper; the paper has no counterpart).
 * Enqueues on `stream` one kernel that fills every SM with blocks_per_sm CTAs
 * of 256 threads, each running 8 independent fused multiply-add chains of
 * `iters` steps in float64 (precision 64) or float32 (32), and writes the
 * floating-point operations it performs (2 per FMA) to *flops (host pointer).
 * Timing it with events on the same stream gives the measured FP64 / FP32
 * throughput of the device.  Asynchronous; allocates nothing. */
int tadmm_fma_probe(int32_t precision, int32_t iters, int32_t blocks_per_sm, double* flops, void* stream);

/* Frees all device memory of the handle (synchronizes the device first). */
void tadmm_destroy(tadmm_handle* h);

/* Message for the last non-OK return on the calling thread ("" if none). */
const char* tadmm_last_error(void);

/* Version string of the library build. */
const char* tadmm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TADMM_H */
