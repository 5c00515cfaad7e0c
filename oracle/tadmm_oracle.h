/*
 * Plain CPU FP64 oracle for the TurboADMM hot path (arXiv 2602.15838).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the GPU library; it is
 * never part of the product path.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header or
 * constant with the CUDA implementation.
 *
 * What it computes (all in double precision, written for readability, not speed):
 *   - orc_agent_qp_solve: the per-agent x-update QP of Sec. IV.A (local QP and
 *     its compact form), assembled densely over z = [x_1..x_T; u_0..u_{T-1}] and
 *     solved by the textbook primal active-set method (Nocedal & Wright,
 *     Numerical Optimization, Alg. 16.3) where every working-set iterate solves
 *     the full dense KKT system by LU with partial pivoting.
 *   - orc_admm: the ADMM iteration of Sec. III.B / IV.A (x-update, consensus
 *     projection, dual update, residuals) in its literal per-side vector form,
 *     optionally with residual balancing of rho (Boyd et al. 2011, Sec. 3.4.1)
 *     over-relaxation (Sec. 3.4.3 there) and acceleration with restart
 *     (Goldstein et al. 2014), extensions toward the iteration-count work the
 *     paper names as future work.
 *   - orc_agent_qp_homotopy: the parametric hot start of qpOASES (Sec. IV.C
 *     names its hot start) as a homotopy in the QP's linear term.
 *   - orc_global_qp: the centralized linearized QP of Eq. (1) condensed in all
 *     inputs and solved by the same active-set method (the ADMM fixed point).
 *   - orc_agent_bruteforce: exhaustive active-set enumeration for tiny QPs.
 *   - orc_global_gradient: implicit differentiation of the global QP's KKT
 *     system at a given active set (held inputs substituted, independent
 *     halfspace rows by pivoted Gram-Schmidt, dense LU).
 *
 * Parity pins: every function here is pinned by tests against closed forms,
 * library routines (bounded least squares), brute force and KKT invariants;
 * the paper prints no worked numeric example, so no value is pinned to a
 * number printed in the paper ("parity unpinned" against the paper itself,
 * only its problem-size table is checked).
 */
#ifndef TADMM_ORACLE_H
#define TADMM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_CONVERGED = 0, ORC_NOT_CONVERGED = 1, ORC_QP_FAIL = 2, ORC_NUMERIC = 3 };
enum { ORC_START_COLD = 0, ORC_START_HOT = 1, ORC_START_TURBO = 2, ORC_START_HOMOTOPY = 3 };
/* per-agent QP start kinds */
enum { ORC_QP_COLD = 0, ORC_QP_LQR = 1, ORC_QP_GIVEN = 2 };

/* One per-agent box-constrained LQ problem (compact form, Sec. IV.A):
 *   min  sum_{t=1..T} (1/2 x_t' diag(Hx_t) x_t + gx_t' x_t) + sum_{t=0..T-1} 1/2 u_t' diag(Hu) u_t
 *   s.t. x_{t+1} = A x_t + B u_t, x_0 given, umin <= u_t <= umax.            */
typedef struct {
  int T, nx, nu;
  const double *A, *B;        /* [nx*nx], [nx*nu] row-major */
  const double *Hx;           /* [T][nx] diagonal Hessian of x_t, t = 1..T */
  const double *gx;           /* [T][nx] linear term of x_t, t = 1..T */
  const double *Hu;           /* [nu] diagonal Hessian of every u_t */
  const double *x0;           /* [nx] */
  const double *umin, *umax;  /* [nu] */
} orc_agent_qp;

/* Working-set codes per input component: 0 free, 1 at lower bound, 2 at upper. */
int orc_agent_qp_solve(const orc_agent_qp* q, int start, int as_max, double eps_rel,
                       double* u, int8_t* W, double* x, double* mu, int* n_eqp);

/* Parametric (homotopy) hot start in the manner of qpOASES: from the optimum
 * (u, W, mu) of the same QP with state linear term gx_old, follow the optimum
 * along gx(tau) = gx_old + tau (q->gx - gx_old), tau from 0 to 1, changing the
 * working set at each breakpoint (a free input reaching a bound, or a bound
 * multiplier reaching zero); then the primal active-set method from the end
 * point confirms optimality.  n_steps = direction solves of the homotopy,
 * n_eqp = all EQP solves. */
int orc_agent_qp_homotopy(const orc_agent_qp* q, const double* gx_old, int as_max, double eps_rel, double* u,
                          int8_t* W, double* x, double* mu, int* n_eqp, int* n_steps);

/* Equality-constrained QP with inputs in W fixed at their bounds (dense KKT). */
int orc_agent_eqp(const orc_agent_qp* q, const int8_t* W, double* u, double* x, double* mu);

/* Enumerates all 3^(T*nu) working sets; returns the number of KKT points found. */
int orc_agent_bruteforce(const orc_agent_qp* q, double tol, double* u, int8_t* W);

typedef struct {
  int N, T, nx, nu, dp;
  const double *A, *B;                 /* shared model */
  const double *Qd, *Rd, *Qfd;         /* [N][nx], [N][nu], [N][nx] */
  const double *x_init, *x_ref;        /* [N][nx] */
  const double *umin, *umax;           /* [nu] */
  const double *a;                     /* [P][T][dp] in pair order, t = 1..T */
  const double *w0;                    /* [N][T][dp] initial consensus positions */
  double d_min, rho;
  int P;                               /* number of listed pairs (ignored when pairs is NULL) */
  const int *pairs;                    /* [P][2] coupled pairs (i < j); NULL: all N(N-1)/2 pairs in
                                          lexicographic order.  Agent i's copy count n_c is its
                                          number of pairs. */
  const double *Ai, *Bi;               /* heterogeneous agents: [N][nx][nx], [N][nx][nu] per-agent
                                          dynamics; NULL: every agent has the shared A, B */
} orc_scenario;

typedef struct {
  int start_mode;     /* ORC_START_* */
  int as_max;         /* cap on EQP solves per agent QP */
  double eps_rel;     /* multiplier drop tolerance scale */
  double tol;         /* residual tolerance */
  int max_iter;       /* ADMM iteration cap */
  int nthreads;       /* OpenMP threads over agents (<=0: serial) */
  int adapt_every;    /* residual balancing of rho every this many iterations (0: fixed rho) */
  double adapt_mu;    /* imbalance ratio that triggers a change */
  double adapt_tau;   /* factor of a change */
  double relax_alpha; /* over-relaxation: the projection and the dual update use
                         alpha p + (1 - alpha) w^k instead of p (0 or 1: none) */
  double restart_eta; /* accelerated ADMM with restart (0: off; in (0, 1): the
                         restart factor) */
} orc_options;

typedef struct {
  double* X;          /* [N][T+1][nx] */
  double* U;          /* [N][T][nu] */
  double* theta;      /* [P][T] last projection step (multiplier / rho) */
  int8_t* W;          /* [N][T][nu] final working sets */
  double* mu;         /* [N][T][nu] bound multipliers of the final x-update */
  double* trace;      /* optional [max_iter][2]: r, s per iteration */
  int iters;
  int status;
  double r, s;
  int64_t as_iters;   /* EQP solves summed over agents and iterations */
  double inv_dev;     /* max |y_i + theta a| and |y_j - theta a| over the run */
  double rho_final;   /* penalty at the end of the run */
  int rho_changes;    /* number of penalty changes */
  int restarts;       /* restarts of the accelerated iteration */
  int64_t homotopy_steps; /* direction solves of the homotopy hot starts (ORC_START_HOMOTOPY) */
} orc_result;

/* Projection of (v_i, v_j) onto {a'(w_i - w_j) >= d}; returns theta >= 0 with
 * w_i = v_i + theta a, w_j = v_j - theta a.  |a| must be 1. */
double orc_halfspace_project(int dp, const double* a, double d, const double* vi, const double* vj,
                             double* wi, double* wj);

/* x-update of agent i alone for a given coupling term h [T][dp] (the sum over
 * partners of consensus copy minus scaled dual); start is an ORC_QP_* kind. */
int orc_agent_xupdate(const orc_scenario* s, int i, const double* h, int start, int as_max, double eps_rel,
                      double* u, int8_t* W, double* x, double* mu, int* n_eqp);

int orc_admm(const orc_scenario* s, const orc_options* o, orc_result* res);
/* Scenarios in parallel (OpenMP dynamic schedule); returns number of threads used. */
int orc_admm_batch(const orc_scenario* s, int n_scen, const orc_options* o, orc_result* res,
                   int nthreads);

/* Centralized QP of Eq. (1) with linearized halfspaces, condensed in all inputs,
 * solved by the primal active-set method from U = 0 (the feasible guess). */
typedef struct {
  double* X;          /* [N][T+1][nx] */
  double* U;          /* [N][T][nu] */
  double* mu_h;       /* [P][T] halfspace multipliers (0 if inactive) */
  uint8_t* act_h;     /* [P][T] halfspace in final working set */
  int8_t* W;          /* [N][T][nu] bound working set */
  double* mu_u;       /* [N][T][nu] bound multipliers */
  int iters;
  int status;
  double obj;         /* objective of Eq. (1) (no constant dropped except x_0 term) */
} orc_global_result;

int orc_global_qp(const orc_scenario* s, int as_max, double eps_rel, orc_global_result* res);

/* Solution of the global QP with the given active set held as equalities
 * (halfspaces with act_h=1 and bounds W), i.e. the polished KKT point, and the
 * gradient of loss = sum_{i,t=1..T} ||C x_{i,t} - target_{i,t}||^2 with respect
 * to diag(Q_i) (with Qf_i = qf_tie * Q_i), diag(R_i) and the goal x_ref_i.
 * Active halfspace rows that are linearly dependent (on the inputs not held at
 * a bound) are allowed: the polished point is the minimizer subject to the
 * active rows with their right-hand side projected (Euclidean, least squares)
 * onto the range of those rows, which equals the plain EQP solution when the
 * rows are consistent; the gradient is that of this solution map.  Optional
 * outputs (NULL to skip): mu_h [P][T] halfspace and mu_u [N][T][nu] bound
 * multipliers of the polished point (0 for rows found dependent and for
 * inactive ones) and the number of dependent active halfspace rows. */
int orc_global_gradient(const orc_scenario* s, const uint8_t* act_h, const int8_t* W,
                        const double* targets /* [N][T][dp] */, double qf_tie,
                        double* X, double* U, double* loss,
                        double* gQ /* [N][nx] */, double* gR /* [N][nu] */,
                        double* gGoal /* [N][nx] */, double* mu_h, double* mu_u, int* n_dependent);

#ifdef __cplusplus
}
#endif
#endif
