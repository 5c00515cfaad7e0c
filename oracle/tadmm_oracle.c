/*
 * Plain CPU FP64 oracle for the TurboADMM hot path (arXiv 2602.15838).
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  See the header for
 * what each function computes and which part of the paper it follows.
 *
 * Readings of the paper used here (the paper is silent or inconsistent on them):
 *  - Objective is Eq. (1) exactly (no 1/2), so the compact form of Sec. IV.A
 *    has Hessian blocks 2Q, 2Q_T, 2R plus rho*n_c*C'C on positions, with
 *    n_c = N-1 consensus copies per agent (the sum over j != i of the local QP).
 *  - The consensus step of Sec. IV.A is read as the Euclidean projection of the
 *    two per-side copies (v_i, v_j) = (p_i + y_i, p_j + y_j) onto the linearized
 *    halfspace a'(w_i - w_j) >= d_min, followed by the scaled dual update
 *    y += p - w (Sec. III.B / IV.A dual update with y = lambda / rho).
 *  - Collision halfspaces act on t = 1..T (x_0 is data), input boxes on
 *    u_0..u_{T-1}, no state bounds.
 *  - Residuals: r = max |p - w|_inf, s = rho * max |w^{k+1} - w^k|_inf over all
 *    pairs, steps and sides; stop when both are <= tol (checked every iteration).
 *  - Initial consensus copies are the guess positions, initial duals zero.
 *  - Active-set rules (Nocedal & Wright Alg. 16.3): after a full step the
 *    multipliers of that solve are used without re-solving; the working-set
 *    entry with the most negative multiplier is dropped if it is below
 *    -eps_rel * max(1, max |mu|); the blocking constraint is the smallest ratio,
 *    ties to the lowest (t, c) index; ratios are clamped at 0.
 *  - Warm (turbo) start: unconstrained LQR solution clipped to the box, working
 *    set = clipped components; if nothing is clipped the LQR solution is the
 *    QP solution.  Cold start: u = clip(0), empty working set.  Hot start: the
 *    previous ADMM iteration's inputs and working set.
 */
#include "tadmm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX2(i, j, ld) ((size_t)(i) * (size_t)(ld) + (size_t)(j))

/* dynamics of agent i: its own (heterogeneous agents) or the shared model */
static const double* agent_A(const orc_scenario* s, int i) {
  return s->Ai ? s->Ai + (size_t)i * s->nx * s->nx : s->A;
}
static const double* agent_B(const orc_scenario* s, int i) {
  return s->Bi ? s->Bi + (size_t)i * s->nx * s->nu : s->B;
}

/* ------------------------------------------------------------------------- */
/* Dense linear algebra                                                        */
/* ------------------------------------------------------------------------- */

/* Solves K x = b by Gaussian elimination with partial pivoting.  K (n x n,
 * row-major) is destroyed; b is overwritten with x.  Returns -1 if a pivot is
 * zero or not finite. */
static int lu_solve(int n, double* K, double* b) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    double best = fabs(K[IDX2(k, k, n)]);
    for (int i = k + 1; i < n; ++i) {
      double v = fabs(K[IDX2(i, k, n)]);
      if (v > best) { best = v; piv = i; }
    }
    if (!(best > 0.0) || !isfinite(best)) return -1;
    if (piv != k) {
      for (int j = 0; j < n; ++j) {
        double tmp = K[IDX2(k, j, n)];
        K[IDX2(k, j, n)] = K[IDX2(piv, j, n)];
        K[IDX2(piv, j, n)] = tmp;
      }
      double tb = b[k]; b[k] = b[piv]; b[piv] = tb;
    }
    for (int i = k + 1; i < n; ++i) {
      double f = K[IDX2(i, k, n)] / K[IDX2(k, k, n)];
      if (f == 0.0) continue;
      for (int j = k; j < n; ++j) K[IDX2(i, j, n)] -= f * K[IDX2(k, j, n)];
      b[i] -= f * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double acc = b[i];
    for (int j = i + 1; j < n; ++j) acc -= K[IDX2(i, j, n)] * b[j];
    b[i] = acc / K[IDX2(i, i, n)];
  }
  return 0;
}

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* x_{t+1} = A x_t + B u_t from x_0. */
static void simulate(int T, int nx, int nu, const double* A, const double* B, const double* x0,
                     const double* u, double* x) {
  memcpy(x, x0, sizeof(double) * nx);
  for (int t = 0; t < T; ++t) {
    const double* xt = x + (size_t)t * nx;
    double* xn = x + (size_t)(t + 1) * nx;
    for (int r = 0; r < nx; ++r) {
      double acc = 0.0;
      for (int c = 0; c < nx; ++c) acc += A[IDX2(r, c, nx)] * xt[c];
      for (int c = 0; c < nu; ++c) acc += B[IDX2(r, c, nu)] * u[(size_t)t * nu + c];
      xn[r] = acc;
    }
  }
}

/* ------------------------------------------------------------------------- */
/* Per-agent QP: dense assembly (compact form of Sec. IV.A)                    */
/* ------------------------------------------------------------------------- */

/* Variables z = [x_1 .. x_T ; u_0 .. u_{T-1}].  KKT system
 *   [ H    E'   Aw' ] [z]   [-g ]
 *   [ E    0    0   ] [nu] = [ e ]
 *   [ Aw   0    0   ] [om]   [ bw]
 * with E the dynamics rows x_{t+1} - A x_t - B u_t = (t==0 ? A x_0 : 0) and Aw
 * the unit rows of the inputs held at a bound.  Multiplier of a lower bound is
 * -om, of an upper bound +om (inequality written as g(z) >= 0). */
int orc_agent_eqp(const orc_agent_qp* q, const int8_t* W, double* u, double* x, double* mu) {
  const int T = q->T, nx = q->nx, nu = q->nu;
  const int nz = T * (nx + nu), ne = T * nx, nU = T * nu;
  int nW = 0;
  for (int k = 0; k < nU; ++k) nW += (W[k] != 0);
  const int nk = nz + ne + nW;
  double* K = (double*)calloc((size_t)nk * nk, sizeof(double));
  double* b = (double*)calloc((size_t)nk, sizeof(double));
  if (!K || !b) { free(K); free(b); return -1; }
  const int ux = T * nx; /* offset of u_0 in z */
  for (int t = 1; t <= T; ++t)
    for (int r = 0; r < nx; ++r) {
      int i = (t - 1) * nx + r;
      K[IDX2(i, i, nk)] = q->Hx[(size_t)(t - 1) * nx + r];
      b[i] = -q->gx[(size_t)(t - 1) * nx + r];
    }
  for (int t = 0; t < T; ++t)
    for (int c = 0; c < nu; ++c) {
      int i = ux + t * nu + c;
      K[IDX2(i, i, nk)] = q->Hu[c];
      b[i] = 0.0;
    }
  for (int t = 0; t < T; ++t)
    for (int r = 0; r < nx; ++r) {
      int row = nz + t * nx + r;
      int col = t * nx + r; /* x_{t+1} */
      K[IDX2(row, col, nk)] += 1.0;
      K[IDX2(col, row, nk)] += 1.0;
      if (t >= 1) {
        for (int c = 0; c < nx; ++c) {
          int cx = (t - 1) * nx + c; /* x_t */
          K[IDX2(row, cx, nk)] -= q->A[IDX2(r, c, nx)];
          K[IDX2(cx, row, nk)] -= q->A[IDX2(r, c, nx)];
        }
        b[row] = 0.0;
      } else {
        double ax0 = 0.0;
        for (int c = 0; c < nx; ++c) ax0 += q->A[IDX2(r, c, nx)] * q->x0[c];
        b[row] = ax0;
      }
      for (int c = 0; c < nu; ++c) {
        int cu = ux + t * nu + c;
        K[IDX2(row, cu, nk)] -= q->B[IDX2(r, c, nu)];
        K[IDX2(cu, row, nk)] -= q->B[IDX2(r, c, nu)];
      }
    }
  int w = 0;
  for (int k = 0; k < nU; ++k) {
    if (!W[k]) continue;
    int row = nz + ne + w;
    int cu = ux + k;
    K[IDX2(row, cu, nk)] = 1.0;
    K[IDX2(cu, row, nk)] = 1.0;
    b[row] = (W[k] == 1) ? q->umin[k % nu] : q->umax[k % nu];
    ++w;
  }
  int rc = lu_solve(nk, K, b);
  if (rc == 0) {
    memcpy(x, q->x0, sizeof(double) * nx);
    for (int t = 1; t <= T; ++t)
      for (int r = 0; r < nx; ++r) x[(size_t)t * nx + r] = b[(t - 1) * nx + r];
    w = 0;
    for (int k = 0; k < nU; ++k) {
      if (W[k]) {
        double om = b[nz + ne + w];
        ++w;
        mu[k] = (W[k] == 1) ? -om : om;
        u[k] = (W[k] == 1) ? q->umin[k % nu] : q->umax[k % nu];
      } else {
        mu[k] = 0.0;
        u[k] = b[ux + k];
      }
    }
  }
  free(K);
  free(b);
  return rc;
}

int orc_agent_qp_solve(const orc_agent_qp* q, int start, int as_max, double eps_rel,
                       double* u, int8_t* W, double* x, double* mu, int* n_eqp) {
  const int T = q->T, nx = q->nx, nu = q->nu, nU = T * nu;
  double* us = (double*)malloc(sizeof(double) * nU);
  double* xs = (double*)malloc(sizeof(double) * (size_t)(T + 1) * nx);
  double* ms = (double*)malloc(sizeof(double) * nU);
  int status = ORC_CONVERGED;
  *n_eqp = 0;
  if (!us || !xs || !ms) { status = ORC_NUMERIC; goto done; }

  if (start == ORC_QP_COLD) {
    for (int k = 0; k < nU; ++k) { u[k] = clampd(0.0, q->umin[k % nu], q->umax[k % nu]); W[k] = 0; }
  } else if (start == ORC_QP_LQR) {
    /* Warm start: unconstrained affine-LQR solution, clipped to the box. */
    for (int k = 0; k < nU; ++k) W[k] = 0;
    if (orc_agent_eqp(q, W, us, xs, ms) != 0) { status = ORC_NUMERIC; goto done; }
    int clipped = 0;
    for (int k = 0; k < nU; ++k) {
      double lo = q->umin[k % nu], hi = q->umax[k % nu];
      if (us[k] < lo) { u[k] = lo; W[k] = 1; clipped = 1; }
      else if (us[k] > hi) { u[k] = hi; W[k] = 2; clipped = 1; }
      else u[k] = us[k];
    }
    if (!clipped) {
      memcpy(x, xs, sizeof(double) * (size_t)(T + 1) * nx);
      for (int k = 0; k < nU; ++k) mu[k] = 0.0;
      goto done;
    }
  }
  /* else: start from the given (u, W). */

  {
    int need_solve = 1;
    for (;;) {
      if (need_solve) {
        if (*n_eqp >= as_max) { status = ORC_QP_FAIL; break; }
        (*n_eqp)++;
        if (orc_agent_eqp(q, W, us, xs, ms) != 0) { status = ORC_NUMERIC; break; }
        double alpha = 1.0;
        int blk = -1, bside = 0;
        for (int k = 0; k < nU; ++k) {
          if (W[k]) continue;
          double p = us[k] - u[k];
          if (p < 0.0) {
            double r = (q->umin[k % nu] - u[k]) / p;
            if (r < 0.0) r = 0.0;
            if (r < alpha) { alpha = r; blk = k; bside = 1; }
          } else if (p > 0.0) {
            double r = (q->umax[k % nu] - u[k]) / p;
            if (r < 0.0) r = 0.0;
            if (r < alpha) { alpha = r; blk = k; bside = 2; }
          }
        }
        if (blk >= 0) {
          for (int k = 0; k < nU; ++k)
            if (!W[k]) u[k] += alpha * (us[k] - u[k]);
          u[blk] = (bside == 1) ? q->umin[blk % nu] : q->umax[blk % nu];
          W[blk] = (int8_t)bside;
          continue;
        }
        memcpy(u, us, sizeof(double) * nU);
        memcpy(x, xs, sizeof(double) * (size_t)(T + 1) * nx);
        memcpy(mu, ms, sizeof(double) * nU);
        need_solve = 0;
      }
      double scale = 1.0;
      for (int k = 0; k < nU; ++k)
        if (W[k] && fabs(mu[k]) > scale) scale = fabs(mu[k]);
      double worst = -eps_rel * scale;
      int drop = -1;
      for (int k = 0; k < nU; ++k)
        if (W[k] && mu[k] < worst) { worst = mu[k]; drop = k; }
      if (drop >= 0) {
        W[drop] = 0;
        need_solve = 1;
        continue;
      }
      break;
    }
  }
  if (status != ORC_CONVERGED) {
    simulate(T, nx, nu, q->A, q->B, q->x0, u, x);
    for (int k = 0; k < nU; ++k) mu[k] = 0.0;
  }
done:
  free(us);
  free(xs);
  free(ms);
  return status;
}

/* Tiny-QP brute force: every pattern in {free, lower, upper}^(T*nu). A pattern
 * is a KKT point if its EQP solution is within the box (to tol) and all its
 * multipliers are >= -tol.  The last KKT point found is returned. */
int orc_agent_bruteforce(const orc_agent_qp* q, double tol, double* u, int8_t* W) {
  const int T = q->T, nx = q->nx, nu = q->nu, nU = T * nu;
  if (nU <= 0 || nU > 12) return -1;
  long n_pat = 1;
  for (int k = 0; k < nU; ++k) n_pat *= 3;
  int8_t* Wt = (int8_t*)malloc((size_t)nU);
  double* ut = (double*)malloc(sizeof(double) * nU);
  double* xt = (double*)malloc(sizeof(double) * (size_t)(T + 1) * nx);
  double* mt = (double*)malloc(sizeof(double) * nU);
  int found = 0;
  for (long pat = 0; pat < n_pat; ++pat) {
    long v = pat;
    for (int k = 0; k < nU; ++k) { Wt[k] = (int8_t)(v % 3); v /= 3; }
    if (orc_agent_eqp(q, Wt, ut, xt, mt) != 0) continue;
    int ok = 1;
    for (int k = 0; k < nU && ok; ++k) {
      if (Wt[k] == 0) {
        if (ut[k] < q->umin[k % nu] - tol || ut[k] > q->umax[k % nu] + tol) ok = 0;
      } else if (mt[k] < -tol) {
        ok = 0;
      }
    }
    if (ok) {
      ++found;
      memcpy(u, ut, sizeof(double) * nU);
      memcpy(W, Wt, nU);
    }
  }
  free(Wt); free(ut); free(xt); free(mt);
  return found;
}

/* ------------------------------------------------------------------------- */
/* ADMM (Sec. III.B, IV.A), literal per-side vector form                       */
/* ------------------------------------------------------------------------- */

/* Coupled pairs of a scenario as an [P][2] list (all pairs, lexicographic, when
 * none are listed) and an N x N table of pair indices (-1: not coupled).
 * Both malloc'd; returns P, or -1 on allocation failure. */
static int scen_pairs(const orc_scenario* s, int** list_out, int** table_out) {
  const int N = s->N;
  const int P = s->pairs ? s->P : N * (N - 1) / 2;
  int* list = (int*)malloc(sizeof(int) * (2 * (size_t)P + 2));
  int* table = (int*)malloc(sizeof(int) * ((size_t)N * N + 1));
  if (!list || !table) { free(list); free(table); return -1; }
  for (size_t k = 0; k < (size_t)N * N; ++k) table[k] = -1;
  if (s->pairs) {
    for (int k = 0; k < P; ++k) { list[2 * k] = s->pairs[2 * k]; list[2 * k + 1] = s->pairs[2 * k + 1]; }
  } else {
    int k = 0;
    for (int i = 0; i < N; ++i)
      for (int j = i + 1; j < N; ++j, ++k) { list[2 * k] = i; list[2 * k + 1] = j; }
  }
  for (int k = 0; k < P; ++k) {
    const int i = list[2 * k], j = list[2 * k + 1];
    table[(size_t)i * N + j] = k;
    table[(size_t)j * N + i] = k;
  }
  *list_out = list;
  *table_out = table;
  return P;
}

static inline int pair_index(int N, int i, int j) { /* i < j, lexicographic */
  return i * N - (i * (i + 1)) / 2 + (j - i - 1);
}

/* Euclidean projection of the stacked copies (v_i, v_j) onto the halfspace
 * a'(w_i - w_j) >= d (consensus step, Sec. IV.A, per-side reading).  The
 * constraint normal is (a, -a) with squared norm 2|a|^2 = 2, so the projection
 * moves both copies by theta = max(0, d - a'(v_i - v_j)) / 2 along +-a.
 * Returns theta. */
double orc_halfspace_project(int dp, const double* a, double d, const double* vi, const double* vj,
                             double* wi, double* wj) {
  double g = d;
  for (int c = 0; c < dp; ++c) g -= a[c] * (vi[c] - vj[c]);
  double th = (g > 0.0 ? g : 0.0) / 2.0;
  for (int c = 0; c < dp; ++c) {
    wi[c] = vi[c] + th * a[c];
    wj[c] = vj[c] - th * a[c];
  }
  return th;
}

/* Local QP of agent i (Sec. IV.A) for a given coupling term
 * h_t = sum_{j != i} (w_ij,t - y_ij,t), t = 1..T, assembled in the compact form
 * (Hessian 2Q, 2Q_T, 2R plus rho n_c C'C on positions; linear term
 * -2 Q_t x_ref - rho C' h_t) and solved by the active-set method. */
int orc_agent_qp_homotopy(const orc_agent_qp* q, const double* gx_old, int as_max, double eps_rel, double* u,
                          int8_t* W, double* x, double* mu, int* n_eqp, int* n_steps) {
  const int T = q->T, nx = q->nx, nu = q->nu, nU = T * nu;
  double* dgx = (double*)malloc(sizeof(double) * (size_t)T * nx);
  double* du = (double*)malloc(sizeof(double) * nU);
  double* dmu = (double*)malloc(sizeof(double) * nU);
  double* dx = (double*)malloc(sizeof(double) * (size_t)(T + 1) * nx);
  double zero[16] = {0.0};
  int steps = 0, st = ORC_CONVERGED;
  *n_eqp = 0;
  if (!dgx || !du || !dmu || !dx) { st = ORC_NUMERIC; goto done; }
  for (size_t k = 0; k < (size_t)T * nx; ++k) dgx[k] = q->gx[k] - gx_old[k];
  {
    /* the direction problem: linear term d gx, x_0 = 0, fixed inputs at 0 */
    orc_agent_qp qd = *q;
    qd.gx = dgx;
    qd.x0 = zero;
    qd.umin = zero;
    qd.umax = zero;
    double tau = 0.0;
    while (steps < as_max) {
      if (orc_agent_eqp(&qd, W, du, dx, dmu) != 0) { st = ORC_NUMERIC; goto done; }
      ++steps;
      /* largest step along the segment: a free input meets a bound (ties: first
       * index), a multiplier meets zero, or the segment ends */
      double best = 1.0 - tau;
      int bk = -1, side = 0;
      for (int k = 0; k < nU; ++k) {
        const int c = k % nu;
        double t;
        int sd;
        if (!W[k]) {
          if (du[k] > 0.0) { t = (q->umax[c] - u[k]) / du[k]; sd = 2; }
          else if (du[k] < 0.0) { t = (q->umin[c] - u[k]) / du[k]; sd = 1; }
          else continue;
        } else {
          if (!(dmu[k] < 0.0)) continue;
          t = mu[k] / -dmu[k];
          sd = 0;
        }
        if (t < 0.0) t = 0.0;
        if (t < best) { best = t; bk = k; side = sd; }
      }
      for (int k = 0; k < nU; ++k) {
        if (!W[k]) u[k] += best * du[k];
        else mu[k] += best * dmu[k];
      }
      tau += best;
      if (bk < 0) break; /* tau = 1 reached */
      if (side) {
        W[bk] = (int8_t)side;
        u[bk] = (side == 1) ? q->umin[bk % nu] : q->umax[bk % nu];
      } else {
        W[bk] = 0;
      }
      mu[bk] = 0.0;
    }
  }
  {
    int ne = 0;
    st = orc_agent_qp_solve(q, ORC_QP_GIVEN, as_max, eps_rel, u, W, x, mu, &ne);
    *n_eqp = steps + ne;
  }
done:
  if (st == ORC_NUMERIC) *n_eqp = steps;
  *n_steps = steps;
  free(dgx); free(du); free(dmu); free(dx);
  return st;
}

/* Local QP data of agent i (Sec. IV.A) for the coupling term h: Hessian
 * diagonals Hx [T][nx], Hu [nu] and the state linear term gx [T][nx]. */
static void agent_qp_data(const orc_scenario* s, int i, const double* h, double* Hx, double* gx, double* Hu) {
  const int N = s->N, T = s->T, nx = s->nx, nu = s->nu, dp = s->dp;
  int nc = N - 1;
  if (s->pairs) {
    nc = 0;
    for (int k = 0; k < s->P; ++k) nc += (s->pairs[2 * k] == i) + (s->pairs[2 * k + 1] == i);
  }
  const double* Qi = s->Qd + (size_t)i * nx;
  const double* Qfi = s->Qfd + (size_t)i * nx;
  const double* xr = s->x_ref + (size_t)i * nx;
  for (int t = 1; t <= T; ++t) {
    const double* Qt = (t < T) ? Qi : Qfi;
    for (int r = 0; r < nx; ++r) {
      double hx = 2.0 * Qt[r];
      double g = -2.0 * Qt[r] * xr[r];
      if (r < dp) {
        hx += s->rho * nc;
        g -= s->rho * h[(t - 1) * dp + r];
      }
      Hx[(size_t)(t - 1) * nx + r] = hx;
      gx[(size_t)(t - 1) * nx + r] = g;
    }
  }
  for (int c = 0; c < nu; ++c) Hu[c] = 2.0 * s->Rd[(size_t)i * nu + c];
}

int orc_agent_xupdate(const orc_scenario* s, int i, const double* h, int start, int as_max, double eps_rel,
                      double* u, int8_t* W, double* x, double* mu, int* n_eqp) {
  const int T = s->T, nx = s->nx, nu = s->nu;
  double* Hx = (double*)malloc(sizeof(double) * (size_t)T * nx);
  double* gx = (double*)malloc(sizeof(double) * (size_t)T * nx);
  double Hu[16];
  agent_qp_data(s, i, h, Hx, gx, Hu);
  orc_agent_qp q = {T, nx, nu, agent_A(s, i), agent_B(s, i), Hx, gx, Hu, s->x_init + (size_t)i * nx, s->umin, s->umax};
  int st = orc_agent_qp_solve(&q, start, as_max, eps_rel, u, W, x, mu, n_eqp);
  free(Hx);
  free(gx);
  return st;
}

/* x-update of agent i by the homotopy from its previous coupling term h_old
 * (whose optimum u, W, mu are given) to h. */
static int agent_xupdate_homotopy(const orc_scenario* s, int i, const double* h_old, const double* h, int as_max,
                                  double eps_rel, double* u, int8_t* W, double* x, double* mu, int* n_eqp,
                                  int* n_steps) {
  const int T = s->T, nx = s->nx, nu = s->nu;
  double* Hx = (double*)malloc(sizeof(double) * (size_t)T * nx);
  double* gx = (double*)malloc(sizeof(double) * (size_t)T * nx);
  double* gx0 = (double*)malloc(sizeof(double) * (size_t)T * nx);
  double Hu[16];
  agent_qp_data(s, i, h_old, Hx, gx0, Hu);
  agent_qp_data(s, i, h, Hx, gx, Hu);
  orc_agent_qp q = {T, nx, nu, agent_A(s, i), agent_B(s, i), Hx, gx, Hu, s->x_init + (size_t)i * nx, s->umin, s->umax};
  int st = orc_agent_qp_homotopy(&q, gx0, as_max, eps_rel, u, W, x, mu, n_eqp, n_steps);
  free(Hx);
  free(gx);
  free(gx0);
  return st;
}

int orc_admm(const orc_scenario* s, const orc_options* o, orc_result* res) {
  const int N = s->N, T = s->T, nx = s->nx, nu = s->nu, dp = s->dp;
  int *plist = NULL, *ptab = NULL;
  const int P = scen_pairs(s, &plist, &ptab);
  if (P < 0) { res->status = ORC_NUMERIC; return -1; }
  const size_t PS = (size_t)P * T * dp;
  double* wi = (double*)malloc(sizeof(double) * (PS + 1));
  double* wj = (double*)malloc(sizeof(double) * (PS + 1));
  double* yi = (double*)calloc(PS + 1, sizeof(double));
  double* yj = (double*)calloc(PS + 1, sizeof(double));
  double* pos = (double*)malloc(sizeof(double) * ((size_t)N * T * dp + 1));
  /* accelerated ADMM with restart: extrapolated copies and duals, previous iterates */
  const int fast = o->restart_eta > 0.0;
  double* whi = (double*)malloc(sizeof(double) * (PS + 1));
  double* whj = (double*)malloc(sizeof(double) * (PS + 1));
  double* yhi = (double*)calloc(PS + 1, sizeof(double));
  double* yhj = (double*)calloc(PS + 1, sizeof(double));
  double* wpi = (double*)malloc(sizeof(double) * (PS + 1));
  double* wpj = (double*)malloc(sizeof(double) * (PS + 1));
  double* ypi = (double*)calloc(PS + 1, sizeof(double));
  double* ypj = (double*)calloc(PS + 1, sizeof(double));
  double acc_a = 1.0, c_prev = INFINITY;
  /* homotopy hot start: each agent's coupling term of the previous x-update */
  const int homotopy = o->start_mode == ORC_START_HOMOTOPY;
  double* h_prev = homotopy ? (double*)calloc((size_t)N * T * dp + 1, sizeof(double)) : NULL;
  int64_t hom_steps = 0;
  int hom_ok = 1; /* 0 right after a penalty change: the Hessian moved, so that x-update starts as a hot start */
  int64_t as_total = 0;
  orc_scenario sc = *s; /* the penalty changes under residual balancing */
  const double alpha = (o->relax_alpha == 0.0) ? 1.0 : o->relax_alpha;
  res->rho_final = s->rho;
  res->rho_changes = 0;
  res->restarts = 0;
  res->homotopy_steps = 0;
  res->status = ORC_NOT_CONVERGED;
  res->iters = 0;
  res->r = INFINITY;
  res->s = INFINITY;
  res->inv_dev = 0.0;
  if (!wi || !wj || !yi || !yj || !pos) {
    free(wi); free(wj); free(yi); free(yj); free(pos); free(plist); free(ptab);
    res->status = ORC_NUMERIC;
    return -1;
  }
  for (int pk = 0; pk < P; ++pk) {
      const int i = plist[2 * pk], j = plist[2 * pk + 1];
      for (int t = 0; t < T; ++t)
        for (int c = 0; c < dp; ++c) {
          wi[((size_t)pk * T + t) * dp + c] = s->w0[((size_t)i * T + t) * dp + c];
          wj[((size_t)pk * T + t) * dp + c] = s->w0[((size_t)j * T + t) * dp + c];
        }
    }
  for (size_t q = 0; q < PS; ++q) {
    whi[q] = wpi[q] = wi[q];
    whj[q] = wpj[q] = wj[q];
  }
  for (size_t k = 0; k < (size_t)P * T; ++k) res->theta[k] = 0.0;
  for (size_t k = 0; k < (size_t)N * T * nu; ++k) { res->U[k] = 0.0; res->W[k] = 0; res->mu[k] = 0.0; }
  for (int i = 0; i < N; ++i) simulate(T, nx, nu, agent_A(s, i), agent_B(s, i), s->x_init + (size_t)i * nx,
                                       res->U + (size_t)i * T * nu, res->X + (size_t)i * (T + 1) * nx);

  for (int k = 0; k < o->max_iter; ++k) {
    int fail = 0;
    /* --- x-update: N independent per-agent QPs --- */
#pragma omp parallel for schedule(dynamic) num_threads(o->nthreads > 0 ? o->nthreads : 1) \
    reduction(+ : as_total, hom_steps) reduction(max : fail)
    for (int i = 0; i < N; ++i) {
      double* h = (double*)calloc((size_t)T * dp, sizeof(double));
      for (int j = 0; j < N; ++j) {
        if (j == i) continue;
        const int pk = ptab[(size_t)i * N + j];
        if (pk < 0) continue;
        const double* w = fast ? ((i < j) ? whi : whj) : ((i < j) ? wi : wj);
        const double* y = fast ? ((i < j) ? yhi : yhj) : ((i < j) ? yi : yj);
        for (int t = 0; t < T; ++t)
          for (int c = 0; c < dp; ++c)
            h[t * dp + c] += w[((size_t)pk * T + t) * dp + c] - y[((size_t)pk * T + t) * dp + c];
      }
      int start;
      if (o->start_mode == ORC_START_COLD) start = ORC_QP_COLD;
      else if (k == 0) start = (o->start_mode != ORC_START_HOT) ? ORC_QP_LQR : ORC_QP_COLD;
      else start = ORC_QP_GIVEN;
      int neqp = 0, st;
      if (homotopy && k > 0 && hom_ok) {
        int nst = 0;
        st = agent_xupdate_homotopy(&sc, i, h_prev + (size_t)i * T * dp, h, o->as_max, o->eps_rel,
                                    res->U + (size_t)i * T * nu, res->W + (size_t)i * T * nu,
                                    res->X + (size_t)i * (T + 1) * nx, res->mu + (size_t)i * T * nu, &neqp, &nst);
        hom_steps += nst;
      } else {
        st = orc_agent_xupdate(&sc, i, h, start, o->as_max, o->eps_rel, res->U + (size_t)i * T * nu,
                               res->W + (size_t)i * T * nu, res->X + (size_t)i * (T + 1) * nx,
                               res->mu + (size_t)i * T * nu, &neqp);
      }
      if (homotopy) memcpy(h_prev + (size_t)i * T * dp, h, sizeof(double) * (size_t)T * dp);
      as_total += neqp;
      if (st > fail) fail = st;
      free(h);
    }
    res->iters = k + 1;
    hom_ok = 1;
    if (fail) { res->status = fail; break; }
    for (int i = 0; i < N; ++i)
      for (int t = 1; t <= T; ++t)
        for (int c = 0; c < dp; ++c)
          pos[((size_t)i * T + (t - 1)) * dp + c] = res->X[((size_t)i * (T + 1) + t) * nx + c];

    /* --- consensus projection and scaled dual update, per pair and step --- */
    double r = 0.0, sd = 0.0, cdu = 0.0, dev = res->inv_dev;
    for (int pk = 0; pk < P; ++pk) {
        const int i = plist[2 * pk], j = plist[2 * pk + 1];
        for (int t = 0; t < T; ++t) {
          size_t o2 = ((size_t)pk * T + t) * dp;
          const double* a = s->a + o2;
          const double* pi = pos + ((size_t)i * T + t) * dp;
          const double* pj = pos + ((size_t)j * T + t) * dp;
          /* over-relaxation (Boyd et al. 2011, Sec. 3.4.3): the relaxed positions
           * alpha p + (1 - alpha) w^k replace p in the projection and the dual
           * update; the residuals keep p */
          double hi[3], hj[3], vi[3], vj[3], nwi[3], nwj[3];
          for (int c = 0; c < dp; ++c) {
            hi[c] = (alpha == 1.0) ? pi[c] : alpha * pi[c] + (1.0 - alpha) * wi[o2 + c];
            hj[c] = (alpha == 1.0) ? pj[c] : alpha * pj[c] + (1.0 - alpha) * wj[o2 + c];
            vi[c] = hi[c] + (fast ? yhi[o2 + c] : yi[o2 + c]);
            vj[c] = hj[c] + (fast ? yhj[o2 + c] : yj[o2 + c]);
          }
          double th = orc_halfspace_project(dp, a, s->d_min, vi, vj, nwi, nwj);
          for (int c = 0; c < dp; ++c) {
            r = fmax(r, fabs(pi[c] - nwi[c]));
            r = fmax(r, fabs(pj[c] - nwj[c]));
            /* dual residual against the copies the x-update used */
            sd = fmax(sd, fabs(nwi[c] - (fast ? whi[o2 + c] : wi[o2 + c])));
            sd = fmax(sd, fabs(nwj[c] - (fast ? whj[o2 + c] : wj[o2 + c])));
            if (fast) {
              yi[o2 + c] = yhi[o2 + c] + hi[c] - nwi[c];
              yj[o2 + c] = yhj[o2 + c] + hj[c] - nwj[c];
              cdu = fmax(cdu, fabs(yi[o2 + c] - yhi[o2 + c]));
              cdu = fmax(cdu, fabs(yj[o2 + c] - yhj[o2 + c]));
            } else {
              yi[o2 + c] += hi[c] - nwi[c];
              yj[o2 + c] += hj[c] - nwj[c];
            }
            wi[o2 + c] = nwi[c];
            wj[o2 + c] = nwj[c];
            dev = fmax(dev, fabs(yi[o2 + c] + th * a[c]));
            dev = fmax(dev, fabs(yj[o2 + c] - th * a[c]));
          }
          res->theta[(size_t)pk * T + t] = th;
        }
      }
    double sres = sc.rho * sd;
    res->r = r;
    res->s = sres;
    res->inv_dev = dev;
    if (res->trace) { res->trace[2 * k] = r; res->trace[2 * k + 1] = sres; }
    if (!isfinite(r) || !isfinite(sres)) { res->status = ORC_NUMERIC; break; }
    if (r <= o->tol && sres <= o->tol) { res->status = ORC_CONVERGED; break; }
    if (fast) {
      /* Goldstein et al. 2014, fast ADMM with restart: combined residual (here
       * in the max norm), Nesterov extrapolation while it falls by eta, else a
       * restart from the previous iterate */
      const double ck = fmax(cdu, sd);
      if (ck < o->restart_eta * c_prev) {
        const double a1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * acc_a * acc_a));
        const double beta = (acc_a - 1.0) / a1;
        for (size_t q = 0; q < PS; ++q) {
          whi[q] = wi[q] + beta * (wi[q] - wpi[q]);
          whj[q] = wj[q] + beta * (wj[q] - wpj[q]);
          yhi[q] = yi[q] + beta * (yi[q] - ypi[q]);
          yhj[q] = yj[q] + beta * (yj[q] - ypj[q]);
        }
        acc_a = a1;
        c_prev = ck;
      } else {
        for (size_t q = 0; q < PS; ++q) {
          whi[q] = wpi[q];
          whj[q] = wpj[q];
          yhi[q] = ypi[q];
          yhj[q] = ypj[q];
        }
        acc_a = 1.0;
        c_prev = c_prev / o->restart_eta;
        res->restarts++;
      }
      for (size_t q = 0; q < PS; ++q) {
        wpi[q] = wi[q];
        wpj[q] = wj[q];
        ypi[q] = yi[q];
        ypj[q] = yj[q];
      }
    }
    /* residual balancing (Boyd et al. 2011, Sec. 3.4.1): raise rho when the
     * primal residual dominates, lower it when the dual one does; the scaled
     * duals y = lambda / rho are rescaled so that lambda is unchanged */
    if (o->adapt_every > 0 && (k + 1) % o->adapt_every == 0) {
      double scale = 1.0;
      if (r > o->adapt_mu * sres) scale = o->adapt_tau;
      else if (sres > o->adapt_mu * r) scale = 1.0 / o->adapt_tau;
      if (scale != 1.0) {
        for (size_t q = 0; q < PS; ++q) {
          yi[q] /= scale;
          yj[q] /= scale;
          yhi[q] /= scale;
          yhj[q] /= scale;
          ypi[q] /= scale;
          ypj[q] /= scale;
        }
        acc_a = 1.0; /* the accelerated iteration starts afresh at the new penalty */
        c_prev = INFINITY;
        sc.rho *= scale;
        res->rho_changes++;
        hom_ok = 0;
      }
    }
  }
  res->rho_final = sc.rho;
  res->as_iters = as_total;
  free(wi); free(wj); free(yi); free(yj); free(pos); free(plist); free(ptab);
  free(whi); free(whj); free(yhi); free(yhj); free(wpi); free(wpj); free(ypi); free(ypj);
  free(h_prev);
  res->homotopy_steps = hom_steps;
  return 0;
}

int orc_admm_batch(const orc_scenario* s, int n_scen, const orc_options* o, orc_result* res,
                   int nthreads) {
  int used = 1;
  orc_options inner = *o;
  inner.nthreads = 0;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
  {
#ifdef _OPENMP
#pragma omp single
    used = omp_get_num_threads();
#endif
#pragma omp for schedule(dynamic, 1)
    for (int k = 0; k < n_scen; ++k) orc_admm(&s[k], &inner, &res[k]);
  }
  return used;
}

/* ------------------------------------------------------------------------- */
/* Global QP of Eq. (1), condensed in all inputs                               */
/* ------------------------------------------------------------------------- */

typedef struct {
  int N, T, nx, nu, dp, P, m, nU, nC;
  double* Phi;   /* [N][T+1][nx][nx]  A_i^t */
  double* G;     /* [N][T][T][nx][nu] G_i[t-1][s] = A_i^{t-1-s} B_i for s < t, else 0 */
  double* H;     /* [nU][nU] */
  double* g;     /* [nU] */
  double* Nc;    /* [nC][nU] constraint rows, c_k(U) = Nc_k' U - bc_k >= 0 */
  double* bc;    /* [nC] */
} global_qp;

static void global_free(global_qp* G) {
  free(G->Phi); free(G->G); free(G->H); free(G->g); free(G->Nc); free(G->bc);
}

static void matmul(int n, int k, int m, const double* X, const double* Y, double* Z) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) {
      double acc = 0.0;
      for (int l = 0; l < k; ++l) acc += X[IDX2(i, l, k)] * Y[IDX2(l, j, m)];
      Z[IDX2(i, j, m)] = acc;
    }
}

/* agent i's blocks: Phi_t [nx][nx] for t = 0..T and G for x_t (t = 1..T) and u_s [nx][nu] */
#define PHI(Q, i, t) ((Q)->Phi + ((size_t)(i) * ((Q)->T + 1) + (t)) * (Q)->nx * (Q)->nx)
#define GM(Q, i, t, s) ((Q)->G + (((size_t)(i) * (Q)->T + (t) - 1) * (Q)->T + (s)) * (Q)->nx * (Q)->nu)

/* Builds prediction matrices, the condensed Hessian/gradient of Eq. (1) (exact
 * objective, written as 1/2 U'HU + g'U + const) and all constraint rows:
 * bounds (agent, t, c; lower then upper) followed by halfspaces (pair, t). */
static int global_build(const orc_scenario* s, global_qp* Q) {
  const int N = s->N, T = s->T, nx = s->nx, nu = s->nu, dp = s->dp;
  Q->N = N; Q->T = T; Q->nx = nx; Q->nu = nu; Q->dp = dp;
  int *plist = NULL, *ptab = NULL;
  Q->P = scen_pairs(s, &plist, &ptab);
  if (Q->P < 0) return -1;
  free(ptab);
  Q->m = T * nu; Q->nU = N * Q->m; Q->nC = 2 * Q->nU + Q->P * T;
  Q->Phi = (double*)calloc((size_t)N * (T + 1) * nx * nx, sizeof(double));
  Q->G = (double*)calloc((size_t)N * T * T * nx * nu, sizeof(double));
  Q->H = (double*)calloc((size_t)Q->nU * Q->nU, sizeof(double));
  Q->g = (double*)calloc((size_t)Q->nU, sizeof(double));
  Q->Nc = (double*)calloc((size_t)Q->nC * Q->nU, sizeof(double));
  Q->bc = (double*)calloc((size_t)Q->nC, sizeof(double));
  if (!Q->Phi || !Q->G || !Q->H || !Q->g || !Q->Nc || !Q->bc) return -1;
  /* per agent: Phi_t = A^t and G[t-1][s] = A^(t-1-s) B, the response of x_t to u_s */
  for (int i = 0; i < N; ++i) {
    for (int r = 0; r < nx; ++r) PHI(Q, i, 0)[IDX2(r, r, nx)] = 1.0;
    for (int t = 1; t <= T; ++t) matmul(nx, nx, nx, agent_A(s, i), PHI(Q, i, t - 1), PHI(Q, i, t));
    for (int t = 1; t <= T; ++t)
      for (int sidx = 0; sidx < t; ++sidx) matmul(nx, nx, nu, PHI(Q, i, t - 1 - sidx), agent_B(s, i), GM(Q, i, t, sidx));
  }
  const int m = Q->m, nU = Q->nU;
  double* xf = (double*)malloc(sizeof(double) * nx);
  for (int i = 0; i < N; ++i) {
    const double* Qi = s->Qd + (size_t)i * nx;
    const double* Qfi = s->Qfd + (size_t)i * nx;
    const double* x0 = s->x_init + (size_t)i * nx;
    const double* xr = s->x_ref + (size_t)i * nx;
    const int off = i * m;
    for (int t = 1; t <= T; ++t) {
      const double* Qt = (t < T) ? Qi : Qfi;
      for (int r = 0; r < nx; ++r) {
        double acc = 0.0;
        for (int c = 0; c < nx; ++c) acc += PHI(Q, i, t)[IDX2(r, c, nx)] * x0[c];
        xf[r] = acc - xr[r];
      }
      /* row r of x_t as a function of U_i: sum_s G[t-1][s][r][:] u_s */
      for (int r = 0; r < nx; ++r) {
        for (int s1 = 0; s1 < t; ++s1)
          for (int c1 = 0; c1 < nu; ++c1) {
            double g1 = GM(Q, i, t, s1)[IDX2(r, c1, nu)];
            if (g1 == 0.0) continue;
            Q->g[off + s1 * nu + c1] += 2.0 * Qt[r] * g1 * xf[r];
            for (int s2 = 0; s2 < t; ++s2)
              for (int c2 = 0; c2 < nu; ++c2) {
                double g2 = GM(Q, i, t, s2)[IDX2(r, c2, nu)];
                Q->H[IDX2(off + s1 * nu + c1, off + s2 * nu + c2, nU)] += 2.0 * Qt[r] * g1 * g2;
              }
          }
      }
    }
    for (int t = 0; t < T; ++t)
      for (int c = 0; c < nu; ++c)
        Q->H[IDX2(off + t * nu + c, off + t * nu + c, nU)] += 2.0 * s->Rd[(size_t)i * nu + c];
  }
  /* bound rows */
  for (int k = 0; k < nU; ++k) {
    int c = k % nu;
    Q->Nc[IDX2(2 * k, k, nU)] = 1.0;
    Q->bc[2 * k] = s->umin[c];
    Q->Nc[IDX2(2 * k + 1, k, nU)] = -1.0;
    Q->bc[2 * k + 1] = -s->umax[c];
  }
  /* halfspace rows: a'(C x_it - C x_jt) >= d */
  int row = 2 * nU;
  for (int pk = 0; pk < Q->P; ++pk) {
      const int i = plist[2 * pk], j = plist[2 * pk + 1];
      for (int t = 1; t <= T; ++t, ++row) {
        const double* a = s->a + ((size_t)pk * T + (t - 1)) * dp;
        double* nr = Q->Nc + (size_t)row * nU;
        double rhs = s->d_min;
        for (int c = 0; c < dp; ++c) {
          double fi = 0.0, fj = 0.0;
          for (int l = 0; l < nx; ++l) {
            fi += PHI(Q, i, t)[IDX2(c, l, nx)] * s->x_init[(size_t)i * nx + l];
            fj += PHI(Q, j, t)[IDX2(c, l, nx)] * s->x_init[(size_t)j * nx + l];
          }
          rhs -= a[c] * (fi - fj);
          for (int s1 = 0; s1 < t; ++s1)
            for (int c1 = 0; c1 < nu; ++c1) {
              nr[i * m + s1 * nu + c1] += a[c] * GM(Q, i, t, s1)[IDX2(c, c1, nu)];
              nr[j * m + s1 * nu + c1] -= a[c] * GM(Q, j, t, s1)[IDX2(c, c1, nu)];
            }
        }
        Q->bc[row] = rhs;
      }
    }
  free(xf);
  free(plist);
  return 0;
}

/* EQP of the condensed global QP with the constraints flagged in Wset held as
 * equalities: [H Nw'; Nw 0][U; om] = [-g; bw]; multipliers mu = -om. */
static int global_eqp(const global_qp* Q, const uint8_t* Wset, double* U, double* mu_all) {
  const int nU = Q->nU, nC = Q->nC;
  int nW = 0;
  for (int k = 0; k < nC; ++k) nW += Wset[k] != 0;
  const int nk = nU + nW;
  double* K = (double*)calloc((size_t)nk * nk, sizeof(double));
  double* b = (double*)calloc((size_t)nk, sizeof(double));
  if (!K || !b) { free(K); free(b); return -1; }
  for (int i = 0; i < nU; ++i) {
    for (int j = 0; j < nU; ++j) K[IDX2(i, j, nk)] = Q->H[IDX2(i, j, nU)];
    b[i] = -Q->g[i];
  }
  int w = 0;
  for (int k = 0; k < nC; ++k) {
    if (!Wset[k]) continue;
    for (int j = 0; j < nU; ++j) {
      K[IDX2(nU + w, j, nk)] = Q->Nc[IDX2(k, j, nU)];
      K[IDX2(j, nU + w, nk)] = Q->Nc[IDX2(k, j, nU)];
    }
    b[nU + w] = Q->bc[k];
    ++w;
  }
  int rc = lu_solve(nk, K, b);
  if (rc == 0) {
    memcpy(U, b, sizeof(double) * nU);
    w = 0;
    for (int k = 0; k < nC; ++k) mu_all[k] = Wset[k] ? -b[nU + (w++)] : 0.0;
  }
  free(K);
  free(b);
  return rc;
}

static void global_outputs(const orc_scenario* s, const global_qp* Q, const double* U, double* X) {
  for (int i = 0; i < s->N; ++i)
    simulate(s->T, s->nx, s->nu, agent_A(s, i), agent_B(s, i), s->x_init + (size_t)i * s->nx, U + (size_t)i * Q->m,
             X + (size_t)i * (s->T + 1) * s->nx);
}

int orc_global_qp(const orc_scenario* s, int as_max, double eps_rel, orc_global_result* res) {
  global_qp Q;
  memset(&Q, 0, sizeof(Q));
  res->status = ORC_NUMERIC;
  res->iters = 0;
  if (global_build(s, &Q) != 0) { global_free(&Q); return -1; }
  const int nU = Q.nU, nC = Q.nC;
  double* U = (double*)calloc(nU, sizeof(double));
  double* Us = (double*)malloc(sizeof(double) * nU);
  double* mu = (double*)calloc(nC, sizeof(double));
  double* ms = (double*)calloc(nC, sizeof(double));
  uint8_t* Wset = (uint8_t*)calloc(nC, 1);
  /* the start U = 0 (the guess trajectories) must be feasible */
  for (int k = 0; k < nC; ++k)
    if (-Q.bc[k] < -1e-9) { res->status = -1; goto out; }
  {
    int need = 1, iters = 0, status = ORC_CONVERGED;
    for (;;) {
      if (need) {
        if (iters >= as_max) { status = ORC_QP_FAIL; break; }
        ++iters;
        if (global_eqp(&Q, Wset, Us, ms) != 0) { status = ORC_NUMERIC; break; }
        double alpha = 1.0;
        int blk = -1;
        for (int k = 0; k < nC; ++k) {
          if (Wset[k]) continue;
          double np = 0.0, cv = -Q.bc[k];
          const double* nr = Q.Nc + (size_t)k * nU;
          for (int j = 0; j < nU; ++j) { np += nr[j] * (Us[j] - U[j]); cv += nr[j] * U[j]; }
          if (np < 0.0) {
            double r = cv / (-np);
            if (r < 0.0) r = 0.0;
            if (r < alpha) { alpha = r; blk = k; }
          }
        }
        if (blk >= 0) {
          for (int j = 0; j < nU; ++j) U[j] += alpha * (Us[j] - U[j]);
          Wset[blk] = 1;
          continue;
        }
        memcpy(U, Us, sizeof(double) * nU);
        memcpy(mu, ms, sizeof(double) * nC);
        need = 0;
      }
      double scale = 1.0;
      for (int k = 0; k < nC; ++k)
        if (Wset[k] && fabs(mu[k]) > scale) scale = fabs(mu[k]);
      double worst = -eps_rel * scale;
      int drop = -1;
      for (int k = 0; k < nC; ++k)
        if (Wset[k] && mu[k] < worst) { worst = mu[k]; drop = k; }
      if (drop >= 0) { Wset[drop] = 0; need = 1; continue; }
      break;
    }
    res->status = status;
    res->iters = iters;
  }
  global_outputs(s, &Q, U, res->X);
  memcpy(res->U, U, sizeof(double) * nU);
  for (int k = 0; k < nU; ++k) {
    res->W[k] = Wset[2 * k] ? 1 : (Wset[2 * k + 1] ? 2 : 0);
    res->mu_u[k] = Wset[2 * k] ? mu[2 * k] : (Wset[2 * k + 1] ? mu[2 * k + 1] : 0.0);
  }
  for (int k = 0; k < Q.P * s->T; ++k) {
    res->act_h[k] = Wset[2 * nU + k];
    res->mu_h[k] = mu[2 * nU + k];
  }
  {
    double obj = 0.0;
    for (int i = 0; i < s->N; ++i) {
      for (int t = 1; t <= s->T; ++t) {
        const double* Qt = (t < s->T) ? s->Qd + (size_t)i * s->nx : s->Qfd + (size_t)i * s->nx;
        for (int r = 0; r < s->nx; ++r) {
          double e = res->X[((size_t)i * (s->T + 1) + t) * s->nx + r] - s->x_ref[(size_t)i * s->nx + r];
          obj += Qt[r] * e * e;
        }
      }
      for (int k = 0; k < Q.m; ++k) {
        double uu = U[(size_t)i * Q.m + k];
        obj += s->Rd[(size_t)i * s->nu + k % s->nu] * uu * uu;
      }
    }
    res->obj = obj;
  }
out:
  free(U); free(Us); free(mu); free(ms); free(Wset);
  global_free(&Q);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Implicit differentiation of the global KKT system at a fixed active set     */
/* ------------------------------------------------------------------------- */

/* Relative size below which an active halfspace row, orthogonalized against
 * the rows already chosen, counts as linearly dependent on them. */
#define ORC_RANK_TOL 1e-10

/* Polished point of the global QP at a fixed active set (bounds W held at
 * their values, halfspaces act_h held as equalities).  The held inputs are
 * substituted, leaving on the free inputs U_F the problem
 *     min 1/2 U_F' H_FF U_F + g_F' U_F   s.t.   G U_F = d
 * with one row of G per active halfspace.  The rows of G may be linearly
 * dependent (several halfspaces through the same agents and steps, or rows
 * whose agents' positions are fixed by held inputs); then the multipliers are
 * not unique and the system may be inconsistent.  The polished point is
 * defined as the minimizer subject to G U_F = d_hat, d_hat the Euclidean
 * projection of d onto the range of G (d_hat = d when consistent), which is
 * unique.  It is computed by a row-pivoted Gram-Schmidt (largest remaining row
 * first) that picks an independent subset B of the rows; the dependent rows
 * are G_D = C G_B with C = G_D G_B' (G_B G_B')^-1; the projection is
 * [y; C y] with (I + C'C) y = d_B + C' d_D; and the EQP
 *     [H_FF G_B'; G_B 0] [U_F; om] = [-g_F; y]
 * is solved by LU.  On return Kf holds that KKT matrix (factor-free copy) for
 * the adjoint solve, Uout the full inputs, mu_all the multipliers of every
 * constraint row (0 for dependent and inactive rows). */
typedef struct {
  int nF, r, m;
  int* free_idx;   /* [nF] */
  int* rows;       /* [m] constraint row of each active halfspace */
  int* basis;      /* [r] indices into rows of the chosen independent subset */
  double* K;       /* [(nF + r)^2] KKT matrix of the reduced EQP */
} reduced_eqp;

static void reduced_free(reduced_eqp* R) {
  free(R->free_idx); free(R->rows); free(R->basis); free(R->K);
}

static int global_eqp_polished(const global_qp* Q, const uint8_t* Wset, double* Uout, double* mu_all,
                               reduced_eqp* R) {
  const int nU = Q->nU, nC = Q->nC;
  memset(R, 0, sizeof(*R));
  int rc = -1;
  /* held inputs at their bound values */
  double* u = (double*)calloc(nU, sizeof(double));
  uint8_t* held = (uint8_t*)calloc(nU, 1);
  R->free_idx = (int*)malloc(sizeof(int) * (nU + 1));
  R->rows = (int*)malloc(sizeof(int) * (nC + 1));
  R->basis = (int*)malloc(sizeof(int) * (nC + 1));
  if (!u || !held || !R->free_idx || !R->rows || !R->basis) goto fail0;
  for (int k = 0; k < nU; ++k) {
    if (Wset[2 * k]) { held[k] = 1; u[k] = Q->bc[2 * k]; }
    else if (Wset[2 * k + 1]) { held[k] = 1; u[k] = -Q->bc[2 * k + 1]; }
    else R->free_idx[R->nF++] = k;
  }
  for (int k = 2 * nU; k < nC; ++k)
    if (Wset[k]) R->rows[R->m++] = k;
  {
    const int nF = R->nF, m = R->m;
    double* G = (double*)calloc((size_t)m * nF + 1, sizeof(double));
    double* d = (double*)calloc((size_t)m + 1, sizeof(double));
    double* V = (double*)calloc((size_t)m * nF + 1, sizeof(double));   /* rows being orthogonalized */
    uint8_t* taken = (uint8_t*)calloc((size_t)m + 1, 1);
    if (!G || !d || !V || !taken) { free(G); free(d); free(V); free(taken); goto fail0; }
    for (int h = 0; h < m; ++h) {
      const double* nr = Q->Nc + (size_t)R->rows[h] * nU;
      double rhs = Q->bc[R->rows[h]];
      for (int j = 0; j < nU; ++j)
        if (held[j]) rhs -= nr[j] * u[j];
      d[h] = rhs;
      for (int f = 0; f < nF; ++f) G[IDX2(h, f, nF)] = nr[R->free_idx[f]];
    }
    memcpy(V, G, sizeof(double) * (size_t)m * nF);
    double maxn = 0.0;
    for (int h = 0; h < m; ++h) {
      double s2 = 0.0;
      for (int f = 0; f < nF; ++f) s2 += G[IDX2(h, f, nF)] * G[IDX2(h, f, nF)];
      if (sqrt(s2) > maxn) maxn = sqrt(s2);
    }
    /* row-pivoted modified Gram-Schmidt */
    for (;;) {
      int best = -1;
      double bn = 0.0;
      for (int h = 0; h < m; ++h) {
        if (taken[h]) continue;
        double s2 = 0.0;
        for (int f = 0; f < nF; ++f) s2 += V[IDX2(h, f, nF)] * V[IDX2(h, f, nF)];
        if (sqrt(s2) > bn) { bn = sqrt(s2); best = h; }
      }
      if (best < 0 || !(bn > ORC_RANK_TOL * maxn)) break;
      taken[best] = 1;
      R->basis[R->r++] = best;
      double* q = V + (size_t)best * nF;
      for (int f = 0; f < nF; ++f) q[f] /= bn;
      for (int h = 0; h < m; ++h) {
        if (taken[h]) continue;
        double dot = 0.0;
        for (int f = 0; f < nF; ++f) dot += V[IDX2(h, f, nF)] * q[f];
        for (int f = 0; f < nF; ++f) V[IDX2(h, f, nF)] -= dot * q[f];
      }
    }
    const int r = R->r, nD = m - r;
    /* consistent right-hand side y of the independent rows */
    double* y = (double*)calloc((size_t)r + 1, sizeof(double));
    for (int b = 0; b < r; ++b) y[b] = d[R->basis[b]];
    if (nD > 0 && r > 0) {
      int* dep = (int*)malloc(sizeof(int) * nD);
      int nd = 0;
      for (int h = 0; h < m; ++h)
        if (!taken[h]) dep[nd++] = h;
      /* Gram matrix M = G_B G_B' and X = M^-1 G_B G_D' (column by column), C = X' */
      double* M = (double*)malloc(sizeof(double) * (size_t)r * r);
      double* Mc = (double*)malloc(sizeof(double) * (size_t)r * r);
      double* Ct = (double*)calloc((size_t)r * nD, sizeof(double));   /* C' [r][nD] */
      double* col = (double*)malloc(sizeof(double) * r);
      for (int a = 0; a < r; ++a)
        for (int b = 0; b < r; ++b) {
          double acc = 0.0;
          for (int f = 0; f < nF; ++f) acc += G[IDX2(R->basis[a], f, nF)] * G[IDX2(R->basis[b], f, nF)];
          M[IDX2(a, b, r)] = acc;
        }
      int ok = 1;
      for (int e = 0; e < nD && ok; ++e) {
        for (int a = 0; a < r; ++a) {
          double acc = 0.0;
          for (int f = 0; f < nF; ++f) acc += G[IDX2(R->basis[a], f, nF)] * G[IDX2(dep[e], f, nF)];
          col[a] = acc;
        }
        memcpy(Mc, M, sizeof(double) * (size_t)r * r);
        if (lu_solve(r, Mc, col) != 0) ok = 0;
        for (int a = 0; a < r; ++a) Ct[IDX2(a, e, nD)] = col[a];
      }
      /* (I + C'C) y = d_B + C' d_D */
      if (ok) {
        for (int a = 0; a < r; ++a)
          for (int b = 0; b < r; ++b) {
            double acc = (a == b) ? 1.0 : 0.0;
            for (int e = 0; e < nD; ++e) acc += Ct[IDX2(a, e, nD)] * Ct[IDX2(b, e, nD)];
            Mc[IDX2(a, b, r)] = acc;
          }
        for (int a = 0; a < r; ++a) {
          double acc = d[R->basis[a]];
          for (int e = 0; e < nD; ++e) acc += Ct[IDX2(a, e, nD)] * d[dep[e]];
          y[a] = acc;
        }
        if (lu_solve(r, Mc, y) != 0) ok = 0;
      }
      free(dep); free(M); free(Mc); free(Ct); free(col);
      if (!ok) { free(G); free(d); free(V); free(taken); free(y); goto fail0; }
    }
    /* reduced EQP */
    const int nk = nF + r;
    R->K = (double*)calloc((size_t)nk * nk + 1, sizeof(double));
    double* K = (double*)malloc(sizeof(double) * ((size_t)nk * nk + 1));
    double* rhs = (double*)calloc((size_t)nk + 1, sizeof(double));
    for (int a = 0; a < nF; ++a) {
      const int ia = R->free_idx[a];
      double gv = Q->g[ia];
      for (int j = 0; j < nU; ++j)
        if (held[j]) gv += Q->H[IDX2(ia, j, nU)] * u[j];
      rhs[a] = -gv;
      for (int b = 0; b < nF; ++b) R->K[IDX2(a, b, nk)] = Q->H[IDX2(ia, R->free_idx[b], nU)];
    }
    for (int b = 0; b < r; ++b) {
      for (int f = 0; f < nF; ++f) {
        R->K[IDX2(nF + b, f, nk)] = G[IDX2(R->basis[b], f, nF)];
        R->K[IDX2(f, nF + b, nk)] = G[IDX2(R->basis[b], f, nF)];
      }
      rhs[nF + b] = y[b];
    }
    memcpy(K, R->K, sizeof(double) * (size_t)nk * nk);
    const int lr = lu_solve(nk, K, rhs);
    if (lr == 0) {
      memcpy(Uout, u, sizeof(double) * nU);
      for (int a = 0; a < nF; ++a) Uout[R->free_idx[a]] = rhs[a];
      for (int k = 0; k < nC; ++k) mu_all[k] = 0.0;
      for (int b = 0; b < r; ++b) mu_all[R->rows[R->basis[b]]] = -rhs[nF + b];
      /* bound multipliers from stationarity H U + g - Nc' mu = 0 on the held inputs */
      for (int j = 0; j < nU; ++j) {
        if (!held[j]) continue;
        double st = Q->g[j];
        for (int l = 0; l < nU; ++l) st += Q->H[IDX2(j, l, nU)] * Uout[l];
        for (int h = 0; h < m; ++h) st -= Q->Nc[IDX2(R->rows[h], j, nU)] * mu_all[R->rows[h]];
        if (Wset[2 * j]) mu_all[2 * j] = st;
        else mu_all[2 * j + 1] = -st;
      }
      rc = 0;
    }
    free(K); free(rhs); free(G); free(d); free(V); free(taken); free(y);
  }
fail0:
  free(u); free(held);
  return rc;
}

int orc_global_gradient(const orc_scenario* s, const uint8_t* act_h, const int8_t* W,
                        const double* targets, double qf_tie, double* X, double* U, double* loss,
                        double* gQ, double* gR, double* gGoal, double* mu_h, double* mu_u, int* n_dependent) {
  global_qp Q;
  memset(&Q, 0, sizeof(Q));
  if (global_build(s, &Q) != 0) { global_free(&Q); return -1; }
  const int N = s->N, T = s->T, nx = s->nx, nu = s->nu, dp = s->dp, m = Q.m, nU = Q.nU, nC = Q.nC;
  uint8_t* Wset = (uint8_t*)calloc(nC, 1);
  double* mu = (double*)calloc(nC, sizeof(double));
  double* dl = (double*)calloc(nU, sizeof(double));
  double* wv = (double*)calloc(nU + nC, sizeof(double));
  double* dH = (double*)malloc(sizeof(double) * (size_t)m * m);
  double* dg = (double*)malloc(sizeof(double) * m);
  reduced_eqp R;
  memset(&R, 0, sizeof(R));
  int rc = 0;
  for (int k = 0; k < nU; ++k) {
    if (W[k] == 1) Wset[2 * k] = 1;
    if (W[k] == 2) Wset[2 * k + 1] = 1;
  }
  for (int k = 0; k < Q.P * T; ++k) Wset[2 * nU + k] = act_h[k] ? 1 : 0;
  /* polished primal solution at this active set */
  if (global_eqp_polished(&Q, Wset, U, mu, &R) != 0) { rc = -2; goto out; }
  global_outputs(s, &Q, U, X);
  if (mu_h)
    for (int k = 0; k < Q.P * T; ++k) mu_h[k] = mu[2 * nU + k];
  if (mu_u)
    for (int k = 0; k < nU; ++k) mu_u[k] = Wset[2 * k] ? mu[2 * k] : (Wset[2 * k + 1] ? mu[2 * k + 1] : 0.0);
  if (n_dependent) *n_dependent = R.m - R.r;
  /* loss and its gradient with respect to U */
  double L = 0.0;
  for (int i = 0; i < N; ++i)
    for (int t = 1; t <= T; ++t)
      for (int c = 0; c < dp; ++c) {
        double e = X[((size_t)i * (T + 1) + t) * nx + c] - targets[((size_t)i * T + (t - 1)) * dp + c];
        L += e * e;
        for (int s1 = 0; s1 < t; ++s1)
          for (int c1 = 0; c1 < nu; ++c1)
            dl[i * m + s1 * nu + c1] +=
                2.0 * e * GM((&Q), i, t, s1)[IDX2(c, c1, nu)];
      }
  *loss = L;
  /* adjoint: [H_FF G_B'; G_B 0] [w_F; nu] = [dl/dU_F; 0] (held inputs: w = 0);
   * the right-hand side of the constraint rows is zero, so any independent
   * subset of the active rows gives the same w */
  {
    const int nk = R.nF + R.r;
    double* K = (double*)malloc(sizeof(double) * ((size_t)nk * nk + 1));
    double* b = (double*)calloc((size_t)nk + 1, sizeof(double));
    memcpy(K, R.K, sizeof(double) * (size_t)nk * nk);
    for (int a = 0; a < R.nF; ++a) b[a] = dl[R.free_idx[a]];
    int lr = lu_solve(nk, K, b);
    if (lr == 0)
      for (int a = 0; a < R.nF; ++a) wv[R.free_idx[a]] = b[a];
    free(K);
    free(b);
    if (lr != 0) { rc = -3; goto out; }
  }
  /* dloss/dparam = -w_U' (dH/dparam U + dg/dparam); only agent i's block depends
   * on agent i's parameters */
  for (int i = 0; i < N; ++i) {
    const double* Ui = U + (size_t)i * m;
    const double* wi = wv + (size_t)i * m;
    const double* x0 = s->x_init + (size_t)i * nx;
    const double* xr = s->x_ref + (size_t)i * nx;
    const double* Qi = s->Qd + (size_t)i * nx;
    /* diag(Q_i)[r], with Qf_i = qf_tie * Q_i */
    for (int r = 0; r < nx; ++r) {
      memset(dH, 0, sizeof(double) * (size_t)m * m);
      memset(dg, 0, sizeof(double) * m);
      for (int t = 1; t <= T; ++t) {
        double wt = (t < T) ? 1.0 : qf_tie;
        double xf = -xr[r];
        for (int l = 0; l < nx; ++l) xf += PHI((&Q), i, t)[IDX2(r, l, nx)] * x0[l];
        for (int s1 = 0; s1 < t; ++s1)
          for (int c1 = 0; c1 < nu; ++c1) {
            double g1 = GM((&Q), i, t, s1)[IDX2(r, c1, nu)];
            dg[s1 * nu + c1] += 2.0 * wt * g1 * xf;
            for (int s2 = 0; s2 < t; ++s2)
              for (int c2 = 0; c2 < nu; ++c2) {
                double g2 = GM((&Q), i, t, s2)[IDX2(r, c2, nu)];
                dH[IDX2(s1 * nu + c1, s2 * nu + c2, m)] += 2.0 * wt * g1 * g2;
              }
          }
      }
      double acc = 0.0;
      for (int a1 = 0; a1 < m; ++a1) {
        double v = dg[a1];
        for (int a2 = 0; a2 < m; ++a2) v += dH[IDX2(a1, a2, m)] * Ui[a2];
        acc += wi[a1] * v;
      }
      gQ[(size_t)i * nx + r] = -acc;
    }
    /* diag(R_i)[c] */
    for (int c = 0; c < nu; ++c) {
      double acc = 0.0;
      for (int t = 0; t < T; ++t) acc += wi[t * nu + c] * 2.0 * Ui[t * nu + c];
      gR[(size_t)i * nu + c] = -acc;
    }
    /* goal x_ref_i[r]: dg = -2 sum_t Q_t[r] G_t[r,:]' */
    for (int r = 0; r < nx; ++r) {
      memset(dg, 0, sizeof(double) * m);
      for (int t = 1; t <= T; ++t) {
        double qt = (t < T) ? Qi[r] : qf_tie * Qi[r];
        for (int s1 = 0; s1 < t; ++s1)
          for (int c1 = 0; c1 < nu; ++c1)
            dg[s1 * nu + c1] -= 2.0 * qt * GM((&Q), i, t, s1)[IDX2(r, c1, nu)];
      }
      double acc = 0.0;
      for (int a1 = 0; a1 < m; ++a1) acc += wi[a1] * dg[a1];
      gGoal[(size_t)i * nx + r] = -acc;
    }
  }
out:
  free(Wset); free(mu); free(dl); free(wv); free(dH); free(dg);
  reduced_free(&R);
  global_free(&Q);
  return rc;
}
