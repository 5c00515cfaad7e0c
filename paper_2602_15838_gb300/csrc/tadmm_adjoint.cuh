// Implicit differentiation of the converged problem (K-d).
//
// At the final active set of a solve (inputs held at a bound by the last
// x-update, and halfspaces whose projection step theta exceeds theta_eps), the
// centralized QP of Eq. (1) with linearized halfspaces reduces to an
// equality-constrained QP.  Its KKT system is differentiated implicitly
// (OptNet-style): per agent, a block-tridiagonal LQ problem solved by the
// Riccati recursion of Sec. IV.B on the global Hessian (2Q, 2Q_T, 2R, no ADMM
// penalty); the coupling through the active halfspaces G z = d is eliminated
// with the dense Schur complement S = G Psi G' of the per-agent position
// responses Psi.  The polished primal solution and the adjoint of a loss
// gradient dl/dX follow from two block solves each; the parameter gradients
// are closed forms in the polished solution and the adjoint.
//
// Active rows may be linearly dependent (several halfspaces through the same
// agents and step, or rows whose positions are fixed by inputs held at a
// bound); S is then singular and the multipliers are not unique.  S is
// factored with diagonal pivoting up to its numerical rank, and the
// multipliers are the least-squares solution of S mu = b in the factor's
// range: the polished point then satisfies the active rows with their
// right-hand side projected onto the range of the rows (exactly the rows
// when they are consistent), and the gradient is that of this solution map.
#pragma once

#include <climits>

namespace tadmm {

struct BwdScen {
  int64_t psi_off;   // per-agent responses [N][T][DP][T][DP]
  int64_t s_off;     // Schur complement [m][m], then the normal matrix [m][m]
  int64_t v_off;     // vectors [3][m]
  int32_t m;         // active halfspaces
  int32_t pad;
};

template <typename F>
struct BwdDev {
  const BwdScen* bs;
  int32_t* act;              // per scenario at ps_off: active pair-step indices q (t-major)
  int32_t* piv;              // per scenario at ps_off: pivot order of the Schur factorization
  int32_t* act_cnt;          // [n_scen]
  unsigned long long* amask; // [agents] bit t-1 set when the agent has an active halfspace at t
  F* psi;
  F* kks;                    // [agents][DP][T][NU] affine gains of the in-flight solves
  F* pos0;                   // [agent-steps][DP] base positions, then adjoint base positions
  F* force;                  // [agent-steps][DP] coupling forces G' mu on each agent
  F* S;
  F* vec;
  F* Xp;                     // polished states, caller layout [agent-state][NX]
  F* Up;                     // polished inputs, caller layout [agent-step][NU]
  F* Wx;                     // adjoint states, caller layout
  F* Wu;                     // adjoint inputs, caller layout
  const double* gX;          // dl/dX, caller layout (float64)
  double* gQ;                // [agents][NX]
  double* gQf;               // [agents][NX]
  double* gR;                // [agents][NU]
  double* gGoal;             // [agents][NX]
  int32_t* bstatus;          // [n_scen]
  int32_t* ndep;             // [n_scen] active rows found dependent (m - rank)
  uint8_t* hmask;            // [pair-steps] active halfspaces (scenario layout [T][P] at ps_off)
  uint16_t* Wb;              // [agent-steps] inputs held at a bound (layout of Wm)
  int32_t* pchg;             // [n_scen] polishing: the active set changed in this round
  int32_t adjoint;           // 0: stop after the polished primal point (polishing rounds)
  double kkt_tol;            // polishing: relative tolerance of the KKT conditions
  double theta_eps;
  double rank_tol;           // relative pivot size below which a row counts as dependent
  int64_t kk_stride;         // Tmax * NU
};

// Active set of the last solve's final iterate: halfspaces whose projection
// step theta exceeds theta_eps and the inputs the last x-update held at a
// bound (one CTA per scenario).
template <typename F, int NX, int NU, int DP>
__global__ void k_bwd_init(Dev<F> D, BwdDev<F> B) {
  const int sc = blockIdx.x;
  const ScenMeta s = D.meta[sc];
  const F* th = D.theta + (size_t)(D.cur_lvl[sc] >> 1) * D.tot_ps + s.ps_off;
  const int64_t PT = (int64_t)s.P * s.T, NT = (int64_t)s.N * s.T;
  for (int64_t q = threadIdx.x; q < PT; q += blockDim.x) B.hmask[s.ps_off + q] = double(th[q]) > B.theta_eps ? 1 : 0;
  for (int64_t e = threadIdx.x; e < NT; e += blockDim.x) B.Wb[s.as_off + e] = D.Wm[s.as_off + e];
}

// Ordered compaction of the active halfspaces of one scenario (one warp).
template <typename F, int NX, int NU, int DP>
__global__ void k_bwd_count(Dev<F> D, BwdDev<F> B) {
  const int sc = blockIdx.x;
  const ScenMeta s = D.meta[sc];
  const int lane = threadIdx.x;
  const uint8_t* hm = B.hmask + s.ps_off;
  for (int i = lane; i < s.N; i += 32) B.amask[s.agent_off + i] = 0ull;
  __syncwarp();
  const int64_t PT = (int64_t)s.P * s.T;
  int count = 0;
  for (int64_t base = 0; base < PT; base += 32) {
    const int64_t q = base + lane;
    const bool on = q < PT && hm[q] != 0;
    const unsigned ball = __ballot_sync(0xffffffffu, on);
    if (on) {
      const int pos = count + __popc(ball & ((1u << lane) - 1u));
      B.act[s.ps_off + pos] = (int32_t)q;
      const int tm1 = (int)(q / s.P), pair = (int)(q - (int64_t)tm1 * s.P);
      const int pk = D.pairs[s.pair_off + pair];
      atomicOr(&B.amask[s.agent_off + (pk & 0xFFFF)], 1ull << tm1);
      atomicOr(&B.amask[s.agent_off + (pk >> 16)], 1ull << tm1);
    }
    count += __popc(ball);
  }
  if (lane == 0) B.act_cnt[sc] = count;
}

// Riccati solve of one agent's equality-constrained LQ problem with the cached
// factors of its working set: linear term lin(t, r) on x_t (t = 1..T), initial
// state x0, inputs of the working set at their bounds (at_bounds) or at zero.
// Emits every state through outx(t, x) and every input through outu(t, u).
template <typename F, int NX, int NU, bool DI, class Lin, class OutX, class OutU>
__device__ void lq_solve(const Model<F, NX, NU>& Mo, const F* cache, const uint16_t* Wm, int N, int i, int T,
                         Lin lin, const F (&x0)[NX], bool at_bounds, F* kk, OutX outx, OutU outu) {
  using CL = CacheLayout<NX, NU>;
  constexpr int H = NX / 2;
  auto C = [&](int t, int e) -> F { return cache[((size_t)t * CL::E + e) * N + i]; };
  F pn[NX];
#pragma unroll
  for (int r = 0; r < NX; ++r) pn[r] = lin(T, r);
  for (int t = T - 1; t >= 0; --t) {
    const uint16_t mask = Wm[(size_t)t * N + i];
    F Pcp[NX];
#pragma unroll
    for (int r = 0; r < NX; ++r) Pcp[r] = pn[r];
    if (mask && at_bounds) {
      F cv[NX];
#pragma unroll
      for (int r = 0; r < NX; ++r) {
        F acc = 0;
#pragma unroll
        for (int c = 0; c < NU; ++c) {
          if (mask & (1u << c)) acc = fma(Mo.B[r][c], Mo.umin[c], acc);
          else if (mask & (0x100u << c)) acc = fma(Mo.B[r][c], Mo.umax[c], acc);
        }
        cv[r] = acc;
      }
#pragma unroll
      for (int r = 0; r < NX; ++r) {
        F acc = Pcp[r];
#pragma unroll
        for (int c = 0; c < NX; ++c) acc = fma(C(t + 1, CL::P + r * NX + c), cv[c], acc);
        Pcp[r] = acc;
      }
    }
    F sv[NU], kv[NU], L[NU][NU];
#pragma unroll
    for (int a = 0; a < NU; ++a) {
      F acc = 0;
#pragma unroll
      for (int r = 0; r < NX; ++r) acc = fma(Mo.B[r][a], Pcp[r], acc);
      sv[a] = (mask & (0x101u << a)) ? F(0) : acc;
#pragma unroll
      for (int b = 0; b < NU; ++b) L[a][b] = C(t, CL::L + (b <= a ? a * NU + b : b * NU + a));
    }
    neg_sinv<F, NU>(L, sv, kv);
#pragma unroll
    for (int a = 0; a < NU; ++a) kk[t * NU + a] = kv[a];
    if (t >= 1) {
#pragma unroll
      for (int r = 0; r < NX; ++r) {
        F acc = lin(t, r);
#pragma unroll
        for (int k = 0; k < NX; ++k) acc = fma(Mo.A[k][r], Pcp[k], acc);
#pragma unroll
        for (int k = 0; k < NU; ++k) acc = fma(C(t, CL::K + k * NX + r), sv[k], acc);
        pn[r] = acc;
      }
    }
  }
  F xv[NX];
#pragma unroll
  for (int r = 0; r < NX; ++r) xv[r] = x0[r];
  outx(0, xv);
  for (int t = 0; t < T; ++t) {
    const uint16_t mask = Wm[(size_t)t * N + i];
    F uv[NU];
#pragma unroll
    for (int a = 0; a < NU; ++a) {
      if (mask & (1u << a)) uv[a] = at_bounds ? Mo.umin[a] : F(0);
      else if (mask & (0x100u << a)) uv[a] = at_bounds ? Mo.umax[a] : F(0);
      else {
        F acc = kk[t * NU + a];
#pragma unroll
        for (int c = 0; c < NX; ++c) acc = fma(C(t, CL::K + a * NX + c), xv[c], acc);
        uv[a] = acc;
      }
    }
    F xn[NX];
    if constexpr (DI) {
#pragma unroll
      for (int c = 0; c < H; ++c) {
        xn[c] = fma(Mo.B[0][0], uv[c], fma(Mo.A[0][H], xv[H + c], xv[c]));
        xn[H + c] = fma(Mo.B[H][0], uv[c], xv[H + c]);
      }
    } else {
#pragma unroll
      for (int r = 0; r < NX; ++r) {
        F acc = 0;
#pragma unroll
        for (int c = 0; c < NX; ++c) acc = fma(Mo.A[r][c], xv[c], acc);
#pragma unroll
        for (int c = 0; c < NU; ++c) acc = fma(Mo.B[r][c], uv[c], acc);
        xn[r] = acc;
      }
    }
    outu(t, uv);
    outx(t + 1, xn);
#pragma unroll
    for (int r = 0; r < NX; ++r) xv[r] = xn[r];
  }
}

// In-place Cholesky S = L L' of an m x m SPD matrix in global memory by one
// CTA (right-looking, lower triangle).  Returns 0, or 1 on a non-positive pivot.
template <typename F>
__device__ int cta_cholesky(F* S, int m, int* s_bad) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int k = 0; k < m; ++k) {
    __syncthreads();
    if (tid == 0) {
      const F dkk = S[(size_t)k * m + k];
      if (!(dkk > F(0))) *s_bad = 1;
      S[(size_t)k * m + k] = sqrt_(dkk > F(0) ? dkk : F(1));
    }
    __syncthreads();
    const F lkk = S[(size_t)k * m + k];
    for (int r = k + 1 + tid; r < m; r += nt) S[(size_t)r * m + k] /= lkk;
    __syncthreads();
    const int rem = m - k - 1;
    for (int e = tid; e < rem * rem; e += nt) {
      const int r = k + 1 + e / rem, c = k + 1 + e % rem;
      if (c <= r) S[(size_t)r * m + c] = fma(-S[(size_t)r * m + k], S[(size_t)c * m + k], S[(size_t)r * m + c]);
    }
  }
  __syncthreads();
  return *s_bad;
}

// x = S^{-1} b with the Cholesky factor of cta_cholesky (one thread).
template <typename F>
__device__ void chol_solve_serial(const F* L, int m, F* x) {
  for (int r = 0; r < m; ++r) {
    F v = x[r];
    for (int k = 0; k < r; ++k) v = fma(-L[(size_t)r * m + k], x[k], v);
    x[r] = v / L[(size_t)r * m + r];
  }
  for (int r = m - 1; r >= 0; --r) {
    F v = x[r];
    for (int k = r + 1; k < m; ++k) v = fma(-L[(size_t)k * m + r], x[k], v);
    x[r] = v / L[(size_t)r * m + r];
  }
}

// Rank-revealing Cholesky of the positive semidefinite m x m matrix S (full
// symmetric storage) by one CTA, with diagonal pivoting: step k takes the
// largest remaining diagonal entry (ties to the lowest position) and stops
// when it is not above rank_tol times the largest diagonal entry of S.  The
// pivot order goes to piv; afterwards L[r][c] = S[piv[r] m + piv[c]] for
// r >= c, c < rank is the factor of the permuted matrix restricted to its
// first `rank` columns ([L11; L21]).  Returns the rank (same in every thread).
template <typename F>
__device__ int cta_pivoted_cholesky(F* S, int m, int* piv, F rank_tol) {
  __shared__ F red_v[128];
  __shared__ int red_i[128];
  __shared__ F s_dref;
  __shared__ int s_stop;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int r = tid; r < m; r += nt) piv[r] = r;
  int rank = m;
  for (int k = 0; k < m; ++k) {
    __syncthreads();
    F bv = F(-1);
    int bi = m;
    for (int j = k + tid; j < m; j += nt) {
      const F v = S[(size_t)piv[j] * m + piv[j]];
      if (v > bv) { bv = v; bi = j; }
    }
    red_v[tid] = bv;
    red_i[tid] = bi;
    __syncthreads();
    for (int w = nt / 2; w > 0; w >>= 1) {
      if (tid < w) {
        const F v2 = red_v[tid + w];
        const int i2 = red_i[tid + w];
        if (v2 > red_v[tid] || (v2 == red_v[tid] && i2 < red_i[tid])) {
          red_v[tid] = v2;
          red_i[tid] = i2;
        }
      }
      __syncthreads();
    }
    if (tid == 0) {
      const F v = red_v[0];
      const int j = red_i[0];
      if (k == 0) s_dref = v;
      if (j >= m || !(v > rank_tol * s_dref)) {
        s_stop = 1;
      } else {
        s_stop = 0;
        const int t = piv[k];
        piv[k] = piv[j];
        piv[j] = t;
        S[(size_t)piv[k] * m + piv[k]] = sqrt_(v);
      }
    }
    __syncthreads();
    if (s_stop) {
      rank = k;
      break;
    }
    const int pk = piv[k];
    const F lkk = S[(size_t)pk * m + pk];
    for (int r = k + 1 + tid; r < m; r += nt) S[(size_t)piv[r] * m + pk] /= lkk;
    __syncthreads();
    const int rem = m - k - 1;
    for (int e = tid; e < rem * rem; e += nt) {
      const int pr = piv[k + 1 + e / rem], pc = piv[k + 1 + e % rem];
      S[(size_t)pr * m + pc] = fma(-S[(size_t)pr * m + pk], S[(size_t)pc * m + pk], S[(size_t)pr * m + pc]);
    }
  }
  __syncthreads();
  return rank;
}

// Normal matrix M = L'L (rank x rank) of the rank-deficient factor and its
// Cholesky factor, by one CTA (nothing to do when rank = m).  Sets *s_bad if
// M is not positive definite.
template <typename F>
__device__ void cta_ls_prepare(const F* S, int m, const int* piv, int rank, F* M, int* s_bad) {
  if (rank == m || rank == 0) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < rank * rank; e += nt) {
    const int a = e / rank, b = e % rank;
    if (b > a) continue;
    F acc = 0;
    for (int i = a; i < m; ++i) acc = fma(S[(size_t)piv[i] * m + piv[a]], S[(size_t)piv[i] * m + piv[b]], acc);
    M[(size_t)a * rank + b] = acc;
    M[(size_t)b * rank + a] = acc;
  }
  cta_cholesky(M, rank, s_bad);
}

// Least-squares solution of S lambda = b within the range of the pivoted
// factor (one thread; b is overwritten by lambda, tmp has m entries):
// v minimizes |L v - b_p| (b_p = b in pivot order), lambda_p = [L11^{-T} v; 0].
// For rank = m this is the plain solve L11^{-T} L11^{-1} b_p.
template <typename F>
__device__ void ls_apply_serial(const F* S, int m, const int* piv, int rank, const F* M, F* b, F* tmp) {
  auto L = [&](int r, int c) -> F { return S[(size_t)piv[r] * m + piv[c]]; };
  if (rank == m) {
    for (int r = 0; r < m; ++r) {
      F v = b[piv[r]];
      for (int k = 0; k < r; ++k) v = fma(-L(r, k), tmp[k], v);
      tmp[r] = v / L(r, r);
    }
  } else {
    for (int a = 0; a < rank; ++a) {
      F acc = 0;
      for (int i = a; i < m; ++i) acc = fma(L(i, a), b[piv[i]], acc);
      tmp[a] = acc;
    }
    if (rank > 0) chol_solve_serial(M, rank, tmp);
  }
  for (int r = rank - 1; r >= 0; --r) {
    F v = tmp[r];
    for (int k = r + 1; k < rank; ++k) v = fma(-L(k, r), tmp[k], v);
    tmp[r] = v / L(r, r);
  }
  for (int r = 0; r < m; ++r) b[piv[r]] = r < rank ? tmp[r] : F(0);
}

template <typename F, int NX, int NU, int DP, bool DI>
__global__ void __launch_bounds__(128) k_bwd_main(Dev<F> D, BwdDev<F> B) {
  using CL = CacheLayout<NX, NU>;
  __shared__ Model<F, NX, NU> Mo;
  __shared__ int s_bad;
  load_model<F, NX, NU>(Mo, D.model);
  const int sc = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const ScenMeta s = D.meta[sc];
  const BwdScen bs = B.bs[sc];
  const int N = s.N, T = s.T, P = s.P, m = bs.m;
  if (tid == 0) s_bad = 0;
  __syncthreads();
  F* cache = D.cache + s.xs_off * CL::E;
  const uint16_t* Wm = B.Wb + s.as_off;
  const int32_t* act = B.act + s.ps_off;
  const F* a = D.a + s.ps_off * DP;
  const int32_t* pr = D.pairs + s.pair_off;
  F* psi = B.psi + bs.psi_off;
  F* Sm = B.S + bs.s_off;
  F* Mn = Sm + (size_t)m * m;
  int* piv = B.piv + s.ps_off;
  F* rhs = B.vec + bs.v_off;
  F* tmp = rhs + 2 * m;
  F* pos0 = B.pos0 + s.as_off * DP;
  F* force = B.force + s.as_off * DP;
  auto Q = [&](int i, int r) { return D.Qd[(s.agent_off + i) * NX + r]; };
  auto Qf = [&](int i, int r) { return D.Qfd[(s.agent_off + i) * NX + r]; };
  auto XR = [&](int i, int r) { return D.x_ref[(s.agent_off + i) * NX + r]; };

  // 1. factorization of the global per-agent Hessian with the final working set
  for (int i = tid; i < N; i += nt) {
    F rbar[NU], qbar[NX];
#pragma unroll
    for (int c = 0; c < NU; ++c) rbar[c] = F(2) * D.Rd[(s.agent_off + i) * NU + c];
#pragma unroll
    for (int r = 0; r < NX; ++r) qbar[r] = F(2) * Q(i, r);
    F Pn[NX][NX];
#pragma unroll
    for (int r = 0; r < NX; ++r)
#pragma unroll
      for (int c = 0; c < NX; ++c) {
        Pn[r][c] = (r == c) ? F(2) * Qf(i, r) : F(0);
        cache[((size_t)T * CL::E + CL::P + r * NX + c) * N + i] = Pn[r][c];
      }
    int bad = 0;
    for (int t = T - 1; t >= 0; --t) {
      const uint16_t mask = Wm[(size_t)t * N + i];
      F Pt[NX][NX], K[NU][NX], L[NU][NU];
      auto put = [&](int r, int c, F v) {
        Pt[r][c] = v;
        Pt[c][r] = v;
      };
      auto putB = [](int, int, F) {};
      bad |= factor_stage<F, NX, NU, DI>(agent_model<F, NX, NU>(D, Mo, s, i), Pn, mask, rbar, t >= 1 ? qbar : nullptr, 1, put, putB, K, L);
#pragma unroll
      for (int r = 0; r < NU; ++r) {
#pragma unroll
        for (int c = 0; c < NX; ++c) cache[((size_t)t * CL::E + CL::K + r * NX + c) * N + i] = K[r][c];
#pragma unroll
        for (int c = 0; c <= r; ++c) cache[((size_t)t * CL::E + CL::L + r * NU + c) * N + i] = L[r][c];
      }
      if (t >= 1) {
#pragma unroll
        for (int r = 0; r < NX; ++r)
#pragma unroll
          for (int c = 0; c < NX; ++c) {
            cache[((size_t)t * CL::E + CL::P + r * NX + c) * N + i] = Pt[r][c];
            Pn[r][c] = Pt[r][c];
          }
      }
    }
    if (bad) atomicOr(&s_bad, 1);
    // the forward factor cache no longer matches: force a refactorization on the next solve
    for (int t = 0; t < T; ++t) D.Cm[s.as_off + (size_t)t * N + i] = 0xFFFF;
  }
  __syncthreads();

  const F zero0[NX] = {};
  // 2. position responses to unit forces at the agent's active times
  for (int task = tid; task < N * DP; task += nt) {
    const int i = task / DP, cin = task % DP;
    const unsigned long long msk = B.amask[s.agent_off + i];
    F* kk = B.kks + ((s.agent_off + i) * DP + cin) * (size_t)B.kk_stride;
    for (int tp = 1; tp <= T; ++tp) {
      if (!((msk >> (tp - 1)) & 1ull)) continue;
      auto lin = [&](int t, int r) -> F { return (t == tp && r == cin) ? F(-1) : F(0); };
      auto outx = [&](int t, const F (&x)[NX]) {
        if (t >= 1) {
#pragma unroll
          for (int c = 0; c < DP; ++c)
            psi[((((size_t)i * T + (tp - 1)) * DP + cin) * T + (t - 1)) * DP + c] = x[c];
        }
      };
      auto outu = [&](int, const F (&)[NU]) {};
      lq_solve<F, NX, NU, DI>(agent_model<F, NX, NU>(D, Mo, s, i), cache, Wm, N, i, T, lin, zero0, false, kk, outx, outu);
    }
  }
  __syncthreads();
  // 3. base solution (cost terms only) for the right-hand side of S mu = d - G z0
  for (int i = tid; i < N; i += nt) {
    F x0[NX];
#pragma unroll
    for (int r = 0; r < NX; ++r) x0[r] = D.x_init[(s.agent_off + i) * NX + r];
    F* kk = B.kks + ((s.agent_off + i) * DP) * (size_t)B.kk_stride;
    auto lin = [&](int t, int r) -> F { return (F(-2) * (t < T ? Q(i, r) : Qf(i, r))) * XR(i, r); };
    auto outx = [&](int t, const F (&x)[NX]) {
      if (t >= 1) {
#pragma unroll
        for (int c = 0; c < DP; ++c) pos0[((size_t)i * T + (t - 1)) * DP + c] = x[c];
      }
    };
    auto outu = [&](int, const F (&)[NU]) {};
    lq_solve<F, NX, NU, DI>(agent_model<F, NX, NU>(D, Mo, s, i), cache, Wm, N, i, T, lin, x0, true, kk, outx, outu);
  }
  __syncthreads();

  // 4. Schur complement S_hk = sum over shared agents of sigma sigma a_h' Psi a_k
  auto hs = [&](int h, int& i, int& j, int& tm1, int& pair) {
    const int q = act[h];
    tm1 = q / P;
    pair = q - tm1 * P;
    const int pk = pr[pair];
    i = pk & 0xFFFF;
    j = pk >> 16;
  };
  for (int e = tid; e < m * m; e += nt) {
    const int h = e / m, k = e % m;
    if (k > h) continue;
    int ih, jh, th, ph, ik, jk, tk, pk2;
    hs(h, ih, jh, th, ph);
    hs(k, ik, jk, tk, pk2);
    F acc = 0;
    const int ag[2] = {ih, jh};
    const F sg[2] = {F(1), F(-1)};
    for (int u = 0; u < 2; ++u) {
      const int ma = ag[u];
      F sk = 0;
      if (ma == ik) sk = F(1);
      else if (ma == jk) sk = F(-1);
      else continue;
      F v = 0;
#pragma unroll
      for (int cin = 0; cin < DP; ++cin) {
        const F ak = a[((size_t)tk * DP + cin) * P + pk2];
#pragma unroll
        for (int cout = 0; cout < DP; ++cout) {
          const F ah = a[((size_t)th * DP + cout) * P + ph];
          v = fma(ah * psi[((((size_t)ma * T + tk) * DP + cin) * T + th) * DP + cout], ak, v);
        }
      }
      acc = fma(sg[u] * sk, v, acc);
    }
    Sm[(size_t)h * m + k] = acc;
    Sm[(size_t)k * m + h] = acc;
  }
  for (int h = tid; h < m; h += nt) {
    int i, j, tm1, pair;
    hs(h, i, j, tm1, pair);
    F v = F(s.d);
#pragma unroll
    for (int c = 0; c < DP; ++c)
      v = fma(-a[((size_t)tm1 * DP + c) * P + pair],
              pos0[((size_t)i * T + tm1) * DP + c] - pos0[((size_t)j * T + tm1) * DP + c], v);
    rhs[h] = v;
  }
  // 5. rank-revealing factorization of S; least-squares multipliers mu
  __syncthreads();
  const int rank = m > 0 ? cta_pivoted_cholesky(Sm, m, piv, F(B.rank_tol)) : 0;
  if (m > 0) cta_ls_prepare(Sm, m, piv, rank, Mn, &s_bad);
  __syncthreads();
  if (tid == 0 && m > 0) ls_apply_serial(Sm, m, piv, rank, Mn, rhs, tmp);
  __syncthreads();

  // 6. coupling forces G' mu, polished primal solve
  auto forces = [&](const F* lam) {
    for (int e = tid; e < N * T * DP; e += nt) force[e] = 0;
    __syncthreads();
    if (tid == 0) {
      for (int h = 0; h < m; ++h) {
        int i, j, tm1, pair;
        hs(h, i, j, tm1, pair);
#pragma unroll
        for (int c = 0; c < DP; ++c) {
          const F f = lam[h] * a[((size_t)tm1 * DP + c) * P + pair];
          force[((size_t)i * T + tm1) * DP + c] += f;
          force[((size_t)j * T + tm1) * DP + c] -= f;
        }
      }
    }
    __syncthreads();
  };
  forces(rhs);
  for (int i = tid; i < N; i += nt) {
    F x0[NX];
#pragma unroll
    for (int r = 0; r < NX; ++r) x0[r] = D.x_init[(s.agent_off + i) * NX + r];
    F* kk = B.kks + ((s.agent_off + i) * DP) * (size_t)B.kk_stride;
    auto lin = [&](int t, int r) -> F {
      F v = (F(-2) * (t < T ? Q(i, r) : Qf(i, r))) * XR(i, r);
      if (r < DP) v -= force[((size_t)i * T + (t - 1)) * DP + r];
      return v;
    };
    F* Xp = B.Xp + (s.xs_off + (int64_t)i * (T + 1)) * NX;
    F* Up = B.Up + (s.as_off + (int64_t)i * T) * NU;
    auto outx = [&](int t, const F (&x)[NX]) {
#pragma unroll
      for (int r = 0; r < NX; ++r) Xp[(size_t)t * NX + r] = x[r];
    };
    auto outu = [&](int t, const F (&u)[NU]) {
#pragma unroll
      for (int c = 0; c < NU; ++c) Up[(size_t)t * NU + c] = u[c];
    };
    lq_solve<F, NX, NU, DI>(agent_model<F, NX, NU>(D, Mo, s, i), cache, Wm, N, i, T, lin, x0, true, kk, outx, outu);
  }
  __syncthreads();

  F* lamw = rhs + m;
  if (!B.adjoint) {
    if (tid == 0) {
      bool fin = true;
      for (int h = 0; h < m; ++h) fin = fin && finite_(rhs[h]);
      B.bstatus[sc] = (s_bad || !fin) ? ST_NUMERIC : ST_CONVERGED;
      B.ndep[sc] = m - rank;
    }
    return;
  }
  // 7. adjoint: w0 = H^{-1} dl/dz (homogeneous), S lam = -G w0, w = w0 + Psi G' lam
  for (int i = tid; i < N; i += nt) {
    const double* g = B.gX + (s.xs_off + (int64_t)i * (T + 1)) * NX;
    F* kk = B.kks + ((s.agent_off + i) * DP) * (size_t)B.kk_stride;
    auto lin = [&](int t, int r) -> F { return -F(g[(size_t)t * NX + r]); };
    auto outx = [&](int t, const F (&x)[NX]) {
      if (t >= 1) {
#pragma unroll
        for (int c = 0; c < DP; ++c) pos0[((size_t)i * T + (t - 1)) * DP + c] = x[c];
      }
    };
    auto outu = [&](int, const F (&)[NU]) {};
    lq_solve<F, NX, NU, DI>(agent_model<F, NX, NU>(D, Mo, s, i), cache, Wm, N, i, T, lin, zero0, false, kk, outx, outu);
  }
  __syncthreads();
  for (int h = tid; h < m; h += nt) {
    int i, j, tm1, pair;
    hs(h, i, j, tm1, pair);
    F v = 0;
#pragma unroll
    for (int c = 0; c < DP; ++c)
      v = fma(-a[((size_t)tm1 * DP + c) * P + pair],
              pos0[((size_t)i * T + tm1) * DP + c] - pos0[((size_t)j * T + tm1) * DP + c], v);
    lamw[h] = v;
  }
  __syncthreads();
  if (tid == 0 && m > 0) ls_apply_serial(Sm, m, piv, rank, Mn, lamw, tmp);
  __syncthreads();
  forces(lamw);
  for (int i = tid; i < N; i += nt) {
    const double* g = B.gX + (s.xs_off + (int64_t)i * (T + 1)) * NX;
    F* kk = B.kks + ((s.agent_off + i) * DP) * (size_t)B.kk_stride;
    auto lin = [&](int t, int r) -> F {
      F v = -F(g[(size_t)t * NX + r]);
      if (r < DP) v -= force[((size_t)i * T + (t - 1)) * DP + r];
      return v;
    };
    F* Wx = B.Wx + (s.xs_off + (int64_t)i * (T + 1)) * NX;
    F* Wu = B.Wu + (s.as_off + (int64_t)i * T) * NU;
    auto outx = [&](int t, const F (&x)[NX]) {
#pragma unroll
      for (int r = 0; r < NX; ++r) Wx[(size_t)t * NX + r] = x[r];
    };
    auto outu = [&](int t, const F (&u)[NU]) {
#pragma unroll
      for (int c = 0; c < NU; ++c) Wu[(size_t)t * NU + c] = u[c];
    };
    lq_solve<F, NX, NU, DI>(agent_model<F, NX, NU>(D, Mo, s, i), cache, Wm, N, i, T, lin, zero0, false, kk, outx, outu);
  }
  __syncthreads();

  // 8. gradients: dl/dtheta = -w' (dH/dtheta z + dg/dtheta)
  for (int i = tid; i < N; i += nt) {
    const int64_t ag = s.agent_off + i;
    const F* Xp = B.Xp + (s.xs_off + (int64_t)i * (T + 1)) * NX;
    const F* Up = B.Up + (s.as_off + (int64_t)i * T) * NU;
    const F* Wx = B.Wx + (s.xs_off + (int64_t)i * (T + 1)) * NX;
    const F* Wu = B.Wu + (s.as_off + (int64_t)i * T) * NU;
#pragma unroll
    for (int r = 0; r < NX; ++r) {
      F gq = 0, gqf = 0, gg = 0;
      for (int t = 1; t <= T; ++t) {
        const F w = Wx[(size_t)t * NX + r];
        const F e = Xp[(size_t)t * NX + r] - XR(i, r);
        if (t < T) {
          gq = fma(F(-2) * w, e, gq);
          gg = fma(F(2) * Q(i, r), w, gg);
        } else {
          gqf = fma(F(-2) * w, e, gqf);
          gg = fma(F(2) * Qf(i, r), w, gg);
        }
      }
      if (B.gQ) B.gQ[ag * NX + r] = double(gq);
      if (B.gQf) B.gQf[ag * NX + r] = double(gqf);
      if (B.gGoal) B.gGoal[ag * NX + r] = double(gg);
    }
#pragma unroll
    for (int c = 0; c < NU; ++c) {
      F gr = 0;
      for (int t = 0; t < T; ++t) gr = fma(F(-2) * Wu[(size_t)t * NU + c], Up[(size_t)t * NU + c], gr);
      if (B.gR) B.gR[ag * NU + c] = double(gr);
    }
  }
  if (tid == 0) {
    bool fin = true;
    for (int h = 0; h < m; ++h) fin = fin && finite_(rhs[h]) && finite_(lamw[h]);
    B.bstatus[sc] = (s_bad || !fin) ? ST_NUMERIC : ST_CONVERGED;
    B.ndep[sc] = m - rank;
  }
}

// One round of active-set polishing on the centralized QP (one CTA per
// scenario), after k_bwd_main (adjoint = 0) has formed the polished point of
// the current active set, its halfspace multipliers mu (in the order of the
// active list) and the coupling forces G' mu.  KKT check at that point:
//   - halfspace rows: active ones need mu >= 0, inactive ones a'(p_i - p_j) >= d;
//   - inputs: held ones need a non-negative bound multiplier, from
//     stationarity mu_lower = 2 R u_t + B' lambda_{t+1} (mu_upper its negative)
//     with the costates lambda_t = 2 Q_t (x_t - x_ref) - C' f_t + A' lambda_{t+1}
//     of the global problem (f_t the coupling force), free ones lie in the box.
// One change per round, as in a primal active-set method: the row with the
// most negative multiplier below -kkt_tol * max(1, largest |multiplier|)
// leaves the set; if there is none, the most violated row (halfspace
// violation relative to max(1, d), box violation relative to max(1, |bound|))
// beyond kkt_tol enters it (an input held at the violated bound).  Ties go to
// the lowest index (halfspace rows in active-list or pair-step order first,
// then inputs by agent, step, component).  pchg[sc] = 1 when the set changed.
template <typename F, int NX, int NU, int DP, bool DI>
__global__ void __launch_bounds__(128) k_bwd_polish(Dev<F> D, BwdDev<F> B) {
  __shared__ Model<F, NX, NU> Mo;
  __shared__ unsigned long long s_scale, s_key;
  __shared__ long long s_idx;
  load_model<F, NX, NU>(Mo, D.model);
  const int sc = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const ScenMeta s = D.meta[sc];
  const BwdScen bs = B.bs[sc];
  const int N = s.N, T = s.T, P = s.P, m = bs.m;
  const int32_t* act = B.act + s.ps_off;
  const F* mu = B.vec + bs.v_off;
  const F* a = D.a + s.ps_off * DP;
  const int32_t* pr = D.pairs + s.pair_off;
  const F* force = B.force + s.as_off * DP;
  uint16_t* Wb = B.Wb + s.as_off;
  uint8_t* hm = B.hmask + s.ps_off;
  const int64_t PT = (int64_t)P * T;
  if (tid == 0) {
    s_scale = ord_bits(F(1));
    s_key = ~0ull;
    s_idx = LLONG_MAX;
  }
  __syncthreads();
  // Costates of agent i backwards from lambda_{T+1} = 0; for every input u_{t-1}
  // visit(t-1, c, working-set mask, u, g) with g = 2 R u_{t-1} + B' lambda_t.
  auto sweep = [&](int i, auto&& visit) {
    const Model<F, NX, NU>& Ma = agent_model<F, NX, NU>(D, Mo, s, i);
    const F* Xp = B.Xp + (s.xs_off + (int64_t)i * (T + 1)) * NX;
    const F* Up = B.Up + (s.as_off + (int64_t)i * T) * NU;
    F lam[NX];
#pragma unroll
    for (int r = 0; r < NX; ++r) lam[r] = F(0);
    for (int t = T; t >= 1; --t) {
      F ln[NX];
#pragma unroll
      for (int r = 0; r < NX; ++r) {
        const F q = t < T ? D.Qd[(s.agent_off + i) * NX + r] : D.Qfd[(s.agent_off + i) * NX + r];
        F acc = (F(2) * q) * (Xp[(size_t)t * NX + r] - D.x_ref[(s.agent_off + i) * NX + r]);
        if (r < DP) acc -= force[((size_t)i * T + (t - 1)) * DP + r];
#pragma unroll
        for (int k = 0; k < NX; ++k) acc = fma(Ma.A[k][r], lam[k], acc);
        ln[r] = acc;
      }
      const uint16_t msk = Wb[(size_t)(t - 1) * N + i];
#pragma unroll
      for (int c = 0; c < NU; ++c) {
        const F u = Up[(size_t)(t - 1) * NU + c];
        F g = (F(2) * D.Rd[(s.agent_off + i) * NU + c]) * u;
#pragma unroll
        for (int r = 0; r < NX; ++r) g = fma(Ma.B[r][c], ln[r], g);
        visit(t - 1, c, msk, u, g, Ma);
      }
#pragma unroll
      for (int r = 0; r < NX; ++r) lam[r] = ln[r];
    }
  };
  auto bound_mu = [](uint16_t msk, int c, F g) -> F { return (msk & (1u << c)) ? g : -g; };
  auto held = [](uint16_t msk, int c) -> bool { return (msk & (0x101u << c)) != 0; };
  // largest |multiplier|
  for (int i = tid; i < N; i += nt)
    sweep(i, [&](int, int c, uint16_t msk, F, F g, const Model<F, NX, NU>&) {
      if (held(msk, c)) atomicMax(&s_scale, abs_bits(bound_mu(msk, c, g)));
    });
  for (int h = tid; h < m; h += nt) atomicMax(&s_scale, abs_bits(mu[h]));
  __syncthreads();
  const F tol = F(B.kkt_tol);
  const F mtol = tol * from_bits(s_scale, F(0));
  // 1. the most negative multiplier (smallest order key), then its lowest index
  for (int h = tid; h < m; h += nt)
    if (mu[h] < -mtol) atomicMin(&s_key, mono_key(mu[h]));
  for (int i = tid; i < N; i += nt)
    sweep(i, [&](int, int c, uint16_t msk, F, F g, const Model<F, NX, NU>&) {
      if (held(msk, c) && bound_mu(msk, c, g) < -mtol) atomicMin(&s_key, mono_key(bound_mu(msk, c, g)));
    });
  __syncthreads();
  const unsigned long long kdrop = s_key;
  if (kdrop != ~0ull) {
    for (int h = tid; h < m; h += nt)
      if (mono_key(mu[h]) == kdrop) atomicMin(&s_idx, (long long)h);
    for (int i = tid; i < N; i += nt)
      sweep(i, [&](int t, int c, uint16_t msk, F, F g, const Model<F, NX, NU>&) {
        if (held(msk, c) && mono_key(bound_mu(msk, c, g)) == kdrop)
          atomicMin(&s_idx, (long long)m + ((long long)i * T + t) * NU + c);
      });
    __syncthreads();
    if (tid == 0) {
      const long long e = s_idx;
      if (e < m) {
        hm[act[e]] = 0;
      } else {
        const long long r = e - m;
        const int c = (int)(r % NU), t = (int)((r / NU) % T), i = (int)(r / ((long long)NU * T));
        Wb[(size_t)t * N + i] = (uint16_t)(Wb[(size_t)t * N + i] & ~(0x101u << c));
      }
      B.pchg[sc] = 1;
    }
    return;
  }
  // 2. the most violated row (largest relative violation), then its lowest index
  const F dscale = F(s.d) > F(1) ? F(s.d) : F(1);
  auto slack_rel = [&](int64_t q) -> F {   // a'(p_i - p_j) - d, relative to max(1, d)
    const int tm1 = (int)(q / P), pair = (int)(q - (int64_t)tm1 * P);
    const int pk = pr[pair], i = pk & 0xFFFF, j = pk >> 16;
    const F* xi = B.Xp + (s.xs_off + (int64_t)i * (T + 1) + tm1 + 1) * NX;
    const F* xj = B.Xp + (s.xs_off + (int64_t)j * (T + 1) + tm1 + 1) * NX;
    F v = -F(s.d);
#pragma unroll
    for (int c = 0; c < DP; ++c) v = fma(a[((size_t)tm1 * DP + c) * P + pair], xi[c] - xj[c], v);
    return v / dscale;
  };
  auto box_rel = [](F u, F lo, F hi) -> F {   // distance outside the box, relative; <= 0 inside
    const F sl = fabs_(lo) > F(1) ? fabs_(lo) : F(1), sh = fabs_(hi) > F(1) ? fabs_(hi) : F(1);
    const F vl = (lo - u) / sl, vh = (u - hi) / sh;
    return vl > vh ? vl : vh;
  };
  for (int64_t q = tid; q < PT; q += nt)
    if (!hm[q]) {
      const F v = -slack_rel(q);
      if (v > tol) atomicMin(&s_key, ~mono_key(v));
    }
  for (int i = tid; i < N; i += nt)
    sweep(i, [&](int, int c, uint16_t msk, F u, F, const Model<F, NX, NU>& Ma) {
      if (!held(msk, c)) {
        const F v = box_rel(u, Ma.umin[c], Ma.umax[c]);
        if (v > tol) atomicMin(&s_key, ~mono_key(v));
      }
    });
  __syncthreads();
  const unsigned long long kadd = s_key;
  if (kadd == ~0ull) {
    if (tid == 0) B.pchg[sc] = 0;   // KKT conditions hold
    return;
  }
  for (int64_t q = tid; q < PT; q += nt)
    if (!hm[q] && ~mono_key(-slack_rel(q)) == kadd) atomicMin(&s_idx, (long long)q);
  for (int i = tid; i < N; i += nt)
    sweep(i, [&](int t, int c, uint16_t msk, F u, F, const Model<F, NX, NU>& Ma) {
      if (!held(msk, c) && ~mono_key(box_rel(u, Ma.umin[c], Ma.umax[c])) == kadd)
        atomicMin(&s_idx, PT + ((long long)i * T + t) * NU + c);
    });
  __syncthreads();
  if (tid == 0) {
    const long long e = s_idx;
    if (e < PT) {
      hm[e] = 1;
    } else {
      const long long r = e - PT;
      const int c = (int)(r % NU), t = (int)((r / NU) % T), i = (int)(r / ((long long)NU * T));
      const F u = B.Up[(s.as_off + (int64_t)i * T + t) * NU + c];
      const Model<F, NX, NU>& Ma = agent_model<F, NX, NU>(D, Mo, s, i);
      const uint16_t bit = (u < Ma.umin[c]) ? (uint16_t)(1u << c) : (uint16_t)(0x100u << c);
      Wb[(size_t)t * N + i] = (uint16_t)(Wb[(size_t)t * N + i] | bit);
    }
    B.pchg[sc] = 1;
  }
}

// Active set in the caller's layouts: halfspace flags [pair-step] (pair-major,
// then t) and held inputs [agent][t][nu] (0 free, 1 lower, 2 upper).
template <typename F>
__global__ void k_bwd_export_set(Dev<F> D, BwdDev<F> B, int nu, uint8_t* act_out, int8_t* W_out) {
  const int sc = blockIdx.x;
  const ScenMeta s = D.meta[sc];
  const int64_t PT = (int64_t)s.P * s.T, NT = (int64_t)s.N * s.T;
  if (act_out)
    for (int64_t q = threadIdx.x; q < PT; q += blockDim.x) {
      const int tm1 = (int)(q / s.P), pair = (int)(q - (int64_t)tm1 * s.P);
      act_out[s.ps_off + (int64_t)pair * s.T + tm1] = B.hmask[s.ps_off + q];
    }
  if (W_out)
    for (int64_t e = threadIdx.x; e < NT; e += blockDim.x) {
      const int t = (int)(e / s.N), i = (int)(e - (int64_t)t * s.N);
      const uint16_t msk = B.Wb[s.as_off + e];
      for (int c = 0; c < nu; ++c)
        W_out[(s.as_off + (int64_t)i * s.T + t) * nu + c] = (msk & (1u << c)) ? 1 : ((msk & (0x100u << c)) ? 2 : 0);
    }
}

template <typename F>
__global__ void k_bwd_export_x(const F* Xp, int64_t n, double* out) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    out[k] = double(Xp[k]);
}

}  // namespace tadmm
