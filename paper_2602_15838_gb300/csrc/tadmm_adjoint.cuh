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
#pragma once

namespace tadmm {

struct BwdScen {
  int64_t psi_off;   // per-agent responses [N][T][DP][T][DP]
  int64_t s_off;     // Schur complement [m][m]
  int64_t v_off;     // vectors [3][m]
  int32_t m;         // active halfspaces
  int32_t pad;
};

template <typename F>
struct BwdDev {
  const BwdScen* bs;
  int32_t* act;              // per scenario at ps_off: active pair-step indices q (t-major)
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
  double theta_eps;
  int64_t kk_stride;         // Tmax * NU
};

// Ordered compaction of the active halfspaces of one scenario (one warp).
template <typename F, int NX, int NU, int DP>
__global__ void k_bwd_count(Dev<F> D, BwdDev<F> B) {
  const int sc = blockIdx.x;
  const ScenMeta s = D.meta[sc];
  const int lane = threadIdx.x;
  const F* th = D.theta + (size_t)(D.cur_lvl[sc] >> 1) * D.tot_ps + s.ps_off;
  for (int i = lane; i < s.N; i += 32) B.amask[s.agent_off + i] = 0ull;
  __syncwarp();
  const int64_t PT = (int64_t)s.P * s.T;
  int count = 0;
  for (int64_t base = 0; base < PT; base += 32) {
    const int64_t q = base + lane;
    const bool on = q < PT && double(th[q]) > B.theta_eps;
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
  const uint16_t* Wm = D.Wm + s.as_off;
  const int32_t* act = B.act + s.ps_off;
  const F* a = D.a + s.ps_off * DP;
  const int32_t* pr = D.pairs + s.pair_off;
  F* psi = B.psi + bs.psi_off;
  F* Sm = B.S + bs.s_off;
  F* rhs = B.vec + bs.v_off;
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
  // 5. factor S and solve for the halfspace multipliers mu
  if (m > 0) cta_cholesky(Sm, m, &s_bad);
  if (tid == 0 && m > 0) chol_solve_serial(Sm, m, rhs);
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

  // 7. adjoint: w0 = H^{-1} dl/dz (homogeneous), S lam = -G w0, w = w0 + Psi G' lam
  F* lamw = rhs + m;
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
  if (tid == 0 && m > 0) chol_solve_serial(Sm, m, lamw);
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
  if (tid == 0) B.bstatus[sc] = s_bad ? ST_NUMERIC : ST_CONVERGED;
}

template <typename F>
__global__ void k_bwd_export_x(const F* Xp, int64_t n, double* out) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    out[k] = double(Xp[k]);
}

}  // namespace tadmm
