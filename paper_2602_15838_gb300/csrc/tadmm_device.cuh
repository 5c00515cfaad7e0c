// Device code of the batched ADMM hot path (arXiv 2602.15838, Sec. III.B-IV).
//
// Three phases per ADMM iteration, written as device functions so that the
// batched persistent kernel (scenario groups, one CTA each) and the per-phase
// kernels of the plain and graph modes share them:
//   x-update  (K-a)  one lane per agent, all lanes of a warp together:
//                    Riccati-factorized primal active set for the
//                    box-constrained local QP (Sec. IV.A-C); stage
//                    refactorizations (and, in the per-phase kernels, EQP
//                    passes) spread over lane groups when few agents need them;
//   pair      (K-b)  per (pair, step): halfspace projection of the consensus
//                    copies, scaled dual update and residuals;
//   gather    (K-b') per (agent, step): the aggregate linear term of the next
//                    x-update, over the agent's pairs in partner order.
//
// Per-scenario internal layouts (agent index fastest, so that consecutive
// threads touch consecutive words):
//   X[lvl]  [T+1][NX][N]   states of the x-update (two levels: p^k and p^{k+1})
//   h       [T][DP][N]     sum over partners of (w - y), t = 1..T
//   U, Us   [T][NU][N]     current active-set iterate and EQP solution
//   Wm, Cm  [T][N]         working-set and cached-factor bit masks
//   cache   [T+1][E][N]    Riccati cache per stage (CacheLayout): P_t, K_t,
//                          S_t^{-1}, k_t, P_{t+1}B, B'p_{t+1}
//   theta   [slot][T][P]   projection steps theta^k (multiplier / rho), three
//                          slots rotating with k mod 3
//   a       [T][DP][P]     halfspace normals
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tadmm_df64.cuh"

#include <type_traits>

namespace tadmm {

enum { ST_CONVERGED = 0, ST_NOT_CONVERGED = 1, ST_QP_FAIL = 2, ST_NUMERIC = 3 };
enum { START_COLD = 0, START_HOT = 1, START_TURBO = 2, START_HOMOTOPY = 3 };
enum { QP_COLD = 0, QP_LQR = 1, QP_GIVEN = 2 };

struct ScenMeta {
  int32_t N, T, P;
  int32_t sparse;     // 1: listed pairs (per-agent adjacency), 0: all pairs
  int64_t agent_off;  // first agent of the scenario (sum of N)
  int64_t as_off;     // agent-step offset (sum of N*T)
  int64_t ps_off;     // pair-step offset (sum of P*T)
  int64_t xs_off;     // agent-state offset (sum of N*(T+1))
  int64_t pair_off;   // pair offset (sum of P)
  double d, rho;
};

template <typename F>
struct Dev {
  const ScenMeta* meta;
  const int32_t* order;   // scenario processing order (largest work first)
  const int32_t* pairs;   // [sum P] packed i | j << 16 (i < j)
  const F* model;         // A [NX*NX], B [NX*NU], umin [NU], umax [NU]
  const F* Qd;            // [agents][NX]
  const F* Rd;            // [agents][NU]
  const F* Qfd;           // [agents][NX]
  const F* x_init;        // [agents][NX]
  const F* x_ref;         // [agents][NX]
  const F* a;             // per scenario [T][DP][P] at ps_off*DP
  const F* w0;            // per scenario [T][DP][N] at as_off*DP
  F* theta;               // slot l (0..2) at l*tot_ps, per scenario [T][P] at ps_off
  F* X;                   // level l at l*tot_xs*NX, per scenario [T+1][NX][N] at xs_off*NX
  F* h;                   // per scenario [T][DP][N] at as_off*DP
  F* U;                   // per scenario [T][NU][N] at as_off*NU
  F* Us;
  uint16_t* Wm;           // per scenario [T][N] at as_off
  uint16_t* Cm;
  F* cache;               // per scenario [T+1][E][N] at xs_off*E
  int64_t tot_ps, tot_xs;
  int32_t n_scen;
  int32_t* status;        // [n_scen]
  int32_t* iters;         // [n_scen]
  int32_t* cur_lvl;       // [n_scen] X level (bit 0) and theta slot (bits 1-2) of the final iterate
  double* res;            // [n_scen][2]
  unsigned long long* eqp;   // [n_scen]
  unsigned long long* fact;  // [n_scen]
  int32_t* queue;            // work-queue head of the persistent kernel
  const int32_t* goff;       // [n_groups + 1] member offsets of the scenario groups
  const int32_t* gmem;       // [n_scen] member scenario ids, group by group
  int32_t n_groups;
  double tol;
  int32_t max_iter;
  int32_t sm_pairs;          // pairs per step that fit the fused pair/gather staging (0: unfused)
  int32_t start_mode;
  int32_t as_max;            // 0: 10*T*NU + 10
  double eps_rel;
  int32_t single_as_group;   // 1: a lone scenario of at most 32 agents also runs the group path
  int32_t coop;              // 1: refactorizations may be spread over lane groups
  int32_t adapt_every;       // residual balancing of rho every adapt_every iterations (0: off)
  double adapt_mu, adapt_tau;
  int32_t relax;             // 1: over-relaxed consensus/dual update with factor alpha (group path)
  double alpha;
  F* phi;                    // [tot_ps] pair part phi of the consensus copies w = s +/- phi a
  F* sx;                     // [tot_as][dp] agent part s of the consensus copies
  const F* models;           // heterogeneous agents: [agents] Model (A, B, umin, umax), or nullptr
  double* rho_out;           // [n_scen] final rho (batched mode), or nullptr
  int32_t* rho_chg;          // [n_scen] number of rho changes
  const int32_t* deg;        // [agents] consensus copies n_c of each agent (its pairs)
  const int32_t* adj_ptr;    // [agents + 1] listed-pair adjacency of sparse scenarios
  const int32_t* adj;        // scenario-local pair index, bit 31 set when the agent is second
  // homotopy hot start (per-phase kernels): per scenario at as_off
  F* hprev;                  // [T][DP][N] coupling term of the agent's previous x-update
  F* mu;                     // [T][NU][N] bound multipliers of the previous x-update's optimum
  F* dmu;                    // [T][NU][N] their direction along the homotopy segment
};

// Per-stage factor cache of one agent (stage t):
//   P   P_t (NX x NX)             K   feedback K_t (NU x NX)
//   L   S_t^{-1}, lower triangle  k   feedforward k_t (NU)
//   PB  P_{t+1} B (NX x NU)       bp  B' p_{t+1} (NU), written by the backward
//                                     pass where the stage holds fixed inputs
template <int NX, int NU>
struct CacheLayout {
  static constexpr int P = 0;
  static constexpr int K = NX * NX;
  static constexpr int L = K + NU * NX;   // S^{-1}, lower triangle (row-major NU x NU slots)
  static constexpr int k = L + NU * NU;
  static constexpr int PB = k + NU;
  static constexpr int bp = PB + NX * NU;
  static constexpr int E = bp + NU;
};

constexpr int kStageBatch = 4;  // stages whose operands the active-set bookkeeping loads ahead

template <typename F, int NX, int NU>
struct Model {
  F A[NX][NX];
  F B[NX][NU];
  F umin[NU];
  F umax[NU];
};

template <typename F, int NX, int NU>
__device__ __forceinline__ void load_model(Model<F, NX, NU>& M, const F* src) {
  for (int e = threadIdx.x; e < NX * NX + NX * NU + 2 * NU; e += blockDim.x) {
    if (e < NX * NX) (&M.A[0][0])[e] = src[e];
    else if (e < NX * NX + NX * NU) (&M.B[0][0])[e - NX * NX] = src[e];
    else if (e < NX * NX + NX * NU + NU) M.umin[e - NX * NX - NX * NU] = src[e];
    else M.umax[e - NX * NX - NX * NU - NU] = src[e];
  }
}

// Non-negative floating values ordered through their bit patterns, so that
// maxima run on the integer pipe (NaN sorts above +inf and survives a max).
__device__ __forceinline__ unsigned long long ord_bits(double v) {
  return (unsigned long long)__double_as_longlong(v);
}
__device__ __forceinline__ unsigned long long ord_bits(float v) {
  return (unsigned long long)(unsigned int)__float_as_int(v);
}
__device__ __forceinline__ double from_bits(unsigned long long b, double) {
  return __longlong_as_double((long long)b);
}
__device__ __forceinline__ float from_bits(unsigned long long b, float) {
  return __int_as_float((int)(unsigned int)b);
}
__device__ __forceinline__ double fabs_(double v) { return fabs(v); }
__device__ __forceinline__ float fabs_(float v) { return fabsf(v); }
__device__ __forceinline__ double sqrt_(double v) { return sqrt(v); }
__device__ __forceinline__ float sqrt_(float v) { return sqrtf(v); }

// |v| as a bit-ordered key (sign bit cleared on the integer pipe).
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ unsigned long long abs_bits(float v) {
  return (unsigned long long)((unsigned int)__float_as_int(v) & 0x7FFFFFFFu);
}
// Order-preserving integer key of a floating value (-0 sorts just below +0),
// so that range checks run on the integer pipe.
__device__ __forceinline__ unsigned long long mono_key(double v) {
  const long long b = __double_as_longlong(v);
  return (unsigned long long)(b ^ ((b >> 63) | (long long)0x8000000000000000ull));
}
__device__ __forceinline__ unsigned long long mono_key(float v) {
  const int b = __float_as_int(v);
  return (unsigned long long)(unsigned int)(b ^ ((b >> 31) | (int)0x80000000u));
}
__device__ __forceinline__ bool sign_set(double v) { return __double_as_longlong(v) < 0; }
__device__ __forceinline__ bool sign_set(float v) { return __float_as_int(v) < 0; }
// NaN test on an abs_bits key.
__device__ __forceinline__ bool nan_key(unsigned long long ab, double) { return ab > 0x7FF0000000000000ull; }
__device__ __forceinline__ bool nan_key(unsigned long long ab, float) { return ab > 0x7F800000ull; }

__device__ __forceinline__ int pair_index(int N, int i, int j) {  // i < j
  return i * N - (i * (i + 1)) / 2 + (j - i - 1);
}

// Consensus copies n_c of agent i: its number of coupled pairs.
template <typename F>
__device__ __forceinline__ int agent_nc(const Dev<F>& D, const ScenMeta& s, int i) {
  return s.sparse ? D.deg[s.agent_off + i] : s.N - 1;
}

// Calls ea(pair, first) for agent i's pairs in increasing partner order (all
// pairs, or the listed ones); `pair` is the scenario-local pair index and
// `first` tells whether i is the pair's first agent.
template <typename F, class EA>
__device__ __forceinline__ void for_partners(const Dev<F>& D, const ScenMeta& s, int i, EA&& ea) {
  if (s.sparse) {
    const int64_t ga = s.agent_off + i;
    const int e1 = D.adj_ptr[ga + 1];
    for (int e = D.adj_ptr[ga]; e < e1; ++e) {
      const uint32_t ent = (uint32_t)D.adj[e];
      ea((int)(ent & 0x7FFFFFFFu), (ent >> 31) == 0u);
    }
  } else {
    const int N = s.N;
    for (int j = 0; j < N; ++j) {
      if (j == i) continue;
      const bool first = i < j;
      ea(first ? pair_index(N, i, j) : pair_index(N, j, i), first);
    }
  }
}


// ---------------------------------------------------------------------------
// K-a: per-agent x-update
// ---------------------------------------------------------------------------

// Result of one equality-constrained solve (EQP) with the working set held at
// its bounds, fused with the ratio test and the multiplier scan.
template <typename F>
struct EqpScan {
  F anum, aden;   // blocking step length as anum / aden (aden > 0); 1/1 = full step
  int blk;        // index t*NU + c of the blocking input, -1 if none
  int bside;      // 1 lower, 2 upper
  F worst;        // most negative multiplier over the working set (0 if none)
  int widx;       // its index, -1 if none
  F scale;        // max(1, max |mu| over the working set)
  int bad;        // non-positive pivot or non-finite value
  int out;        // some free input of the EQP solution left the box
};

// Per-agent constants of the local QP used at every stage, kept in shared
// memory (one column per thread, stride = threads of the CTA) rather than in
// registers.  The terminal-stage terms and x_0 are read from global memory.
template <int NX, int NU>
struct AgentConst {
  static constexpr int QB = 0;             // Hessian diagonal of x_t, t < T
  static constexpr int QL = NX;            // -2 Q x_ref
  static constexpr int RB = 2 * NX;        // Hessian diagonal of u_t
  static constexpr int RHO = 2 * NX + NU;  // penalty parameter
  static constexpr int KC = 2 * NX + NU + 1;
};

// Pieces of the linear term q_t = -2 Q_t x_ref - rho C' h_t, shared by every
// code path that forms it so that all form it with the same operations.
template <typename F>
__device__ __forceinline__ F lin_term(F base, F rho, F hr) { return fma(-rho, hr, base); }
template <typename F>
__device__ __forceinline__ F terminal_lin(F qf, F xr) { return (F(-2) * qf) * xr; }

template <typename F, int NX, int NU, int DP>
struct AgentCtx {
  const Model<F, NX, NU>* M;
  int N, T, i;
  F* cache;          // scenario base
  uint16_t* Wm;      // scenario base
  uint16_t* Cm;
  F* U;
  F* Us;
  F* Xo;             // output level, scenario base
  const F* h;        // scenario base
  const F* kc;       // this thread's constants (AgentConst layout), stride ks
  int ks;
  const F* qf;       // the agent's rows of Qf, x_ref and x_init
  const F* xr;
  const F* xi;
  int coop;          // cooperative refactorization allowed (uniform over the warp)
  int nc;            // consensus copies of the agent (its number of pairs)

  __device__ __forceinline__ F k(int e) const { return kc[e * ks]; }

  // 32-bit indices within the scenario (the host rejects scenarios whose
  // per-stage arrays would need more than 2^31 elements)
  __device__ __forceinline__ F& C(int t, int e) const {
    return cache[(t * CacheLayout<NX, NU>::E + e) * N + i];
  }
  __device__ __forceinline__ uint16_t& W(int t) const { return Wm[t * N + i]; }
  __device__ __forceinline__ uint16_t& CM(int t) const { return Cm[t * N + i]; }
  __device__ __forceinline__ F& u(int t, int c) const { return U[(t * NU + c) * N + i]; }
  __device__ __forceinline__ F& us(int t, int c) const { return Us[(t * NU + c) * N + i]; }
  __device__ __forceinline__ F& x(int t, int r) const { return Xo[(t * NX + r) * N + i]; }
  // Hessian diagonal of x_T
  __device__ __forceinline__ F qbarT(int r) const {
    return F(2) * qf[r] + (r < DP ? k(AgentConst<NX, NU>::RHO) * F(nc) : F(0));
  }
  // h_t component r (r < DP) of stage t = 1..T
  __device__ __forceinline__ F hv(int t, int r) const { return h[((t - 1) * DP + r) * N + i]; }
  // linear term of x_t, t < T, from a loaded h_t component
  __device__ __forceinline__ F q_h(int r, F hr) const {
    using AC = AgentConst<NX, NU>;
    F v = k(AC::QL + r);
    if (r < DP) v = lin_term(v, k(AC::RHO), hr);
    return v;
  }
  // linear term of x_t (t = 1..T): -2 Q_t x_ref - rho C' h_t
  __device__ __forceinline__ F q(int t, int r) const {
    using AC = AgentConst<NX, NU>;
    F v = (t < T) ? k(AC::QL + r) : terminal_lin(qf[r], xr[r]);
    if (r < DP) v = lin_term(v, k(AC::RHO), h[((size_t)(t - 1) * DP + r) * N + i]);
    return v;
  }
};

// Factorization of one stage with inputs in `mask` fixed (Riccati backward
// recursion of Sec. IV.B restricted to the free inputs):
//   S = Rbar + B'P B, M = B'P A (fixed rows/cols replaced by identity / zero),
//   K = -S^{-1} M, P_t = Qbar_t + A'P A + M'K; L receives S^{-1}.
// DI: A = [[I, dt I], [0, I]], B = [[b1 I], [b2 I]] (double integrator, checked
// exactly on the host); the products skip the structural zeros and ones but
// accumulate the remaining terms in the order of the dense loops.
// Inverse of the symmetric NU x NU matrix S (NU = 2 or 3) by its adjugate;
// returns 1 unless S is positive definite (Sylvester's criterion: positive
// leading principal minors).  Si receives the full symmetric inverse.
template <typename F, int NU>
__device__ __forceinline__ int sym_inverse(const F (&S)[NU][NU], F (&Si)[NU][NU]) {
  static_assert(NU == 2 || NU == 3, "input dimension 2 or 3");
  if constexpr (NU == 2) {
    const F det = fma(S[0][0], S[1][1], -(S[0][1] * S[0][1]));
    const int bad = !(S[0][0] > F(0)) || !(det > F(0));
    const F id = F(1) / det;
    Si[0][0] = S[1][1] * id;
    Si[1][1] = S[0][0] * id;
    Si[0][1] = Si[1][0] = -(S[0][1] * id);
    return bad;
  } else {
    const F c00 = fma(S[1][1], S[2][2], -(S[1][2] * S[1][2]));
    const F c01 = fma(S[0][2], S[1][2], -(S[0][1] * S[2][2]));
    const F c02 = fma(S[0][1], S[1][2], -(S[0][2] * S[1][1]));
    const F c11 = fma(S[0][0], S[2][2], -(S[0][2] * S[0][2]));
    const F c12 = fma(S[0][1], S[0][2], -(S[0][0] * S[1][2]));
    const F c22 = fma(S[0][0], S[1][1], -(S[0][1] * S[0][1]));
    const F det = fma(S[0][2], c02, fma(S[0][1], c01, S[0][0] * c00));
    const int bad = !(S[0][0] > F(0)) || !(c22 > F(0)) || !(det > F(0));
    const F id = F(1) / det;
    Si[0][0] = c00 * id;
    Si[1][1] = c11 * id;
    Si[2][2] = c22 * id;
    Si[0][1] = Si[1][0] = c01 * id;
    Si[0][2] = Si[2][0] = c02 * id;
    Si[1][2] = Si[2][1] = c12 * id;
    return bad;
  }
}

// out = -S^{-1} v with the symmetric inverse Si.
template <typename F, int NU>
__device__ __forceinline__ void neg_sinv(const F (&Si)[NU][NU], const F (&v)[NU], F (&out)[NU]) {
#pragma unroll
  for (int a = 0; a < NU; ++a) {
    F acc = Si[a][0] * v[0];
#pragma unroll
    for (int b = 1; b < NU; ++b) acc = fma(Si[a][b], v[b], acc);
    out[a] = -acc;
  }
}

// P_t entry (r, c), r <= c, is handed to put(r, c, value) as soon as it is
// formed, and entry (r, a) of P_{t+1} B to putB(r, a, value).
template <typename F, int NX, int NU, bool DI, class PutP, class PutB>
__device__ __forceinline__ int factor_stage(const Model<F, NX, NU>& Mo, const F (&Pn)[NX][NX],
                                            uint16_t mask, const F* rbar, const F* qdiag, int ks,
                                            PutP&& put, PutB&& putB, F (&K)[NU][NX], F (&L)[NU][NU]) {
  constexpr int H = NX / 2;
  F PA[NX][NX], PB[NX][NU];
#pragma unroll
  for (int r = 0; r < NX; ++r) {
    if constexpr (DI) {
      const F dt = Mo.A[0][H], b1 = Mo.B[0][0], b2 = Mo.B[H][0];
#pragma unroll
      for (int c = 0; c < H; ++c) {
        PA[r][c] = Pn[r][c];
        PA[r][H + c] = fma(Pn[r][H + c], F(1), Pn[r][c] * dt);
        PB[r][c] = fma(Pn[r][H + c], b2, Pn[r][c] * b1);
      }
    } else {
#pragma unroll
      for (int c = 0; c < NX; ++c) {
        F acc = 0;
#pragma unroll
        for (int k = 0; k < NX; ++k) acc = fma(Pn[r][k], Mo.A[k][c], acc);
        PA[r][c] = acc;
      }
#pragma unroll
      for (int c = 0; c < NU; ++c) {
        F acc = 0;
#pragma unroll
        for (int k = 0; k < NX; ++k) acc = fma(Pn[r][k], Mo.B[k][c], acc);
        PB[r][c] = acc;
      }
    }
  }
#pragma unroll
  for (int r = 0; r < NX; ++r)
#pragma unroll
    for (int c = 0; c < NU; ++c) putB(r, c, PB[r][c]);
  F S[NU][NU], Mm[NU][NX];
#pragma unroll
  for (int a = 0; a < NU; ++a) {
    const bool fa = (mask >> a) & 0x101;
#pragma unroll
    for (int b = 0; b < NU; ++b) {
      const bool fb = (mask >> b) & 0x101;
      F acc = (a == b) ? rbar[a * ks] : F(0);
      if constexpr (DI) {
        acc = fma(Mo.B[0][0], PB[a][b], acc);
        acc = fma(Mo.B[H][0], PB[H + a][b], acc);
      } else {
#pragma unroll
        for (int r = 0; r < NX; ++r) acc = fma(Mo.B[r][a], PB[r][b], acc);
      }
      S[a][b] = (fa || fb) ? F(a == b ? 1 : 0) : acc;
    }
#pragma unroll
    for (int c = 0; c < NX; ++c) {
      F acc = 0;
      if constexpr (DI) {
        acc = fma(Mo.B[0][0], PA[a][c], acc);
        acc = fma(Mo.B[H][0], PA[H + a][c], acc);
      } else {
#pragma unroll
        for (int r = 0; r < NX; ++r) acc = fma(Mo.B[r][a], PA[r][c], acc);
      }
      Mm[a][c] = fa ? F(0) : acc;
    }
  }
  // S^{-1} and K = -S^{-1} M, column by column
  const int bad = sym_inverse<F, NU>(S, L);
#pragma unroll
  for (int c = 0; c < NX; ++c) {
    F mc[NU], kc[NU];
#pragma unroll
    for (int r = 0; r < NU; ++r) mc[r] = Mm[r][c];
    neg_sinv<F, NU>(L, mc, kc);
#pragma unroll
    for (int r = 0; r < NU; ++r) K[r][c] = kc[r];
  }
  if (qdiag != nullptr) {
    // P_t = Qbar_t + A'(P A) + M'K, upper triangle mirrored
#pragma unroll
    for (int r = 0; r < NX; ++r) {
#pragma unroll
      for (int c = r; c < NX; ++c) {
        F acc = (r == c) ? qdiag[r * ks] : F(0);
        if constexpr (DI) {
          if (r < H) {
            acc = acc + PA[r][c];
          } else {
            acc = fma(Mo.A[0][H], PA[r - H][c], acc);
            acc = acc + PA[r][c];
          }
        } else {
#pragma unroll
          for (int k = 0; k < NX; ++k) acc = fma(Mo.A[k][r], PA[k][c], acc);
        }
#pragma unroll
        for (int k = 0; k < NU; ++k) acc = fma(Mm[k][r], K[k][c], acc);
        put(r, c, acc);
      }
    }
  }
  return bad;
}

// ---------------------------------------------------------------------------
// Stage factorizations of a warp's agents (the refactorization part of the
// Riccati backward recursion, Sec. IV.B), taken before an EQP pass.  Every
// lane of the warp calls this together; `own` marks the lanes whose agent
// needs stages dirty..0 refactored.  When few agents need it, the work of each
// agent's stage is spread over a group of lanes (one lane per row of P): the
// FP64 pipe costs the warp the same per instruction whatever the number of
// active lanes, so a refactorization that serves a handful of agents is
// otherwise paid at full price.  Each value is formed by the same operations,
// in the same order, as in factor_stage, so both forms give identical bits.
// ---------------------------------------------------------------------------
template <int NX>
struct CoopShape {
  static constexpr int GS = NX <= 4 ? 4 : 8;      // lanes per agent group
  static constexpr int NG = 32 / GS;               // groups per warp
  static constexpr int MAXOWN = NX <= 4 ? 16 : 16; // largest owner count taken cooperatively
};

template <typename F>
__device__ __forceinline__ F shfl_f(F v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// v[idx] for a lane-dependent idx without local-memory indexing.
template <typename F, int N>
__device__ __forceinline__ F pick(const F (&v)[N], int idx) {
  F r = v[0];
#pragma unroll
  for (int c = 1; c < N; ++c)
    if (idx == c) r = v[c];
  return r;
}

template <typename F, int NX, int NU, int DP, bool DI>
__device__ void refactor_sweep(const AgentCtx<F, NX, NU, DP>& A, bool own, int dirty, unsigned long long& nfact,
                               int& bad_out) {
  using CL = CacheLayout<NX, NU>;
  using AC = AgentConst<NX, NU>;
  constexpr unsigned FULL = 0xffffffffu;
  const unsigned owners = __ballot_sync(FULL, own && dirty >= 0);
  if (!owners) return;
  const int lane = threadIdx.x & 31;
  const bool mine = own && dirty >= 0;
  if (mine && dirty >= A.T - 1) {
    // P_T = Qbar_T
#pragma unroll
    for (int r = 0; r < NX; ++r)
#pragma unroll
      for (int c = 0; c < NX; ++c) A.C(A.T, CL::P + r * NX + c) = (r == c) ? A.qbarT(r) : F(0);
  }
  if (mine) nfact += (unsigned long long)(dirty + 1);
  __syncwarp();
  const int n = __popc(owners);
  constexpr bool coop_type = std::is_same<F, double>::value || std::is_same<F, float>::value;
  if (!(DI && coop_type) || n > CoopShape<NX>::MAXOWN || !A.coop) {
    // one lane per agent
    const int maxd = __reduce_max_sync(FULL, mine ? dirty : -1);
    __syncwarp();
    for (int t = maxd; t >= 0; --t) {
      if (mine && t <= dirty) {
        const uint16_t mask = A.W(t);
        F Pn[NX][NX], K[NU][NX], L[NU][NU];
#pragma unroll
        for (int r = 0; r < NX; ++r)
#pragma unroll
          for (int c = 0; c < NX; ++c) Pn[r][c] = A.C(t + 1, CL::P + r * NX + c);
        auto put = [&](int r, int c, F v) {
          A.C(t, CL::P + r * NX + c) = v;
          if (c != r) A.C(t, CL::P + c * NX + r) = v;
        };
        auto putB = [&](int r, int a, F v) { A.C(t, CL::PB + r * NU + a) = v; };
        bad_out |= factor_stage<F, NX, NU, DI>(*A.M, Pn, mask, A.kc + AC::RB * A.ks,
                                               t >= 1 ? A.kc + AC::QB * A.ks : nullptr, A.ks, put, putB, K, L);
#pragma unroll
        for (int a = 0; a < NU; ++a) {
#pragma unroll
          for (int c = 0; c < NX; ++c) A.C(t, CL::K + a * NX + c) = K[a][c];
#pragma unroll
          for (int b = 0; b <= a; ++b) A.C(t, CL::L + a * NU + b) = L[a][b];
        }
        A.CM(t) = mask;
      }
    }
    __syncwarp();
    return;
  }
  if constexpr (DI && coop_type) {
    constexpr int GS = CoopShape<NX>::GS, NG = CoopShape<NX>::NG, H = NX / 2;
    static_assert(NU == H, "double integrator: one input per position axis");
    const Model<F, NX, NU>& Mo = *A.M;
    const F dt = Mo.A[0][H], b1 = Mo.B[0][0], b2 = Mo.B[H][0];
    const int g = lane / GS, r = lane % GS, gbase = g * GS;
    const int rr = r < NX ? r : NX - 1;  // row of this lane (lanes past NX mirror the last row, never store)
    int gbad = 0;
    unsigned rem = owners;
    while (rem) {
      // the next NG owners, in lane order; group g takes the g-th of them
      unsigned chunk = 0, m = rem;
      for (int k = 0; k < NG && m; ++k) {
        chunk |= m & (0u - m);
        m &= m - 1;
      }
      rem &= ~chunk;
      int olane = -1;
      {
        unsigned c2 = chunk;
        for (int k = 0; k < g && c2; ++k) c2 &= c2 - 1;
        if (c2) olane = __ffs(c2) - 1;
      }
      const int src = olane >= 0 ? olane : lane;
      F* const ocache = (F*)__shfl_sync(FULL, (unsigned long long)A.cache, src);
      uint16_t* const oW = (uint16_t*)__shfl_sync(FULL, (unsigned long long)A.Wm, src);
      uint16_t* const oC = (uint16_t*)__shfl_sync(FULL, (unsigned long long)A.Cm, src);
      const F* const okc = (const F*)__shfl_sync(FULL, (unsigned long long)A.kc, src);
      const int oks = __shfl_sync(FULL, A.ks, src);
      const int oN = __shfl_sync(FULL, A.N, src);
      const int oi = __shfl_sync(FULL, A.i, src);
      const int od = __shfl_sync(FULL, mine ? dirty : -1, src);
      const bool gact = olane >= 0;
      const int maxd = __reduce_max_sync(FULL, gact ? od : -1);
      auto OC = [&](int t, int e) -> F& { return ocache[((size_t)t * CL::E + e) * oN + oi]; };
      for (int t = maxd; t >= 0; --t) {
        const bool act = gact && t <= od;
        const bool row = act && r < NX;
        const uint16_t mask = act ? oW[(size_t)t * oN + oi] : (uint16_t)0;
        F Pr[NX];
#pragma unroll
        for (int c = 0; c < NX; ++c) Pr[c] = act ? OC(t + 1, CL::P + rr * NX + c) : F(0);
        F PAr[NX], PBr[NU];
#pragma unroll
        for (int c = 0; c < H; ++c) {
          PAr[c] = Pr[c];
          PAr[H + c] = fma(Pr[H + c], F(1), Pr[c] * dt);
          PBr[c] = fma(Pr[H + c], b2, Pr[c] * b1);
        }
        // rows H + a of PA and PB for the lanes a < NU
        const int shi = gbase + (r < NU ? r + H : rr);
        F PAh[NX], PBh[NU];
#pragma unroll
        for (int c = 0; c < NX; ++c) PAh[c] = shfl_f(PAr[c], shi);
#pragma unroll
        for (int c = 0; c < NU; ++c) PBh[c] = shfl_f(PBr[c], shi);
        // row ra = min(r, NU - 1) of S and of M = B'P A (fixed rows/cols replaced)
        const int ra = r < NU ? r : NU - 1;
        const bool fa = (mask >> ra) & 0x101;
        F Srow[NU], Mrow[NX];
#pragma unroll
        for (int b = 0; b < NU; ++b) {
          const bool fb = (mask >> b) & 0x101;
          F acc = (ra == b) ? (act ? okc[(AC::RB + ra) * oks] : F(1)) : F(0);
          acc = fma(b1, PBr[b], acc);
          acc = fma(b2, PBh[b], acc);
          Srow[b] = (fa || fb) ? F(ra == b ? 1 : 0) : acc;
        }
#pragma unroll
        for (int c = 0; c < NX; ++c) {
          F acc = 0;
          acc = fma(b1, PAr[c], acc);
          acc = fma(b2, PAh[c], acc);
          Mrow[c] = fa ? F(0) : acc;
        }
        // S, M on every lane of the group; S^{-1}; column rr of K
        F S[NU][NU], Mm[NU][NX], Si[NU][NU];
#pragma unroll
        for (int a = 0; a < NU; ++a) {
#pragma unroll
          for (int b = 0; b < NU; ++b) S[a][b] = shfl_f(Srow[b], gbase + a);
#pragma unroll
          for (int c = 0; c < NX; ++c) Mm[a][c] = shfl_f(Mrow[c], gbase + a);
        }
        const int sbad = sym_inverse<F, NU>(S, Si);
        if (act && r == 0) gbad |= sbad;
        F kcol[NU];
        {
          F mc[NU];
#pragma unroll
          for (int b = 0; b < NU; ++b) mc[b] = pick<F, NX>(Mm[b], rr);
          neg_sinv<F, NU>(Si, mc, kcol);
        }
        if (row) {
#pragma unroll
          for (int a = 0; a < NU; ++a) OC(t, CL::K + a * NX + rr) = kcol[a];
#pragma unroll
          for (int a = 0; a < NU; ++a) OC(t, CL::PB + rr * NU + a) = PBr[a];
        }
        if (act && r == 0) {
#pragma unroll
          for (int a = 0; a < NU; ++a)
#pragma unroll
            for (int b = 0; b <= a; ++b) OC(t, CL::L + a * NU + b) = Si[a][b];
          oC[(size_t)t * oN + oi] = mask;
        }
        if (t >= 1) {
          // P_t row rr: Qbar_t + A'(P A) + M'K, entries c >= rr
          F K[NU][NX], PAl[NX];
#pragma unroll
          for (int c = 0; c < NX; ++c)
#pragma unroll
            for (int a = 0; a < NU; ++a) K[a][c] = shfl_f(kcol[a], gbase + c);
          const int slo = gbase + (rr >= H ? rr - H : rr);
#pragma unroll
          for (int c = 0; c < NX; ++c) PAl[c] = shfl_f(PAr[c], slo);
          const F qd = act ? okc[(AC::QB + rr) * oks] : F(0);
          F mr[NU];
#pragma unroll
          for (int k = 0; k < NU; ++k) mr[k] = pick<F, NX>(Mm[k], rr);
#pragma unroll
          for (int c = 0; c < NX; ++c) {
            if (c < rr) continue;
            F acc = (rr == c) ? qd : F(0);
            if (rr < H) {
              acc = acc + PAr[c];
            } else {
              acc = fma(dt, PAl[c], acc);
              acc = acc + PAr[c];
            }
#pragma unroll
            for (int k = 0; k < NU; ++k) acc = fma(mr[k], K[k][c], acc);
            if (row) {
              OC(t, CL::P + rr * NX + c) = acc;
              if (c != rr) OC(t, CL::P + c * NX + rr) = acc;
            }
          }
        }
        __syncwarp();
      }
      // each owner of the chunk takes its group's status
      const int gi = __popc(chunk & ((1u << lane) - 1u));
      const int b = __shfl_sync(FULL, gbad, (mine && ((chunk >> lane) & 1u) ? gi : 0) * GS);
      if (mine && ((chunk >> lane) & 1u)) bad_out |= b;
      gbad = 0;
    }
  }
}

// One EQP solve with the cached stage factors (refactor_sweep brings them up to
// date first): backward affine pass, then forward pass (Sec. IV.B forward rollout) writing Us and X.
// The forward pass also scans the working-set multipliers
// mu = +-(Rbar u + B' lambda_{t+1}) with the costate lambda_{t+1} =
// P_{t+1} x_{t+1} + p_{t+1} (Sec. IV.B dual recovery), evaluated only at stages
// that hold fixed inputs, and flags free inputs that left the box (integer
// keys); the exact ratio test runs only when such an input exists.
template <typename F, int NX, int NU, int DP, bool DI>
__device__ EqpScan<F> eqp_solve(const AgentCtx<F, NX, NU, DP>& A) {
  constexpr int H = NX / 2;
  using CL = CacheLayout<NX, NU>;
  const Model<F, NX, NU>& Mo = *A.M;
  const int T = A.T;
  EqpScan<F> o;
  o.anum = 1; o.aden = 1; o.blk = -1; o.bside = 0; o.worst = 0; o.widx = -1; o.scale = 1; o.bad = 0; o.out = 0;

  F pn[NX];
#pragma unroll
  for (int r = 0; r < NX; ++r) pn[r] = A.q(T, r);

  // the mask, cached gains and h of the next stage are loaded one stage ahead
  uint16_t mask_n = A.W(T - 1);
  F Kn[NU][NX], Ln[NU][NU], hn[DP];
#pragma unroll
  for (int a = 0; a < NU; ++a) {
#pragma unroll
    for (int c = 0; c < NX; ++c) Kn[a][c] = A.C(T - 1, CL::K + a * NX + c);
#pragma unroll
    for (int b = 0; b < NU; ++b) Ln[a][b] = A.C(T - 1, CL::L + (b <= a ? a * NU + b : b * NU + a));
  }
#pragma unroll
  for (int r = 0; r < DP; ++r) hn[r] = (T - 1 >= 1) ? A.hv(T - 1, r) : F(0);
  for (int t = T - 1; t >= 0; --t) {
    const uint16_t mask = mask_n;
    F K[NU][NX], L[NU][NU], ht[DP];
#pragma unroll
    for (int r = 0; r < DP; ++r) ht[r] = hn[r];
#pragma unroll
    for (int a = 0; a < NU; ++a) {
#pragma unroll
      for (int c = 0; c < NX; ++c) K[a][c] = Kn[a][c];
#pragma unroll
      for (int b = 0; b < NU; ++b) L[a][b] = Ln[a][b];
    }
    if (t >= 1) {
      mask_n = A.W(t - 1);
#pragma unroll
      for (int a = 0; a < NU; ++a) {
#pragma unroll
        for (int c = 0; c < NX; ++c) Kn[a][c] = A.C(t - 1, CL::K + a * NX + c);
#pragma unroll
        for (int b = 0; b < NU; ++b) Ln[a][b] = A.C(t - 1, CL::L + (b <= a ? a * NU + b : b * NU + a));
      }
#pragma unroll
      for (int r = 0; r < DP; ++r) hn[r] = (t - 1 >= 1) ? A.hv(t - 1, r) : F(0);
    }
    // affine pass: P_{t+1} c + p_{t+1} with c = B_fixed u_fixed, i.e.
    // p_{t+1} + sum over the fixed inputs a of (P_{t+1} B)[:, a] u_a
    F Pcp[NX];
#pragma unroll
    for (int r = 0; r < NX; ++r) Pcp[r] = pn[r];
    if (mask) {
#pragma unroll
      for (int a = 0; a < NU; ++a) {
        if (!(mask & (0x101u << a))) continue;
        const F ub = (mask & (1u << a)) ? Mo.umin[a] : Mo.umax[a];
#pragma unroll
        for (int r = 0; r < NX; ++r) Pcp[r] = fma(A.C(t, CL::PB + r * NU + a), ub, Pcp[r]);
      }
      // B' p_{t+1} for the multipliers of the forward pass
#pragma unroll
      for (int a = 0; a < NU; ++a) {
        F acc = 0;
        if constexpr (DI) {
          acc = fma(Mo.B[0][0], pn[a], acc);
          acc = fma(Mo.B[H][0], pn[H + a], acc);
        } else {
#pragma unroll
          for (int r = 0; r < NX; ++r) acc = fma(Mo.B[r][a], pn[r], acc);
        }
        A.C(t, CL::bp + a) = acc;
      }
    }
    F sv[NU], kk[NU];
#pragma unroll
    for (int a = 0; a < NU; ++a) {
      F acc = 0;
      if constexpr (DI) {
        acc = fma(Mo.B[0][0], Pcp[a], acc);
        acc = fma(Mo.B[H][0], Pcp[H + a], acc);
      } else {
#pragma unroll
        for (int r = 0; r < NX; ++r) acc = fma(Mo.B[r][a], Pcp[r], acc);
      }
      sv[a] = (mask & (0x101u << a)) ? F(0) : acc;
    }
    neg_sinv<F, NU>(L, sv, kk);
#pragma unroll
    for (int a = 0; a < NU; ++a) A.C(t, CL::k + a) = kk[a];
    if (t >= 1) {
#pragma unroll
      for (int r = 0; r < NX; ++r) {
        F acc = A.q_h(r, r < DP ? ht[r] : F(0));
        if constexpr (DI) {
          if (r < H) {
            acc = acc + Pcp[r];
          } else {
            acc = fma(Mo.A[0][H], Pcp[r - H], acc);
            acc = acc + Pcp[r];
          }
        } else {
#pragma unroll
          for (int k = 0; k < NX; ++k) acc = fma(Mo.A[k][r], Pcp[k], acc);
        }
#pragma unroll
        for (int k = 0; k < NU; ++k) acc = fma(K[k][r], sv[k], acc);
        pn[r] = acc;
      }
    }
  }

  // forward rollout
  unsigned long long kmin[NU], kmax[NU];
#pragma unroll
  for (int a = 0; a < NU; ++a) {
    kmin[a] = mono_key(Mo.umin[a]);
    kmax[a] = mono_key(Mo.umax[a]);
  }
  F xv[NX];
#pragma unroll
  for (int r = 0; r < NX; ++r) {
    xv[r] = A.xi[r];
    A.x(0, r) = xv[r];
  }
  // the mask and feedback of the next stage are loaded one stage ahead
  uint16_t fmask_n = A.W(0);
  F kf_n[NU], Kf_n[NU][NX];
#pragma unroll
  for (int a = 0; a < NU; ++a) {
    kf_n[a] = A.C(0, CL::k + a);
#pragma unroll
    for (int c = 0; c < NX; ++c) Kf_n[a][c] = A.C(0, CL::K + a * NX + c);
  }
  for (int t = 0; t < T; ++t) {
    const uint16_t mask = fmask_n;
    F kf[NU], Kf[NU][NX];
#pragma unroll
    for (int a = 0; a < NU; ++a) {
      kf[a] = kf_n[a];
#pragma unroll
      for (int c = 0; c < NX; ++c) Kf[a][c] = Kf_n[a][c];
    }
    if (t + 1 < T) {
      fmask_n = A.W(t + 1);
#pragma unroll
      for (int a = 0; a < NU; ++a) {
        kf_n[a] = A.C(t + 1, CL::k + a);
#pragma unroll
        for (int c = 0; c < NX; ++c) Kf_n[a][c] = A.C(t + 1, CL::K + a * NX + c);
      }
    }
    F uv[NU];
#pragma unroll
    for (int a = 0; a < NU; ++a) {
      if (mask & (1u << a)) uv[a] = Mo.umin[a];
      else if (mask & (0x100u << a)) uv[a] = Mo.umax[a];
      else {
        F acc = kf[a];
#pragma unroll
        for (int c = 0; c < NX; ++c) acc = fma(Kf[a][c], xv[c], acc);
        uv[a] = acc;
        const unsigned long long ku = mono_key(acc);
        o.out |= (ku < kmin[a]) | (ku > kmax[a]);
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
    if (mask) {
#pragma unroll
      for (int a = 0; a < NU; ++a) {
        if (!(mask & (0x101u << a))) continue;
        // Rbar u + B' lambda_{t+1} with B' lambda_{t+1} = (P_{t+1} B)' x_{t+1} + B' p_{t+1}
        F g = A.C(t, CL::bp + a);
#pragma unroll
        for (int c = 0; c < NX; ++c) g = fma(A.C(t, CL::PB + c * NU + a), xn[c], g);
        g = fma(A.k(AgentConst<NX, NU>::RB + a), uv[a], g);
        const F mu = (mask & (1u << a)) ? g : -g;
        // comparisons on integer keys (the FP64 pipe is kept for arithmetic)
        const unsigned long long ab = abs_bits(mu);
        if (ab > abs_bits(o.scale)) o.scale = from_bits(ab, F(0));
        if (mono_key(mu) < mono_key(o.worst)) { o.worst = mu; o.widx = t * NU + a; }
        if (nan_key(ab, F(0))) o.bad = 1;
      }
    }
#pragma unroll
    for (int a = 0; a < NU; ++a) A.us(t, a) = uv[a];
#pragma unroll
    for (int r = 0; r < NX; ++r) {
      A.x(t + 1, r) = xn[r];
      xv[r] = xn[r];
    }
  }
#pragma unroll
  for (int r = 0; r < NX; ++r)
    if (!(xv[r] == xv[r]) || fabs_(xv[r]) > F(1e30)) o.bad = 1;
  return o;
}

// EQP solve of the agents of up to CoopShape<NX>::NG lanes of the warp, each
// agent on a group of lanes with one lane per state row: the backward affine
// pass and the forward rollout exchange rows by warp shuffles, so that an
// agent's stage recurrence is a few operations long instead of a few dozen.
// Every value is formed by the same operations, in the same order, as in
// eqp_solve, so both give identical bits.  Every lane of the warp calls this;
// `go` marks the lanes whose agent takes the pass (at most NG of them, the
// caller checks).  The owner lane receives its agent's scan.  Used by the
// per-phase x-update kernels, where few agents share a warp and each agent's
// recurrence latency sets the time, and by the register-unbounded variant 0 of
// the persistent kernel for its later active-set rounds, which serve a few
// agents of the warp (variant 1's 168-register budget leaves it out).
template <typename F, int NX, int NU, int DP>
__device__ EqpScan<F> eqp_coop(const AgentCtx<F, NX, NU, DP>& A, bool go) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int GS = CoopShape<NX>::GS, H = NX / 2;
  using CL = CacheLayout<NX, NU>;
  using AC = AgentConst<NX, NU>;
  const Model<F, NX, NU>& Mo = *A.M;
  const F dt = Mo.A[0][H], b1 = Mo.B[0][0], b2 = Mo.B[H][0];
  const int lane = threadIdx.x & 31, g = lane / GS, r = lane % GS, gbase = g * GS;
  const int rr = r < NX ? r : NX - 1;  // state row of this lane
  const int ra = r < NU ? r : NU - 1;  // input of this lane
  const unsigned owners = __ballot_sync(FULL, go);
  int olane = -1;
  {
    unsigned m = owners;
    for (int k = 0; k < g && m; ++k) m &= m - 1;
    if (m) olane = __ffs(m) - 1;
  }
  const int src = olane >= 0 ? olane : lane;
  auto sp = [&](auto p) { return (decltype(p))__shfl_sync(FULL, (unsigned long long)p, src); };
  F* const cache = sp(A.cache);
  uint16_t* const Wm = sp(A.Wm);
  F* const Us = sp(A.Us);
  F* const Xo = sp(A.Xo);
  const F* const hp = sp(A.h);
  const F* const kc = sp(A.kc);
  const F* const qf = sp(A.qf);
  const F* const xr = sp(A.xr);
  const F* const xi = sp(A.xi);
  const int ks = __shfl_sync(FULL, A.ks, src), N = __shfl_sync(FULL, A.N, src);
  const int ai = __shfl_sync(FULL, A.i, src), T = __shfl_sync(FULL, A.T, src);
  const bool gact = olane >= 0;
  const bool row = gact && r < NX;
  const int Tm = __reduce_max_sync(FULL, gact ? T : 0);
  auto C = [&](int t, int e) -> F& { return cache[((size_t)t * CL::E + e) * N + ai]; };
  const F rho = gact ? kc[AC::RHO * ks] : F(0);

  // backward affine pass; this lane carries p_{t+1}[rr]
  F pn = F(0);
  if (gact) {
    pn = terminal_lin(qf[rr], xr[rr]);
    if (rr < DP) pn = lin_term(pn, rho, hp[((size_t)(T - 1) * DP + rr) * N + ai]);
  }
  // this lane's operands of a stage, loaded one stage ahead: mask, row rr of
  // P_{t+1}B, row ra of S^{-1}, column rr of K, h_t[rr]
  uint16_t mk_n = 0;
  F pb_n[NU], si_n[NU], kq_n[NU], h_n = F(0);
  auto load_back = [&](int t) {
    const bool act = gact && t >= 0 && t < T;
    mk_n = act ? Wm[(size_t)t * N + ai] : (uint16_t)0;
#pragma unroll
    for (int a = 0; a < NU; ++a) {
      pb_n[a] = act ? C(t, CL::PB + rr * NU + a) : F(0);
      si_n[a] = act ? C(t, CL::L + (a <= ra ? ra * NU + a : a * NU + ra)) : F(0);
      kq_n[a] = act ? C(t, CL::K + a * NX + rr) : F(0);
    }
    h_n = (act && t >= 1 && rr < DP) ? hp[((size_t)(t - 1) * DP + rr) * N + ai] : F(0);
  };
  load_back(Tm - 1);
  for (int t = Tm - 1; t >= 0; --t) {
    const bool act = gact && t < T;
    const uint16_t mask = mk_n;
    F pbv[NU], si[NU], kq[NU];
#pragma unroll
    for (int a = 0; a < NU; ++a) {
      pbv[a] = pb_n[a];
      si[a] = si_n[a];
      kq[a] = kq_n[a];
    }
    const F hv = h_n;
    if (t >= 1) load_back(t - 1);
    F Pcp = pn;
    if (mask) {
#pragma unroll
      for (int a = 0; a < NU; ++a) {
        if (!(mask & (0x101u << a))) continue;
        const F ub = (mask & (1u << a)) ? Mo.umin[a] : Mo.umax[a];
        Pcp = fma(pbv[a], ub, Pcp);
      }
    }
    // rows H + ra of p_{t+1} and of P_{t+1} c + p_{t+1}
    const int shi = gbase + H + ra;
    const F pnh = shfl_f(pn, shi), Pcph = shfl_f(Pcp, shi);
    if (mask && r < NU) {
      F acc = 0;
      acc = fma(b1, pn, acc);
      acc = fma(b2, pnh, acc);
      C(t, CL::bp + ra) = acc;
    }
    F svl = 0;
    {
      F acc = 0;
      acc = fma(b1, Pcp, acc);
      acc = fma(b2, Pcph, acc);
      svl = (mask & (0x101u << ra)) ? F(0) : acc;
    }
    F sv[NU];
#pragma unroll
    for (int b = 0; b < NU; ++b) sv[b] = shfl_f(svl, gbase + b);
    if (act && r < NU) {
      // k_t row ra = -(S^{-1} s)[ra]
      F acc = si[0] * sv[0];
#pragma unroll
      for (int b = 1; b < NU; ++b) acc = fma(si[b], sv[b], acc);
      C(t, CL::k + ra) = -acc;
    }
    if (t >= 1) {
      const F Pcpl = shfl_f(Pcp, gbase + (rr >= H ? rr - H : rr));
      if (act) {
        F acc = kc[(AC::QL + rr) * ks];
        if (rr < DP) acc = lin_term(acc, rho, hv);
        if (rr < H) {
          acc = acc + Pcp;
        } else {
          acc = fma(dt, Pcpl, acc);
          acc = acc + Pcp;
        }
#pragma unroll
        for (int k = 0; k < NU; ++k) acc = fma(kq[k], sv[k], acc);
        pn = acc;
      }
    }
  }
  __syncwarp();

  // forward rollout; this lane carries x_t[rr]
  EqpScan<F> o;
  o.anum = 1; o.aden = 1; o.blk = -1; o.bside = 0; o.worst = 0; o.widx = -1; o.scale = 1; o.bad = 0; o.out = 0;
  const unsigned long long kmin = mono_key(Mo.umin[ra]), kmax = mono_key(Mo.umax[ra]);
  F xl = gact ? xi[rr] : F(0);
  if (row) Xo[(size_t)rr * N + ai] = xl;
  // this lane's operands of a stage, loaded one stage ahead: mask, k_t[ra],
  // row ra of K_t, B'p_{t+1}[ra], column ra of P_{t+1}B
  uint16_t fm_n = 0;
  F kf_n = F(0), Kr_n[NX], bp_n = F(0), pbc_n[NX];
  auto load_fwd = [&](int t) {
    const bool act = gact && t < T;
    fm_n = act ? Wm[(size_t)t * N + ai] : (uint16_t)0;
    kf_n = act ? C(t, CL::k + ra) : F(0);
    bp_n = act ? C(t, CL::bp + ra) : F(0);
#pragma unroll
    for (int c = 0; c < NX; ++c) {
      Kr_n[c] = act ? C(t, CL::K + ra * NX + c) : F(0);
      pbc_n[c] = act ? C(t, CL::PB + c * NU + ra) : F(0);
    }
  };
  load_fwd(0);
  for (int t = 0; t < Tm; ++t) {
    const bool act = gact && t < T;
    const uint16_t mask = fm_n;
    const F kfv = kf_n, bpv = bp_n;
    F Kr[NX], pbc[NX];
#pragma unroll
    for (int c = 0; c < NX; ++c) {
      Kr[c] = Kr_n[c];
      pbc[c] = pbc_n[c];
    }
    if (t + 1 < Tm) load_fwd(t + 1);
    F xv[NX];
#pragma unroll
    for (int c = 0; c < NX; ++c) xv[c] = shfl_f(xl, gbase + c);
    F ul;
    if (mask & (1u << ra)) ul = Mo.umin[ra];
    else if (mask & (0x100u << ra)) ul = Mo.umax[ra];
    else {
      F acc = kfv;
#pragma unroll
      for (int c = 0; c < NX; ++c) acc = fma(Kr[c], xv[c], acc);
      ul = acc;
      const unsigned long long ku = mono_key(acc);
      if (act && r < NU) o.out |= (ku < kmin) | (ku > kmax);
    }
    F uv[NU];
#pragma unroll
    for (int b = 0; b < NU; ++b) uv[b] = shfl_f(ul, gbase + b);
    F xn;
    if (rr < H) xn = fma(b1, pick<F, NU>(uv, rr), fma(dt, pick<F, NX>(xv, H + rr), xl));
    else xn = fma(b2, pick<F, NU>(uv, rr - H), xl);
    // every lane takes part in the shuffles (the masks differ between groups)
    F xnv[NX];
#pragma unroll
    for (int c = 0; c < NX; ++c) xnv[c] = shfl_f(xn, gbase + c);
    if (mask) {
      if (act && r < NU && (mask & (0x101u << ra))) {
        F gg = bpv;
#pragma unroll
        for (int c = 0; c < NX; ++c) gg = fma(pbc[c], xnv[c], gg);
        gg = fma(kc[(AC::RB + ra) * ks], ul, gg);
        const F mu = (mask & (1u << ra)) ? gg : -gg;
        const unsigned long long ab = abs_bits(mu);
        if (ab > abs_bits(o.scale)) o.scale = from_bits(ab, F(0));
        if (mono_key(mu) < mono_key(o.worst)) { o.worst = mu; o.widx = t * NU + ra; }
        if (nan_key(ab, F(0))) o.bad = 1;
      }
    }
    if (act && r < NU) Us[((size_t)t * NU + ra) * N + ai] = ul;
    if (act && r < NX) Xo[((size_t)(t + 1) * NX + rr) * N + ai] = xn;
    xl = xn;
  }
  if (row && (!(xl == xl) || fabs_(xl) > F(1e30))) o.bad = 1;
  // combine the group's lanes: first (lowest index) most negative multiplier,
  // largest |mu|, any flag
#pragma unroll
  for (int off = GS / 2; off > 0; off >>= 1) {
    const F w2 = shfl_f(o.worst, lane ^ off);
    const int i2 = __shfl_sync(FULL, o.widx, lane ^ off);
    const F s2 = shfl_f(o.scale, lane ^ off);
    const int b2i = __shfl_sync(FULL, o.bad, lane ^ off), o2 = __shfl_sync(FULL, o.out, lane ^ off);
    const unsigned long long k1 = mono_key(o.worst), k2 = mono_key(w2);
    if (i2 >= 0 && (o.widx < 0 || k2 < k1 || (k2 == k1 && i2 < o.widx))) {
      o.worst = w2;
      o.widx = i2;
    }
    if (abs_bits(s2) > abs_bits(o.scale)) o.scale = s2;
    o.bad |= b2i;
    o.out |= o2;
  }
  // the owner takes its group's result
  const int gi = __popc(owners & ((1u << lane) - 1u));
  const int from = (go ? gi : g) * GS;
  EqpScan<F> res;
  res.anum = 1; res.aden = 1; res.blk = -1; res.bside = 0;
  res.worst = shfl_f(o.worst, from);
  res.widx = __shfl_sync(FULL, o.widx, from);
  res.scale = shfl_f(o.scale, from);
  res.bad = __shfl_sync(FULL, o.bad, from);
  res.out = __shfl_sync(FULL, o.out, from);
  __syncwarp();
  return res;
}

// Ratio test of the primal active set (Nocedal & Wright Alg. 16.3) for the step
// p = us - u over the free inputs: smallest blocking ratio (clamped at 0), ties
// to the lowest (t, c) index, ratios compared as num*aden < anum*den.
template <typename F, int NX, int NU, int DP>
__device__ void ratio_test(const AgentCtx<F, NX, NU, DP>& A, EqpScan<F>& o) {
  const Model<F, NX, NU>& Mo = *A.M;
  for (int t0 = 0; t0 < A.T; t0 += kStageBatch) {
    // the operands of kStageBatch stages are loaded before they are used
    uint16_t mk[kStageBatch];
    F cuv[kStageBatch][NU], suv[kStageBatch][NU];
#pragma unroll
    for (int j = 0; j < kStageBatch; ++j) {
      const int t = t0 + j;
      mk[j] = t < A.T ? A.W(t) : (uint16_t)0xFFFF;
#pragma unroll
      for (int a = 0; a < NU; ++a) {
        cuv[j][a] = t < A.T ? A.u(t, a) : F(0);
        suv[j][a] = t < A.T ? A.us(t, a) : F(0);
      }
    }
#pragma unroll
    for (int j = 0; j < kStageBatch; ++j)
#pragma unroll
    for (int a = 0; a < NU; ++a) {
      const int t = t0 + j;
      if (mk[j] & (0x101u << a)) continue;
      const F cu = cuv[j][a];
      const F p = suv[j][a] - cu;
      // signs and the ratio comparison on integer keys: p < 0 (side 1) or
      // p > 0 (side 2); num = distance to the bound, clamped at +0; den = |p|;
      // blocking when num / den < anum / aden, compared as num*aden < anum*den
      const unsigned long long pb = abs_bits(p);
      if (pb == 0) continue;
      const bool lower = sign_set(p);
      const F hi = lower ? cu : Mo.umax[a], lo = lower ? Mo.umin[a] : cu;
      F num = hi - lo;
      if (sign_set(num)) num = F(0);
      const F den = from_bits(pb, F(0));
      if (mono_key(num * o.aden) < mono_key(o.anum * den)) {
        o.anum = num;
        o.aden = den;
        o.blk = t * NU + a;
        o.bside = lower ? 1 : 2;
      }
    }
  }
}

// u <- u + alpha (us - u) (alpha < 1) or u <- us (alpha = 1 passed as full),
// kStageBatch stages at a time with the loads ahead of the stores.
template <typename F, int NX, int NU, int DP>
__device__ __forceinline__ void step_inputs(const AgentCtx<F, NX, NU, DP>& A, int T, bool full, F alpha) {
  for (int t0 = 0; t0 < T; t0 += kStageBatch) {
    F cuv[kStageBatch][NU], suv[kStageBatch][NU];
#pragma unroll
    for (int j = 0; j < kStageBatch; ++j)
#pragma unroll
      for (int a = 0; a < NU; ++a) {
        const int t = t0 + j;
        cuv[j][a] = (t < T && !full) ? A.u(t, a) : F(0);
        suv[j][a] = t < T ? A.us(t, a) : F(0);
      }
#pragma unroll
    for (int j = 0; j < kStageBatch; ++j)
#pragma unroll
      for (int a = 0; a < NU; ++a) {
        const int t = t0 + j;
        if (t < T) A.u(t, a) = full ? suv[j][a] : fma(alpha, suv[j][a] - cuv[j][a], cuv[j][a]);
      }
  }
}

// Box-constrained local QP of agent i (Sec. IV.A) by the primal active-set
// method (Nocedal & Wright Alg. 16.3) over Riccati EQP solves.
// start_kind: QP_COLD (u = clip(0), W empty), QP_LQR (clipped affine-LQR warm
// start, Sec. IV.B-C) or QP_GIVEN (hot start from the stored u, W and factors).
// All 32 lanes of the warp call this together; a lane with has = false owns no
// agent and only helps the others' refactorizations.  The lanes step through
// their active-set iterations in rounds: in each round every lane that needs
// an EQP solve takes it in the same pass, since a pass costs the warp the same
// whatever number of lanes it serves.  Each lane's own sequence of working
// sets, steps and multiplier tests is unchanged.
// Returns ST_CONVERGED, ST_QP_FAIL or ST_NUMERIC.
template <typename F, int NX, int NU, int DP, bool DI, bool COOP_EQP>
__device__ int xupdate_agent(const AgentCtx<F, NX, NU, DP>& A, bool has, int start_kind, int as_max, F eps_rel,
                             unsigned long long& neqp, unsigned long long& nfact) {
  constexpr unsigned FULL = 0xffffffffu;
  const int T = has ? A.T : 0;
  const Model<F, NX, NU>& Mo = *A.M;
  int status = has ? -1 : ST_CONVERGED;  // -1: running
  int dirty = -1;
  if (has) {
    if (start_kind == QP_COLD) {
      for (int t = 0; t < T; ++t) {
        A.W(t) = 0;
#pragma unroll
        for (int a = 0; a < NU; ++a) {
          F z = 0;
          if (z < Mo.umin[a]) z = Mo.umin[a];
          if (z > Mo.umax[a]) z = Mo.umax[a];
          A.u(t, a) = z;
        }
      }
    } else if (start_kind == QP_LQR) {
      for (int t = 0; t < T; ++t) A.W(t) = 0;
    }
    // stages whose cached factors do not match the working set
    for (int t0 = 0; t0 < T; t0 += kStageBatch) {
      uint16_t cm[kStageBatch], w[kStageBatch];
#pragma unroll
      for (int j = 0; j < kStageBatch; ++j) {
        cm[j] = t0 + j < T ? A.CM(t0 + j) : (uint16_t)0;
        w[j] = t0 + j < T ? A.W(t0 + j) : (uint16_t)0;
      }
#pragma unroll
      for (int j = 0; j < kStageBatch; ++j)
        if (cm[j] != w[j]) dirty = t0 + j;
    }
  }

  const bool lqr = has && start_kind == QP_LQR;
  if (__any_sync(FULL, lqr)) {
    int bad = 0;
    refactor_sweep<F, NX, NU, DP, DI>(A, lqr, dirty, nfact, bad);
    if (lqr) {
      const EqpScan<F> o = eqp_solve<F, NX, NU, DP, DI>(A);
      if (bad || o.bad) {
        status = ST_NUMERIC;
      } else {
        dirty = -1;
        bool clipped = false;
        for (int t = 0; t < T; ++t) {
          uint16_t m = 0;
#pragma unroll
          for (int a = 0; a < NU; ++a) {
            F v = A.us(t, a);
            if (v < Mo.umin[a]) { v = Mo.umin[a]; m |= (uint16_t)(1u << a); }
            else if (v > Mo.umax[a]) { v = Mo.umax[a]; m |= (uint16_t)(0x100u << a); }
            A.u(t, a) = v;
          }
          if (m) { A.W(t) = m; clipped = true; dirty = t; }
        }
        if (!clipped) status = ST_CONVERGED;  // the LQR solution is the QP solution
      }
    }
  }

  for (;;) {
    bool go = false;
    if (status < 0) {
      if (as_max <= 0) status = ST_QP_FAIL;
      else go = true;
    }
    if (!__any_sync(FULL, go)) break;
    int bad = 0;
    refactor_sweep<F, NX, NU, DP, DI>(A, go, dirty, nfact, bad);
    // few agents in this round: each takes its pass on a group of lanes
    EqpScan<F> o;
    bool coop_pass = false;
    if constexpr (COOP_EQP && DI && (std::is_same<F, double>::value || std::is_same<F, float>::value)) {
      if (A.coop && __popc(__ballot_sync(FULL, go)) <= CoopShape<NX>::NG) {
        o = eqp_coop<F, NX, NU, DP>(A, go);
        coop_pass = true;
      }
    }
    if (go) {
      --as_max;
      ++neqp;
      if (!coop_pass) o = eqp_solve<F, NX, NU, DP, DI>(A);
      if (bad || o.bad) {
        status = ST_NUMERIC;
      } else {
        dirty = -1;
        if (o.out) ratio_test<F, NX, NU, DP>(A, o);
        if (o.blk >= 0) {
          const F alpha = o.anum / o.aden;
          step_inputs<F, NX, NU, DP>(A, T, false, alpha);
          const int bt = o.blk / NU, ba = o.blk - bt * NU;
          A.u(bt, ba) = (o.bside == 1) ? Mo.umin[ba] : Mo.umax[ba];
          A.W(bt) = (uint16_t)(A.W(bt) | (o.bside == 1 ? (1u << ba) : (0x100u << ba)));
          dirty = bt;
        } else {
          step_inputs<F, NX, NU, DP>(A, T, true, F(1));
          if (o.widx >= 0 && o.worst < -eps_rel * o.scale) {
            const int bt = o.widx / NU, ba = o.widx - bt * NU;
            A.W(bt) = (uint16_t)(A.W(bt) & ~(0x101u << ba));
            dirty = bt;
          } else {
            status = ST_CONVERGED;
          }
        }
      }
    }
  }
  return status;
}

// ---------------------------------------------------------------------------
// Scenario-level phases
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool finite_(double v) { return isfinite(v); }
__device__ __forceinline__ bool finite_(float v) { return isfinite(v); }

// State of one scenario at its first iteration: consensus copies w = w0 (the
// guess positions, stored as the previous positions p^0), duals zero
// (theta^0 = theta^{-1} = 0), aggregate h = n_c w0, caches invalid.
template <typename F, int NX, int NU, int DP>
__device__ void init_phase(const Dev<F>& D, const ScenMeta& s, int64_t t0, int64_t stride) {
  const int N = s.N, T = s.T, P = s.P;
  F* X0 = D.X + s.xs_off * NX;
  F* h = D.h + s.as_off * DP;
  const F* w0 = D.w0 + s.as_off * DP;
  F* U = D.U + s.as_off * NU;
  for (int64_t idx = t0; idx < (int64_t)N * T; idx += stride) {
    const int tm1 = (int)(idx / N), i = (int)(idx - (int64_t)tm1 * N);
    const F nc = F(agent_nc(D, s, i));
#pragma unroll
    for (int c = 0; c < DP; ++c) {
      const F w = w0[((size_t)tm1 * DP + c) * N + i];
      X0[((size_t)(tm1 + 1) * NX + c) * N + i] = w;
      h[((size_t)tm1 * DP + c) * N + i] = nc * w;
    }
#pragma unroll
    for (int c = 0; c < NU; ++c) U[((size_t)tm1 * NU + c) * N + i] = 0;
    D.Wm[s.as_off + idx] = 0;
    D.Cm[s.as_off + idx] = 0xFFFF;
  }
  for (int l = 0; l < 3; ++l) {
    F* th = D.theta + (size_t)l * D.tot_ps + s.ps_off;
    for (int64_t q = t0; q < (int64_t)P * T; q += stride) th[q] = 0;
  }
  if (D.relax) {
    // over-relaxation: consensus copies w^0 = s^0 = the guess positions, phi^0 = 0
    F* sx = D.sx + s.as_off * DP;
    for (int64_t q = t0; q < (int64_t)N * T * DP; q += stride) sx[q] = w0[q];
    F* ph = D.phi + s.ps_off;
    for (int64_t q = t0; q < (int64_t)P * T; q += stride) ph[q] = 0;
  }
}

// Dynamics of agent i of scenario s: its own when the batch has per-agent
// models (heterogeneous agents), else the shared model M.
template <typename F, int NX, int NU>
__device__ __forceinline__ const Model<F, NX, NU>& agent_model(const Dev<F>& D, const Model<F, NX, NU>& M,
                                                              const ScenMeta& s, int i) {
  return D.models ? reinterpret_cast<const Model<F, NX, NU>*>(D.models)[s.agent_off + i] : M;
}

// Agent context of agent i; its constants are written to the thread's column
// kc (stride ks) of a shared-memory table.
template <typename F, int NX, int NU, int DP, bool DI>
__device__ __forceinline__ AgentCtx<F, NX, NU, DP> make_agent(const Dev<F>& D, const Model<F, NX, NU>& M,
                                                              const ScenMeta& s, int i, int lvl_out, F* kc,
                                                              int ks, double rho) {
  using AC = AgentConst<NX, NU>;
  AgentCtx<F, NX, NU, DP> A;
  A.M = DI ? &M : &agent_model<F, NX, NU>(D, M, s, i);  // the structured path has one model
  A.N = s.N;
  A.T = s.T;
  A.i = i;
  A.cache = D.cache + s.xs_off * CacheLayout<NX, NU>::E;
  A.Wm = D.Wm + s.as_off;
  A.Cm = D.Cm + s.as_off;
  A.U = D.U + s.as_off * NU;
  A.Us = D.Us + s.as_off * NU;
  A.Xo = D.X + (size_t)lvl_out * D.tot_xs * NX + s.xs_off * NX;
  A.h = D.h + s.as_off * DP;
  A.kc = kc;
  A.ks = ks;
  A.coop = D.coop;
  const int64_t ag = s.agent_off + i;
  A.qf = D.Qfd + ag * NX;
  A.xr = D.x_ref + ag * NX;
  A.xi = D.x_init + ag * NX;
  A.nc = agent_nc(D, s, i);
  const F rnc = F(rho) * F(A.nc);
  kc[AC::RHO * ks] = F(rho);
#pragma unroll
  for (int r = 0; r < NX; ++r) {
    const F q = D.Qd[ag * NX + r], xr = D.x_ref[ag * NX + r];
    kc[(AC::QB + r) * ks] = F(2) * q + (r < DP ? rnc : F(0));
    kc[(AC::QL + r) * ks] = (F(-2) * q) * xr;
  }
#pragma unroll
  for (int c = 0; c < NU; ++c) kc[(AC::RB + c) * ks] = F(2) * D.Rd[ag * NU + c];
  return A;
}

// Context of a lane that owns no agent in this x-update (it only helps).
template <typename F, int NX, int NU, int DP>
__device__ __forceinline__ AgentCtx<F, NX, NU, DP> idle_agent(const Model<F, NX, NU>& M, F* kc, int ks, int coop) {
  AgentCtx<F, NX, NU, DP> A;
  A.M = &M;
  A.N = 1;
  A.T = 0;
  A.i = 0;
  A.cache = nullptr;
  A.Wm = nullptr;
  A.Cm = nullptr;
  A.U = nullptr;
  A.Us = nullptr;
  A.Xo = nullptr;
  A.h = nullptr;
  A.kc = kc;
  A.ks = ks;
  A.qf = nullptr;
  A.xr = nullptr;
  A.xi = nullptr;
  A.coop = coop;
  A.nc = 0;
  return A;
}

template <typename F>
__device__ __forceinline__ int start_kind_of(const Dev<F>& D, int k) {
  if (D.start_mode == START_COLD) return QP_COLD;
  if (k == 0) return (D.start_mode == START_TURBO || D.start_mode == START_HOMOTOPY) ? QP_LQR : QP_COLD;
  return QP_GIVEN;
}

// ---------------------------------------------------------------------------
// Parametric (homotopy) hot start of the per-agent QP, in the manner of
// qpOASES's hot start (Sec. IV.C names qpOASES's hotstart as the source of the
// paper's hot start): the optimum is followed from the previous x-update's
// linear term q_old to the new one along q(tau) = q_old + tau (q - q_old),
// tau: 0 -> 1.  On each segment the working set W is fixed and the optimum
// moves linearly, u(tau) = u + tau du, mu(tau) = mu + tau dmu, where (du, dmu)
// solve the equality-constrained problem with linear term q - q_old, x_0 = 0
// and the held inputs at 0 (the direction solve).  The segment ends where a
// free input meets a bound or a held input's multiplier meets zero (smallest
// step, ties to the lowest (t, c) index; steps clamped at 0); the working set
// changes there and the next segment starts.  The primal active set then
// confirms the end point (one EQP solve when the homotopy reached tau = 1).
// ---------------------------------------------------------------------------

// u + s v with a separate product and sum (no contraction), the order in which
// the plain definition of the segment step is written.
__device__ __forceinline__ double step_rn(double u, double s, double v) { return __dadd_rn(u, __dmul_rn(s, v)); }
__device__ __forceinline__ float step_rn(float u, float s, float v) { return __fadd_rn(u, __fmul_rn(s, v)); }
__device__ __forceinline__ df64 step_rn(df64 u, df64 s, df64 v) { return u + s * v; }

// Direction solve of one agent with the cached stage factors (one lane per
// agent): linear term q_t - q_old,t (t = 1..T), x_0 = 0, held inputs at 0.
// Writes du to Us and the held inputs' multiplier directions
// dmu = +-(B' dlambda_{t+1}) (no Rbar term: a held input's direction is 0) to
// dmu; returns 1 on a non-finite value.
template <typename F, int NX, int NU, int DP, bool DI>
__device__ int eqp_direction(const AgentCtx<F, NX, NU, DP>& A, const F* hprev, F* dmu) {
  constexpr int H = NX / 2;
  using CL = CacheLayout<NX, NU>;
  const Model<F, NX, NU>& Mo = *A.M;
  const int T = A.T, N = A.N, i = A.i;
  auto dq = [&](int t, int r) -> F {   // (q - q_old)_t row r
    if (r >= DP) return F(0);
    const F hp = hprev[((size_t)(t - 1) * DP + r) * N + i];
    if (t < T) return A.q_h(r, A.hv(t, r)) - A.q_h(r, hp);
    const F base = terminal_lin(A.qf[r], A.xr[r]);
    return lin_term(base, A.k(AgentConst<NX, NU>::RHO), A.hv(t, r)) -
           lin_term(base, A.k(AgentConst<NX, NU>::RHO), hp);
  };
  F pn[NX];
#pragma unroll
  for (int r = 0; r < NX; ++r) pn[r] = dq(T, r);
  for (int t = T - 1; t >= 0; --t) {
    const uint16_t mask = A.W(t);
    F K[NU][NX], L[NU][NU];
#pragma unroll
    for (int a = 0; a < NU; ++a) {
#pragma unroll
      for (int c = 0; c < NX; ++c) K[a][c] = A.C(t, CL::K + a * NX + c);
#pragma unroll
      for (int b = 0; b < NU; ++b) L[a][b] = A.C(t, CL::L + (b <= a ? a * NU + b : b * NU + a));
    }
    F bpn[NU], sv[NU], kk[NU];
#pragma unroll
    for (int a = 0; a < NU; ++a) {
      F acc = 0;
      if constexpr (DI) {
        acc = fma(Mo.B[0][0], pn[a], acc);
        acc = fma(Mo.B[H][0], pn[H + a], acc);
      } else {
#pragma unroll
        for (int r = 0; r < NX; ++r) acc = fma(Mo.B[r][a], pn[r], acc);
      }
      bpn[a] = acc;
      sv[a] = (mask & (0x101u << a)) ? F(0) : acc;
    }
    if (mask) {
#pragma unroll
      for (int a = 0; a < NU; ++a) A.C(t, CL::bp + a) = bpn[a];
    }
    neg_sinv<F, NU>(L, sv, kk);
#pragma unroll
    for (int a = 0; a < NU; ++a) A.C(t, CL::k + a) = kk[a];
    if (t >= 1) {
      F np[NX];
#pragma unroll
      for (int r = 0; r < NX; ++r) {
        F acc = dq(t, r);
#pragma unroll
        for (int k = 0; k < NX; ++k) acc = fma(Mo.A[k][r], pn[k], acc);
#pragma unroll
        for (int k = 0; k < NU; ++k) acc = fma(K[k][r], sv[k], acc);
        np[r] = acc;
      }
#pragma unroll
      for (int r = 0; r < NX; ++r) pn[r] = np[r];
    }
  }
  F xv[NX];
#pragma unroll
  for (int r = 0; r < NX; ++r) xv[r] = F(0);
  int bad = 0;
  for (int t = 0; t < T; ++t) {
    const uint16_t mask = A.W(t);
    F uv[NU];
#pragma unroll
    for (int a = 0; a < NU; ++a) {
      if (mask & (0x101u << a)) {
        uv[a] = F(0);
      } else {
        F acc = A.C(t, CL::k + a);
#pragma unroll
        for (int c = 0; c < NX; ++c) acc = fma(A.C(t, CL::K + a * NX + c), xv[c], acc);
        uv[a] = acc;
      }
    }
    F xn[NX];
#pragma unroll
    for (int r = 0; r < NX; ++r) {
      F acc = 0;
#pragma unroll
      for (int c = 0; c < NX; ++c) acc = fma(Mo.A[r][c], xv[c], acc);
#pragma unroll
      for (int c = 0; c < NU; ++c) acc = fma(Mo.B[r][c], uv[c], acc);
      xn[r] = acc;
    }
#pragma unroll
    for (int a = 0; a < NU; ++a) {
      A.us(t, a) = uv[a];
      F d = F(0);
      if (mask & (0x101u << a)) {
        // B' dlambda_{t+1} = (P_{t+1} B)' dx_{t+1} + B' dp_{t+1}
        F g = A.C(t, CL::bp + a);
#pragma unroll
        for (int c = 0; c < NX; ++c) g = fma(A.C(t, CL::PB + c * NU + a), xn[c], g);
        d = (mask & (1u << a)) ? g : -g;
      }
      dmu[((size_t)t * NU + a) * N + i] = d;
      if (!finite_(d) || !finite_(uv[a])) bad = 1;
    }
#pragma unroll
    for (int r = 0; r < NX; ++r) xv[r] = xn[r];
  }
  return bad;
}

// Homotopy segments of the warp's agents from (u, W, mu) of the previous
// x-update (all lanes call this together; lanes with has = false only help
// the refactorizations).  Counts every direction solve in neqp.  Returns
// ST_NUMERIC on a non-finite value, else ST_CONVERGED (the confirming primal
// active-set solve follows in xupdate_agent).
template <typename F, int NX, int NU, int DP, bool DI>
__device__ int homotopy_agent(const AgentCtx<F, NX, NU, DP>& A, bool has, const F* hprev, F* mu, F* dmu,
                              int as_max, unsigned long long& neqp, unsigned long long& nfact) {
  constexpr unsigned FULL = 0xffffffffu;
  const Model<F, NX, NU>& Mo = *A.M;
  const int T = has ? A.T : 0, N = A.N, i = A.i;
  auto MU = [&](F* b, int t, int c) -> F& { return b[((size_t)t * NU + c) * N + i]; };
  int dirty = -1;
  for (int t = 0; t < T; ++t)
    if (A.CM(t) != A.W(t)) dirty = t;
  bool done = !has;
  int status = ST_CONVERGED, steps = 0;
  F tau = F(0);
  for (;;) {
    const bool go = !done && steps < as_max;
    if (!__any_sync(FULL, go)) break;
    int bad = 0;
    refactor_sweep<F, NX, NU, DP, DI>(A, go, dirty, nfact, bad);
    if (!go) continue;
    ++steps;
    ++neqp;
    if (bad || eqp_direction<F, NX, NU, DP, DI>(A, hprev, dmu)) {
      status = ST_NUMERIC;
      done = true;
      continue;
    }
    dirty = -1;
    F best = F(1) - tau;
    int bk = -1, side = 0;
    for (int t = 0; t < T; ++t) {
      const uint16_t w = A.W(t);
#pragma unroll
      for (int c = 0; c < NU; ++c) {
        F r;
        int sd;
        if (!(w & (0x101u << c))) {
          const F du = A.us(t, c), u = A.u(t, c);
          if (du > F(0)) { r = (Mo.umax[c] - u) / du; sd = 2; }
          else if (du < F(0)) { r = (Mo.umin[c] - u) / du; sd = 1; }
          else continue;
        } else {
          const F dm = MU(dmu, t, c);
          if (!(dm < F(0))) continue;
          r = MU(mu, t, c) / -dm;
          sd = 0;
        }
        if (r < F(0)) r = F(0);
        if (r < best) { best = r; bk = t * NU + c; side = sd; }
      }
    }
    for (int t = 0; t < T; ++t) {
      const uint16_t w = A.W(t);
#pragma unroll
      for (int c = 0; c < NU; ++c) {
        if (!(w & (0x101u << c))) A.u(t, c) = step_rn(A.u(t, c), best, A.us(t, c));
        else MU(mu, t, c) = step_rn(MU(mu, t, c), best, MU(dmu, t, c));
      }
    }
    tau = tau + best;
    if (bk < 0) {
      done = true;   // tau = 1: the segment reached the new problem
      continue;
    }
    const int bt = bk / NU, ba = bk - bt * NU;
    if (side) {
      A.W(bt) = (uint16_t)(A.W(bt) | (side == 1 ? (1u << ba) : (0x100u << ba)));
      A.u(bt, ba) = side == 1 ? Mo.umin[ba] : Mo.umax[ba];
    } else {
      A.W(bt) = (uint16_t)(A.W(bt) & ~(0x101u << ba));
    }
    MU(mu, bt, ba) = F(0);
    dirty = bt;
  }
  return status;
}

// Bound multipliers of the agent's QP optimum (for the next homotopy) from the
// costate recursion lambda_T = Qbar_T x_T + q_T, lambda_t = Qbar_t x_t + q_t +
// A' lambda_{t+1} (Sec. IV.B dual recovery): mu = +-(Rbar u_t + B' lambda_{t+1})
// on the held inputs (lower: +, upper: -), 0 on the free ones; and the coupling
// term of this x-update becomes the agent's previous one.
template <typename F, int NX, int NU, int DP>
__device__ void homotopy_store(const AgentCtx<F, NX, NU, DP>& A, F* hprev, F* mu) {
  using AC = AgentConst<NX, NU>;
  const Model<F, NX, NU>& Mo = *A.M;
  const int T = A.T, N = A.N, i = A.i;
  F lam[NX];
#pragma unroll
  for (int r = 0; r < NX; ++r) lam[r] = F(0);
  for (int t = T; t >= 1; --t) {
    F ln[NX];
#pragma unroll
    for (int r = 0; r < NX; ++r) {
      const F qb = t < T ? A.k(AC::QB + r) : A.qbarT(r);
      F acc = fma(qb, A.x(t, r), A.q(t, r));
#pragma unroll
      for (int k = 0; k < NX; ++k) acc = fma(Mo.A[k][r], lam[k], acc);
      ln[r] = acc;
    }
    const uint16_t w = A.W(t - 1);
#pragma unroll
    for (int c = 0; c < NU; ++c) {
      F m = F(0);
      if (w & (0x101u << c)) {
        F g = A.k(AC::RB + c) * A.u(t - 1, c);
#pragma unroll
        for (int r = 0; r < NX; ++r) g = fma(Mo.B[r][c], ln[r], g);
        m = (w & (1u << c)) ? g : -g;
      }
      mu[((size_t)(t - 1) * NU + c) * N + i] = m;
    }
#pragma unroll
    for (int r = 0; r < NX; ++r) lam[r] = ln[r];
#pragma unroll
    for (int r = 0; r < DP; ++r) hprev[((size_t)(t - 1) * DP + r) * N + i] = A.hv(t, r);
  }
}

// x-update of agents i0, i0 + stride, ... of scenario s (none when in_scen is
// false).  Every lane of the warp calls this; all lanes take the same number
// of rounds, so that xupdate_agent always runs warp-wide.
template <typename F, int NX, int NU, int DP, bool DI, bool COOP_EQP = false, bool HOMO = false>
__device__ int xupdate_phase(const Dev<F>& D, const Model<F, NX, NU>& M, const ScenMeta& s, bool in_scen, int k,
                             int lvl_out, int i0, int stride, unsigned long long& neqp,
                             unsigned long long& nfact, F* kcs) {
  const int kind = start_kind_of(D, k);
  const int as_max = D.as_max > 0 ? D.as_max : 10 * s.T * NU + 10;
  const F eps = D.eps_rel > 0 ? F(D.eps_rel) : (sizeof(F) == 8 ? F(1e-12) : F(1e-5));
  const int mine = (in_scen && i0 < s.N) ? (s.N - i0 + stride - 1) / stride : 0;
  const int rounds = __reduce_max_sync(0xffffffffu, mine);
  int st = ST_CONVERGED;
  for (int r = 0; r < rounds; ++r) {
    const bool has = r < mine;
    const AgentCtx<F, NX, NU, DP> A =
        has ? make_agent<F, NX, NU, DP, DI>(D, M, s, i0 + r * stride, lvl_out, kcs + threadIdx.x, blockDim.x, s.rho)
            : idle_agent<F, NX, NU, DP>(M, kcs + threadIdx.x, blockDim.x, D.coop);
    int res = ST_CONVERGED;
    if constexpr (HOMO) {
      // warp-collective: every lane enters when any lane's agent takes a
      // homotopy (lanes of other iterations or of stopped scenarios only help)
      const bool hh = has && k > 0;
      if (__any_sync(0xffffffffu, hh))
        res = homotopy_agent<F, NX, NU, DP, DI>(A, hh, D.hprev + s.as_off * DP, D.mu + s.as_off * NU,
                                               D.dmu + s.as_off * NU, as_max, neqp, nfact);
    }
    const int r2 = xupdate_agent<F, NX, NU, DP, DI, COOP_EQP>(A, has && res == ST_CONVERGED, kind, as_max, eps,
                                                             neqp, nfact);
    if (res == ST_CONVERGED) res = r2;
    if constexpr (HOMO) {
      if (has && res == ST_CONVERGED) homotopy_store<F, NX, NU, DP>(A, D.hprev + s.as_off * DP, D.mu + s.as_off * NU);
    }
    if (has && res > st) st = res;
  }
  return st;
}

// Consensus projection + scaled dual update in theta form and the primal
// residual.  theta^{k+1} = max(0, theta^k + (d - a'(p_i - p_j)) / 2); the dual
// copies are y_i = -theta a, y_j = +theta a; r = |theta^{k+1} - theta^k| max|a_c|.
// X level xl holds p^k, xl^1 holds p^{k+1}; theta slots tk -> tkp1.
template <typename F, int NX, int NU, int DP>
__device__ void pair_phase(const Dev<F>& D, const ScenMeta& s, int xl, int tk, int tkp1, int64_t q0,
                           int64_t stride, unsigned long long& rb) {
  const int N = s.N, P = s.P;
  const int64_t PT = (int64_t)P * s.T;
  const F* Xn = D.X + (size_t)(xl ^ 1) * D.tot_xs * NX + s.xs_off * NX;
  const F* thk = D.theta + (size_t)tk * D.tot_ps + s.ps_off;
  F* thn = D.theta + (size_t)tkp1 * D.tot_ps + s.ps_off;
  const F* a = D.a + s.ps_off * DP;
  const int32_t* pr = D.pairs + s.pair_off;
  const F d = F(s.d);
  for (int64_t q = q0; q < PT; q += stride) {
    const int tm1 = (int)(q / P);
    const int pair = (int)(q - (int64_t)tm1 * P);
    const int pk = pr[pair];
    const int i = pk & 0xFFFF, j = pk >> 16;
    F g = d;  // d - a'(p_i - p_j)
    unsigned long long amax = 0;
#pragma unroll
    for (int c = 0; c < DP; ++c) {
      const F av = a[((size_t)tm1 * DP + c) * P + pair];
      const size_t ro = ((size_t)(tm1 + 1) * NX + c) * N;
      g = fma(-av, Xn[ro + i] - Xn[ro + j], g);
      const unsigned long long ab = abs_bits(av);
      amax = ab > amax ? ab : amax;
    }
    const F th = thk[q];
    F tn = fma(g, F(0.5), th);
    if (sign_set(tn)) tn = F(0);
    thn[q] = tn;
    const unsigned long long v = abs_bits((tn - th) * from_bits(amax, F(0)));
    rb = v > rb ? v : rb;
  }
}

// Dual residual s / rho = max |Delta p +- (theta^{k+1} - 2 theta^k + theta^{k-1}) a|
// over pairs, steps, sides and components (the change of the consensus copies);
// with rb, also the exact primal residual max |(theta^{k+1} - theta^k) a_c|.
template <typename F, int NX, int NU, int DP>
__device__ void dual_phase(const Dev<F>& D, const ScenMeta& s, int xl, int tkm1, int tk, int tkp1, int64_t q0,
                           int64_t stride, unsigned long long& sb, unsigned long long* rb = nullptr) {
  const int N = s.N, P = s.P;
  const int64_t PT = (int64_t)P * s.T;
  const F* Xn = D.X + (size_t)(xl ^ 1) * D.tot_xs * NX + s.xs_off * NX;
  const F* Xc = D.X + (size_t)xl * D.tot_xs * NX + s.xs_off * NX;
  const F* thm = D.theta + (size_t)tkm1 * D.tot_ps + s.ps_off;
  const F* thk = D.theta + (size_t)tk * D.tot_ps + s.ps_off;
  const F* thn = D.theta + (size_t)tkp1 * D.tot_ps + s.ps_off;
  const F* a = D.a + s.ps_off * DP;
  const int32_t* pr = D.pairs + s.pair_off;
  for (int64_t q = q0; q < PT; q += stride) {
    const int tm1 = (int)(q / P);
    const int pair = (int)(q - (int64_t)tm1 * P);
    const int pk = pr[pair];
    const int i = pk & 0xFFFF, j = pk >> 16;
    const F th = thk[q];
    const F e2 = (thn[q] - th) - (th - thm[q]);
#pragma unroll
    for (int c = 0; c < DP; ++c) {
      const F av = a[((size_t)tm1 * DP + c) * P + pair];
      if (rb) {
        // primal residual term |(theta' - theta) a_c|: their maximum has the bits
        // of the product with max_c |a_c| (rounding is monotone)
        const unsigned long long rv = abs_bits((thn[q] - th) * av);
        *rb = rv > *rb ? rv : *rb;
      }
      const size_t ro = ((size_t)(tm1 + 1) * NX + c) * N;
      const unsigned long long v1 = abs_bits(fma(e2, av, Xn[ro + i] - Xc[ro + i]));
      const unsigned long long v2 = abs_bits(fma(-e2, av, Xn[ro + j] - Xc[ro + j]));
      sb = v1 > sb ? v1 : sb;
      sb = v2 > sb ? v2 : sb;
    }
  }
}

// Aggregate linear term of the next x-update for agent i at step t:
// h_it = sum_{j != i} (w_i - y_i) = n_c p_it + sum_j sigma_ij (2 theta^{k+1} - theta^k) a_ijt,
// sigma = +1 when i is the first agent of the pair, -1 otherwise.
template <typename F, int NX, int NU, int DP>
__device__ void gather_phase(const Dev<F>& D, const ScenMeta& s, int xl_new, int tkp1, int tk, int64_t t0,
                             int64_t stride) {
  const int N = s.N, P = s.P;
  const F* Xn = D.X + (size_t)xl_new * D.tot_xs * NX + s.xs_off * NX;
  const F* thn = D.theta + (size_t)tkp1 * D.tot_ps + s.ps_off;
  const F* tho = D.theta + (size_t)tk * D.tot_ps + s.ps_off;
  const F* a = D.a + s.ps_off * DP;
  F* h = D.h + s.as_off * DP;
  for (int64_t idx = t0; idx < (int64_t)N * s.T; idx += stride) {
    const int tm1 = (int)(idx / N), i = (int)(idx - (int64_t)tm1 * N);
    const F nc = F(agent_nc(D, s, i));
    F acc[DP];
#pragma unroll
    for (int c = 0; c < DP; ++c) acc[c] = nc * Xn[((size_t)(tm1 + 1) * NX + c) * N + i];
    const size_t qb = (size_t)tm1 * P;
    for_partners(D, s, i, [&](int pair, bool first) {
      F e = fma(F(2), thn[qb + pair], -tho[qb + pair]);
      if (!first) e = -e;
#pragma unroll
      for (int c = 0; c < DP; ++c) acc[c] = fma(e, a[((size_t)tm1 * DP + c) * P + pair], acc[c]);
    });
#pragma unroll
    for (int c = 0; c < DP; ++c) h[((size_t)tm1 * DP + c) * N + i] = acc[c];
  }
}

// Shared-memory tile of the tiled gather: for 32 own agents (rows) x 32
// partners (columns), the signed weight sigma (2 theta^{k+1} - theta^k) and the
// DP components of the pair normal.  Rows padded to 33 against bank conflicts.
template <typename F, int DP>
struct GatherTile {
  F e[32][33];
  F a[DP][32][33];
};

// The aggregate h of gather_phase for the agents i0..i0+31 of one scenario at
// step tm1, computed by one warp.  Partners are swept in blocks of 32 in
// increasing order; each block's weights and normals are staged through
// coalesced row loads (pairs (i, j), i < j, are contiguous in j; pairs (j, i),
// j < i, contiguous in i and staged transposed).  Each agent then adds its
// partners' terms in increasing j: the same values, operations and order as
// gather_phase, so the result is bitwise the same.
template <typename F, int NX, int NU, int DP>
__device__ void gather_tile(const Dev<F>& D, const ScenMeta& s, int xl_new, int tkp1, int tk, int i0, int tm1,
                            GatherTile<F, DP>& ts) {
  const int N = s.N, P = s.P, lane = threadIdx.x & 31;
  const F* Xn = D.X + (size_t)xl_new * D.tot_xs * NX + s.xs_off * NX;
  const F* thn = D.theta + (size_t)tkp1 * D.tot_ps + s.ps_off + (size_t)tm1 * P;
  const F* tho = D.theta + (size_t)tk * D.tot_ps + s.ps_off + (size_t)tm1 * P;
  const F* a = D.a + s.ps_off * DP + (size_t)tm1 * DP * P;
  const int i = i0 + lane;
  const bool own = i < N;
  const int rows = min(32, N - i0);
  F acc[DP];
#pragma unroll
  for (int c = 0; c < DP; ++c) acc[c] = own ? F(agent_nc(D, s, i)) * Xn[((size_t)(tm1 + 1) * NX + c) * N + i] : F(0);
  if (s.sparse) {
    // listed pairs: each lane sums its own agent's pairs (no tile)
    if (own) {
      for_partners(D, s, i, [&](int pair, bool first) {
        F e = fma(F(2), thn[pair], -tho[pair]);
        if (!first) e = -e;
#pragma unroll
        for (int c = 0; c < DP; ++c) acc[c] = fma(e, a[(size_t)c * P + pair], acc[c]);
      });
      F* h = D.h + s.as_off * DP;
#pragma unroll
      for (int c = 0; c < DP; ++c) h[((size_t)tm1 * DP + c) * N + i] = acc[c];
    }
    return;
  }
  for (int j0 = 0; j0 < N; j0 += 32) {
    const int cols = min(32, N - j0);
    __syncwarp();
    if (i0 < j0 + cols - 1) {
      // pairs (i, j) with i < j: row r = own agent, lane = partner
      const int j = j0 + lane;
#pragma unroll 8
      for (int r = 0; r < rows; ++r) {
        const int ii = i0 + r;
        if (lane < cols && ii < j) {
          const int pair = pair_index(N, ii, j);
          ts.e[r][lane] = fma(F(2), thn[pair], -tho[pair]);
#pragma unroll
          for (int c = 0; c < DP; ++c) ts.a[c][r][lane] = a[(size_t)c * P + pair];
        }
      }
    }
    if (j0 < i0 + rows - 1) {
      // pairs (j, i) with j < i: row r = partner, lane = own agent (transposed)
#pragma unroll 8
      for (int r = 0; r < cols; ++r) {
        const int jj = j0 + r;
        if (own && jj < i) {
          const int pair = pair_index(N, jj, i);
          ts.e[lane][r] = -fma(F(2), thn[pair], -tho[pair]);
#pragma unroll
          for (int c = 0; c < DP; ++c) ts.a[c][lane][r] = a[(size_t)c * P + pair];
        }
      }
    }
    __syncwarp();
    if (own) {
      for (int cidx = 0; cidx < cols; ++cidx) {
        if (j0 + cidx == i) continue;
        const F e = ts.e[lane][cidx];
#pragma unroll
        for (int c = 0; c < DP; ++c) acc[c] = fma(e, ts.a[c][lane][cidx], acc[c]);
      }
    }
  }
  if (own) {
    F* h = D.h + s.as_off * DP;
#pragma unroll
    for (int c = 0; c < DP; ++c) h[((size_t)tm1 * DP + c) * N + i] = acc[c];
  }
}

// Pair phase and gather fused per time step for a CTA-resident scenario: the
// projection steps of step t are computed for all pairs (coalesced), the
// coupling weights e = 2 theta^{k+1} - theta^k and the normals of step t are
// staged in shared memory, then each agent sums its partners' terms from
// shared memory.  Same arithmetic, in the same order, as pair_phase followed by
// gather_phase.  sm holds (DP + 1) * P values.
template <typename F, int NX, int NU, int DP>
__device__ void pair_gather_fused(const Dev<F>& D, const ScenMeta& s, int xl, int tk, int tkp1, F* sm,
                                  unsigned long long& rb) {
  const int N = s.N, P = s.P, tid = threadIdx.x, nt = blockDim.x;
  const F* Xn = D.X + (size_t)(xl ^ 1) * D.tot_xs * NX + s.xs_off * NX;
  const F* thk = D.theta + (size_t)tk * D.tot_ps + s.ps_off;
  F* thn = D.theta + (size_t)tkp1 * D.tot_ps + s.ps_off;
  const F* a = D.a + s.ps_off * DP;
  const int32_t* pr = D.pairs + s.pair_off;
  F* h = D.h + s.as_off * DP;
  F* smE = sm;
  F* smA = sm + P;
  const F d = F(s.d);
  for (int tm1 = 0; tm1 < s.T; ++tm1) {
    const size_t qb = (size_t)tm1 * P;
    for (int pair = tid; pair < P; pair += nt) {
      const int pk = pr[pair];
      const int i = pk & 0xFFFF, j = pk >> 16;
      F g = d;  // d - a'(p_i - p_j)
      unsigned long long amax = 0;
#pragma unroll
      for (int c = 0; c < DP; ++c) {
        const F av = a[((size_t)tm1 * DP + c) * P + pair];
        smA[c * P + pair] = av;
        const size_t ro = ((size_t)(tm1 + 1) * NX + c) * N;
        g = fma(-av, Xn[ro + i] - Xn[ro + j], g);
        const unsigned long long ab = abs_bits(av);
        amax = ab > amax ? ab : amax;
      }
      const F th = thk[qb + pair];
      F tn = fma(g, F(0.5), th);
      if (sign_set(tn)) tn = F(0);
      thn[qb + pair] = tn;
      smE[pair] = fma(F(2), tn, -th);
      const unsigned long long v = abs_bits((tn - th) * from_bits(amax, F(0)));
      rb = v > rb ? v : rb;
    }
    __syncthreads();
    for (int i = tid; i < N; i += nt) {
      const F nc = F(agent_nc(D, s, i));
      F acc[DP];
#pragma unroll
      for (int c = 0; c < DP; ++c) acc[c] = nc * Xn[((size_t)(tm1 + 1) * NX + c) * N + i];
      for_partners(D, s, i, [&](int pair, bool first) {
        F e = smE[pair];
        if (!first) e = -e;
#pragma unroll
        for (int c = 0; c < DP; ++c) acc[c] = fma(e, smA[c * P + pair], acc[c]);
      });
#pragma unroll
      for (int c = 0; c < DP; ++c) h[((size_t)tm1 * DP + c) * N + i] = acc[c];
    }
    __syncthreads();
  }
}

// Maximum of a non-negative bit-ordered value over the CTA; every thread
// receives the result.  Contains two barriers.
__device__ __forceinline__ unsigned long long block_max1(unsigned long long a, unsigned long long* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long oa = __shfl_xor_sync(0xffffffffu, a, o);
    a = oa > a ? oa : a;
  }
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = a;
  __syncthreads();
  a = 0;
  for (int k = 0; k < nw; ++k) a = red[k] > a ? red[k] : a;
  __syncthreads();
  return a;
}

// Shared-memory scratch of one scenario CTA.
struct CtaScratch {
  unsigned long long red[32];
  unsigned long long cnt[2];
  int flag;
};

// Every ADMM iteration of scenario `sc` on one CTA (Sec. III.B): x-update of
// all agents, consensus/dual update with the primal residual, the dual residual
// when the primal test passes (or on the last iteration), convergence test,
// then the aggregate coupling term of the next x-update.  Writes status,
// iterations, residuals, work counters and the levels of the final iterate.
template <typename F, int NX, int NU, int DP, bool DI>
__device__ void run_scenario(const Dev<F>& D, const Model<F, NX, NU>& M, const ScenMeta& s, int sc,
                             CtaScratch& cs, F* sm, int sm_pairs, F* kcs) {
  const bool fused = sm != nullptr && s.P <= sm_pairs;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) {
    cs.flag = 0;
    cs.cnt[0] = 0;
    cs.cnt[1] = 0;
  }
  init_phase<F, NX, NU, DP>(D, s, tid, nt);
  __syncthreads();
  int xl = 0, status = ST_NOT_CONVERGED, iters = 0, tfin = 0;
  F r = F(0), sres = F(0);
  unsigned long long neqp = 0, nfact = 0;
  for (int k = 0; k < D.max_iter; ++k) {
    const int tk = k % 3, tkp1 = (k + 1) % 3, tkm1 = (k + 2) % 3;
    const int st = xupdate_phase<F, NX, NU, DP, DI>(D, M, s, true, k, xl ^ 1, tid, nt, neqp, nfact, kcs);
    if (st) atomicMax(&cs.flag, st);
    __syncthreads();
    iters = k + 1;
    const int flag = cs.flag;
    if (flag) { status = flag; tfin = tk; break; }
    unsigned long long rb = 0;
    if (fused) pair_gather_fused<F, NX, NU, DP>(D, s, xl, tk, tkp1, sm, rb);
    else pair_phase<F, NX, NU, DP>(D, s, xl, tk, tkp1, tid, nt, rb);
    r = from_bits(block_max1(rb, cs.red), F(0));
    tfin = tkp1;
    if (!finite_(r)) { status = ST_NUMERIC; xl ^= 1; break; }
    const bool last = (k + 1 == D.max_iter);
    if (r <= F(D.tol) || last) {
      unsigned long long sb = 0;
      dual_phase<F, NX, NU, DP>(D, s, xl, tkm1, tk, tkp1, tid, nt, sb);
      sres = F(s.rho) * from_bits(block_max1(sb, cs.red), F(0));
      if (!finite_(sres)) { status = ST_NUMERIC; xl ^= 1; break; }
      if (r <= F(D.tol) && sres <= F(D.tol)) { status = ST_CONVERGED; xl ^= 1; break; }
      if (last) { xl ^= 1; break; }
    }
    if (!fused) {
      gather_phase<F, NX, NU, DP>(D, s, xl ^ 1, tkp1, tk, tid, nt);
      __syncthreads();
    }
    xl ^= 1;
  }
  if (neqp) atomicAdd(&cs.cnt[0], neqp);
  if (nfact) atomicAdd(&cs.cnt[1], nfact);
  __syncthreads();
  if (tid == 0) {
    D.status[sc] = status;
    D.iters[sc] = iters;
    D.cur_lvl[sc] = xl | (tfin << 1);
    D.res[2 * sc] = double(r);
    D.res[2 * sc + 1] = double(sres);
    D.eqp[sc] = cs.cnt[0];
    D.fact[sc] = cs.cnt[1];
    if (D.rho_out) {
      D.rho_out[sc] = s.rho;
      D.rho_chg[sc] = 0;
    }
  }
}


// ---------------------------------------------------------------------------
// Scenario groups: several same-horizon scenarios with at most 32 agents in
// total share one CTA; each lane of the x-update owns one agent of one member,
// the pair and gather sweeps run over the members' flattened units, and every
// decision (residuals, convergence, outputs) stays per scenario.
// ---------------------------------------------------------------------------
constexpr int kGroupMax = 32;
constexpr int kPairBatch = 4;  // pairs whose operands a thread loads before computing

constexpr int kGroupPairs = kGroupMax * (kGroupMax - 1) / 2;

template <typename F, int DP>
struct GroupStage {
  uint32_t pair[kGroupPairs];   // flattened agent indices fi | fj << 8 of every member pair
  uint8_t mem[kGroupPairs];     // member of every flattened pair
  F pos[DP][kGroupMax];         // positions p^{k+1} of the group's agents at the current step
  F sxs[DP][kGroupMax];         // over-relaxation: agent parts s^k of the consensus copies at that step
};

struct GroupSm {
  ScenMeta meta[kGroupMax];
  int sid[kGroupMax];
  int aoff[kGroupMax + 1];
  int poff[kGroupMax + 1];
  int active[kGroupMax];
  int flag[kGroupMax];
  int need[kGroupMax];
  unsigned long long rb[kGroupMax];  // primal residual key (unrelaxed: max |theta' - theta|, a bound)
  unsigned long long sb[kGroupMax];
  unsigned long long rx[kGroupMax];  // exact primal residual key from the lazy pass
  unsigned long long cnt[kGroupMax][2];
  double rho[kGroupMax];    // current penalty per member (residual balancing)
  double scale[kGroupMax];  // this iteration's penalty factor per member
  int rhoc[kGroupMax];      // penalty changes per member
  int adapt[kGroupMax];     // member's penalty changed this iteration
  int G, nA, nP, T, any, anyad;
};

// Member owning flattened index u given exclusive prefix sums off[0..G].
__device__ __forceinline__ int member_of(const int* off, int G, int u) {
  int m = 0;
  while (m + 1 < G && off[m + 1] <= u) ++m;
  return m;
}

// Over-relaxed consensus projection, dual update and gather of a group, step by
// step (an extension; Boyd et al. 2011, Sec. 3.4.3): the relaxed positions
// alpha p + (1 - alpha) w^k take the place of p in the projection and in the
// dual update.  The scaled duals stay y_i = -theta a, y_j = theta a, and the
// consensus copies split into w_i = s_i + phi a, w_j = s_j - phi a, with s per
// agent and step and phi per pair and step, so that one iteration reads
//   theta' = max(0, theta + (d - alpha a.(p_i - p_j) - (1 - alpha)(a.(s_i - s_j) + 2 phi)) / 2),
//   phi'   = (1 - alpha) phi + theta' - theta,   s' = alpha p + (1 - alpha) s,
//   h_i    = n_c s_i' + sum_j sigma_ij (phi' + theta') a_ij
// (alpha = 1 gives back s = p, phi' = theta' - theta).  The residuals keep the
// unrelaxed p: r = max |p - w'| = max |(1 - alpha)(p - s) -/+ phi' a| and the
// dual residual max |w' - w| = max |alpha (p - s) +/- (phi' - phi) a|, both
// formed in this sweep.
template <typename F, int NX, int DP>
__device__ void group_relaxed_sweep(const Dev<F>& D, GroupSm& gs, GroupStage<F, DP>& st, F* smE, F* smA,
                                    int my_m, int my_i, int xl, int tk, int tkp1) {
  const int tid = threadIdx.x, nt = blockDim.x, nP = gs.nP, T = gs.T;
  const F al = F(D.alpha), om = F(1.0 - D.alpha);
  const bool mine = my_m >= 0 && gs.active[my_m];
  const F* Xm = nullptr;
  F* Sm = nullptr;
  int Nm = 1;
  if (mine) {
    const ScenMeta& s = gs.meta[my_m];
    Xm = D.X + (size_t)(xl ^ 1) * D.tot_xs * NX + s.xs_off * NX;
    Sm = D.sx + s.as_off * DP;
    Nm = s.N;
  }
  for (int tm1 = 0; tm1 < T; ++tm1) {
    if (mine) {
#pragma unroll
      for (int c = 0; c < DP; ++c) {
        st.pos[c][tid] = Xm[((size_t)(tm1 + 1) * NX + c) * Nm + my_i];
        st.sxs[c][tid] = Sm[((size_t)tm1 * DP + c) * Nm + my_i];
      }
    }
    __syncthreads();
    for (int u = tid; u < nP; u += nt) {
      const int m = st.mem[u];
      if (!gs.active[m]) continue;
      const ScenMeta& s = gs.meta[m];
      const int P = s.P, pair = u - gs.poff[m];
      const size_t q = s.ps_off + (size_t)tm1 * P + pair;
      const F* a = D.a + s.ps_off * DP;
      const uint32_t fij = st.pair[u];
      const int fi = fij & 0xFF, fj = fij >> 8;
      const F th = D.theta[(size_t)tk * D.tot_ps + q];
      const F ph = D.phi[q];
      F av[DP];
      F ap = F(0), as = F(0);  // a.(p_i - p_j), a.(s_i - s_j)
#pragma unroll
      for (int c = 0; c < DP; ++c) {
        av[c] = a[((size_t)tm1 * DP + c) * P + pair];
        smA[c * nP + u] = av[c];
        ap = fma(av[c], st.pos[c][fi] - st.pos[c][fj], ap);
        as = fma(av[c], st.sxs[c][fi] - st.sxs[c][fj], as);
      }
      const F ahat = fma(al, ap, om * fma(F(2), ph, as));
      F tn = fma(F(s.d) - ahat, F(0.5), th);
      if (sign_set(tn)) tn = F(0);
      const F pn = fma(om, ph, tn - th);
      D.theta[(size_t)tkp1 * D.tot_ps + q] = tn;
      D.phi[q] = pn;
      smE[u] = pn + tn;
      const F dph = pn - ph;
      unsigned long long rv = 0, sv = 0;
#pragma unroll
      for (int c = 0; c < DP; ++c) {
        const F ei = st.pos[c][fi] - st.sxs[c][fi], ej = st.pos[c][fj] - st.sxs[c][fj];
        const unsigned long long r1 = abs_bits(fma(-pn, av[c], om * ei));
        const unsigned long long r2 = abs_bits(fma(pn, av[c], om * ej));
        const unsigned long long s1 = abs_bits(fma(dph, av[c], al * ei));
        const unsigned long long s2 = abs_bits(fma(-dph, av[c], al * ej));
        rv = r1 > rv ? r1 : rv;
        rv = r2 > rv ? r2 : rv;
        sv = s1 > sv ? s1 : sv;
        sv = s2 > sv ? s2 : sv;
      }
      if (rv > gs.rb[m]) atomicMax(&gs.rb[m], rv);
      if (sv > gs.sb[m]) atomicMax(&gs.sb[m], sv);
    }
    __syncthreads();
    if (mine) {
      const ScenMeta& s = gs.meta[my_m];
      const int N = s.N, i = my_i, base = gs.poff[my_m];
      const F nc = F(agent_nc(D, s, i));
      F sn[DP], acc[DP];
#pragma unroll
      for (int c = 0; c < DP; ++c) {
        sn[c] = fma(al, st.pos[c][tid], om * st.sxs[c][tid]);
        acc[c] = nc * sn[c];
      }
      for_partners(D, s, i, [&](int lp, bool first) {
        const int pair = base + lp;
        F e = smE[pair];
        if (!first) e = -e;
#pragma unroll
        for (int c = 0; c < DP; ++c) acc[c] = fma(e, smA[c * nP + pair], acc[c]);
      });
      F* h = D.h + s.as_off * DP;
#pragma unroll
      for (int c = 0; c < DP; ++c) {
        h[((size_t)tm1 * DP + c) * N + i] = acc[c];
        Sm[((size_t)tm1 * DP + c) * N + i] = sn[c];
      }
    }
    __syncthreads();
  }
}

// COOP_EQP: active-set rounds that serve at most CoopShape<NX>::NG agents of the
// warp take their EQP pass on lane groups (eqp_coop, the same bits as eqp_solve).
template <typename F, int NX, int NU, int DP, bool DI, bool COOP_EQP = false>
__device__ void run_group(const Dev<F>& D, const Model<F, NX, NU>& M, const int* members, int G, GroupSm& gs,
                          GroupStage<F, DP>& st, F* sm, F* kcs) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid < G) {
    const int sc = members[tid];
    gs.sid[tid] = sc;
    gs.meta[tid] = D.meta[sc];
    gs.active[tid] = 1;
    gs.flag[tid] = 0;
    gs.need[tid] = 0;
    gs.rb[tid] = 0;
    gs.sb[tid] = 0;
    gs.rx[tid] = 0;
    gs.cnt[tid][0] = 0;
    gs.cnt[tid][1] = 0;
    gs.rho[tid] = gs.meta[tid].rho;
    gs.rhoc[tid] = 0;
    gs.adapt[tid] = 0;
  }
  __syncthreads();
  if (tid == 0) {
    int a = 0, p = 0;
    for (int m = 0; m < G; ++m) {
      gs.aoff[m] = a;
      gs.poff[m] = p;
      a += gs.meta[m].N;
      p += gs.meta[m].P;
    }
    gs.aoff[G] = a;
    gs.poff[G] = p;
    gs.G = G;
    gs.nA = a;
    gs.nP = p;
    gs.T = gs.meta[0].T;
  }
  __syncthreads();
  for (int m = 0; m < G; ++m) init_phase<F, NX, NU, DP>(D, gs.meta[m], tid, nt);
  const int nA = gs.nA, nP = gs.nP, T = gs.T;
  for (int u = tid; u < nP; u += nt) {
    const int m = member_of(gs.poff, G, u);
    const int pk = D.pairs[gs.meta[m].pair_off + (u - gs.poff[m])];
    st.mem[u] = (uint8_t)m;
    st.pair[u] = (uint32_t)(gs.aoff[m] + (pk & 0xFFFF)) | ((uint32_t)(gs.aoff[m] + (pk >> 16)) << 8);
  }
  __syncthreads();
  // the lane's agent (fixed for the whole run)
  const int my_m = tid < nA ? member_of(gs.aoff, G, tid) : -1;
  const int my_i = tid < nA ? tid - gs.aoff[my_m] : 0;
  unsigned long long neqp = 0, nfact = 0;
  F* smE = sm;
  F* smA = sm + nP;
  int xl = 0;
  for (int k = 0; k < D.max_iter; ++k) {
    const int tk = k % 3, tkp1 = (k + 1) % 3, tkm1 = (k + 2) % 3;
    const bool last = (k + 1 == D.max_iter);
    const bool adapt_iter = D.adapt_every > 0 && (k + 1) % D.adapt_every == 0;
    // x-update (every lane of the warp takes part; lanes without an active agent help)
    {
      const bool has = my_m >= 0 && gs.active[my_m] != 0;
      const ScenMeta& s = gs.meta[has ? my_m : 0];
      const AgentCtx<F, NX, NU, DP> A = has ? make_agent<F, NX, NU, DP, DI>(D, M, s, my_i, xl ^ 1, kcs + tid, nt,
                                                                        gs.rho[my_m])
                                            : idle_agent<F, NX, NU, DP>(M, kcs + tid, nt, D.coop);
      const int as_max = D.as_max > 0 ? D.as_max : 10 * s.T * NU + 10;
      const F eps = D.eps_rel > 0 ? F(D.eps_rel) : (sizeof(F) == 8 ? F(1e-12) : F(1e-5));
      const int st = xupdate_agent<F, NX, NU, DP, DI, COOP_EQP>(A, has, start_kind_of(D, k), as_max, eps, neqp,
                                                                nfact);
      if (has && st) atomicMax(&gs.flag[my_m], st);
    }
    __syncthreads();
    if (tid < G && gs.active[tid] && gs.flag[tid]) {
      const int sc = gs.sid[tid];
      gs.active[tid] = 0;
      D.status[sc] = gs.flag[tid];
      D.iters[sc] = k + 1;
      D.cur_lvl[sc] = xl | (tk << 1);
    }
    __syncthreads();
    // fused consensus projection / dual update and gather, step by step; the
    // step's positions and the pair table are read from shared memory.  The
    // next step's positions, and the operands of each batch of kPairBatch
    // pairs, are loaded ahead of their use so that the load latency overlaps
    // the arithmetic.
    if (D.relax) {
      group_relaxed_sweep<F, NX, DP>(D, gs, st, smE, smA, my_m, my_i, xl, tk, tkp1);
    } else {
      const bool mine = my_m >= 0 && gs.active[my_m];
      const F* Xmine = nullptr;
      int Nmine = 1;
      F pnext[DP];
      if (mine) {
        const ScenMeta& s = gs.meta[my_m];
        Xmine = D.X + (size_t)(xl ^ 1) * D.tot_xs * NX + s.xs_off * NX;
        Nmine = s.N;
#pragma unroll
        for (int c = 0; c < DP; ++c) pnext[c] = Xmine[((size_t)NX + c) * Nmine + my_i];
      }
      for (int tm1 = 0; tm1 < T; ++tm1) {
        if (mine) {
#pragma unroll
          for (int c = 0; c < DP; ++c) st.pos[c][tid] = pnext[c];
        }
        __syncthreads();
        for (int ub = tid; ub < nP; ub += kPairBatch * nt) {
          F av[kPairBatch][DP], thv[kPairBatch];
          int mk[kPairBatch];
#pragma unroll
          for (int b = 0; b < kPairBatch; ++b) {
            const int u = ub + b * nt;
            mk[b] = -1;
            if (u < nP) {
              const int m = st.mem[u];
              if (gs.active[m]) {
                mk[b] = m;
                const ScenMeta& s = gs.meta[m];
                const int P = s.P, pair = u - gs.poff[m];
                const F* a = D.a + s.ps_off * DP;
#pragma unroll
                for (int c = 0; c < DP; ++c) av[b][c] = a[((size_t)tm1 * DP + c) * P + pair];
                thv[b] = D.theta[(size_t)tk * D.tot_ps + s.ps_off + (size_t)tm1 * P + pair];
              }
            }
          }
#pragma unroll
          for (int b = 0; b < kPairBatch; ++b) {
            if (mk[b] < 0) continue;
            const int u = ub + b * nt, m = mk[b];
            const ScenMeta& s = gs.meta[m];
            const int P = s.P, pair = u - gs.poff[m];
            const uint32_t fij = st.pair[u];
            const int fi = fij & 0xFF, fj = fij >> 8;
            F g = F(s.d);  // d - a'(p_i - p_j)
#pragma unroll
            for (int c = 0; c < DP; ++c) {
              const F avc = av[b][c];
              smA[c * nP + u] = avc;
              g = fma(-avc, st.pos[c][fi] - st.pos[c][fj], g);
            }
            const F th = thv[b];
            F tn = fma(g, F(0.5), th);
            if (sign_set(tn)) tn = F(0);
            D.theta[(size_t)tkp1 * D.tot_ps + s.ps_off + (size_t)tm1 * P + pair] = tn;
            smE[u] = fma(F(2), tn, -th);
            // max |theta' - theta| bounds the primal residual r = max |(theta' - theta) a_c|
            // (|a| = 1): r <= it <= sqrt(dp) r; the exact r is formed in the lazy pass
            const unsigned long long v = abs_bits(tn - th);
            if (v > gs.rb[m]) atomicMax(&gs.rb[m], v);
          }
        }
        __syncthreads();
        if (mine && tm1 + 1 < T) {
#pragma unroll
          for (int c = 0; c < DP; ++c) pnext[c] = Xmine[((size_t)(tm1 + 2) * NX + c) * Nmine + my_i];
        }
        if (mine) {
          const ScenMeta& s = gs.meta[my_m];
          const int N = s.N, i = my_i, base = gs.poff[my_m];
          F acc[DP];
#pragma unroll
          for (int c = 0; c < DP; ++c) acc[c] = F(agent_nc(D, s, i)) * st.pos[c][tid];
          for_partners(D, s, i, [&](int lp, bool first) {
            const int pair = base + lp;
            F e = smE[pair];
            if (!first) e = -e;
#pragma unroll
            for (int c = 0; c < DP; ++c) acc[c] = fma(e, smA[c * nP + pair], acc[c]);
          });
          F* h = D.h + s.as_off * DP;
#pragma unroll
          for (int c = 0; c < DP; ++c) h[((size_t)tm1 * DP + c) * N + i] = acc[c];
        }
        __syncthreads();
      }
    }
    // primal residual tests on the bound, then the exact primal and the dual
    // residual in a lazy pass only where they decide (the over-relaxed sweep has
    // formed both exactly)
    if (tid < G) {
      gs.need[tid] = 0;
      if (gs.active[tid]) {
        const F r = from_bits(gs.rb[tid], F(0));
        if (!finite_(r)) {
          const int sc = gs.sid[tid];
          gs.active[tid] = 0;
          D.status[sc] = ST_NUMERIC;
          D.iters[sc] = k + 1;
          D.cur_lvl[sc] = (xl ^ 1) | (tkp1 << 1);
          D.res[2 * sc] = double(r);
        } else if ((D.relax ? r <= F(D.tol) : r <= F(2) * F(D.tol)) || last || adapt_iter) {
          // unrelaxed: the bound max |dtheta| is at most sqrt(dp) < 2 times the exact r,
          // so every scenario whose exact r may pass the test takes the lazy pass
          gs.need[tid] = 1;
        }
      }
    }
    __syncthreads();
    if (tid == 0) {
      int any = 0;
      for (int m = 0; m < G; ++m) any |= gs.need[m];
      gs.any = any;
    }
    __syncthreads();
    if (gs.any && !D.relax) {
      for (int tm1 = 0; tm1 < T; ++tm1) {
        for (int u = tid; u < nP; u += nt) {
          const int m = st.mem[u];
          if (!gs.need[m]) continue;
          const ScenMeta& s = gs.meta[m];
          unsigned long long sb = 0, rx = 0;
          dual_phase<F, NX, NU, DP>(D, s, xl, tkm1, tk, tkp1, (int64_t)tm1 * s.P + (u - gs.poff[m]),
                                    (int64_t)s.P * s.T, sb, &rx);
          if (sb > gs.sb[m]) atomicMax(&gs.sb[m], sb);
          if (rx > gs.rx[m]) atomicMax(&gs.rx[m], rx);
        }
      }
      __syncthreads();
    }
    if (tid < G && gs.active[tid]) {
      const int sc = gs.sid[tid];
      const F r = from_bits((gs.need[tid] && !D.relax) ? gs.rx[tid] : gs.rb[tid], F(0));
      D.res[2 * sc] = double(r);
      if (gs.need[tid]) {
        const F sres = F(gs.rho[tid]) * from_bits(gs.sb[tid], F(0));
        D.res[2 * sc + 1] = double(sres);
        int stop = 0, status = ST_NOT_CONVERGED;
        if (!finite_(sres)) { stop = 1; status = ST_NUMERIC; }
        else if (r <= F(D.tol) && sres <= F(D.tol)) { stop = 1; status = ST_CONVERGED; }
        else if (last) stop = 1;
        if (stop) {
          gs.active[tid] = 0;
          D.status[sc] = status;
          D.iters[sc] = k + 1;
          D.cur_lvl[sc] = (xl ^ 1) | (tkp1 << 1);
        } else if (adapt_iter) {
          // residual balancing (Boyd et al. 2011, Sec. 3.4.1)
          double scale = 1.0;
          if (double(r) > D.adapt_mu * double(sres)) scale = D.adapt_tau;
          else if (double(sres) > D.adapt_mu * double(r)) scale = 1.0 / D.adapt_tau;
          if (scale != 1.0) {
            gs.adapt[tid] = 1;
            gs.scale[tid] = scale;
            gs.rho[tid] *= scale;
            gs.rhoc[tid] += 1;
          }
        }
      }
      gs.rb[tid] = 0;
      gs.sb[tid] = 0;
      gs.rx[tid] = 0;
    }
    __syncthreads();
    if (tid == 0) {
      int any = 0, anyad = 0;
      for (int m = 0; m < G; ++m) {
        any |= gs.active[m];
        anyad |= gs.adapt[m];
      }
      gs.any = any;
      gs.anyad = anyad;
    }
    __syncthreads();
    if (gs.anyad) {
      // rho changed by `scale` for the flagged members: the scaled duals
      // become theta^{k+1} / scale; the previous slot is set to
      // theta^k - theta^{k+1} + theta^{k+1} / scale so that the consensus
      // copies w (and the next dual residual) are unchanged; then the
      // aggregate h of the next x-update is formed again, and every stage is
      // refactorized (the Hessian holds rho)
      for (int tm1 = 0; tm1 < T; ++tm1) {
        for (int u = tid; u < nP; u += nt) {
          const int m = st.mem[u];
          if (!gs.adapt[m]) continue;
          const ScenMeta& s = gs.meta[m];
          const int P = s.P, pair = u - gs.poff[m];
          const size_t q = s.ps_off + (size_t)tm1 * P + pair;
          F* const t1p = D.theta + (size_t)tkp1 * D.tot_ps + q;
          F* const t0p = D.theta + (size_t)tk * D.tot_ps + q;
          const F th1 = *t1p, th0 = *t0p;
          const F t1 = th1 / F(gs.scale[m]);
          *t1p = t1;
          if (D.relax) {
            // w = s + phi a does not hold theta: only the duals change
            smE[u] = D.phi[q] + t1;
          } else {
            const F t0 = (th0 - th1) + t1;
            *t0p = t0;
            smE[u] = fma(F(2), t1, -t0);
          }
          const F* a = D.a + s.ps_off * DP;
#pragma unroll
          for (int c = 0; c < DP; ++c) smA[c * nP + u] = a[((size_t)tm1 * DP + c) * P + pair];
        }
        __syncthreads();
        if (my_m >= 0 && gs.adapt[my_m]) {
          const ScenMeta& s = gs.meta[my_m];
          const int N = s.N, i = my_i, base = gs.poff[my_m];
          const F* Xn = D.X + (size_t)(xl ^ 1) * D.tot_xs * NX + s.xs_off * NX;
          const F* Sx = D.relax ? D.sx + s.as_off * DP : nullptr;
          F acc[DP];
#pragma unroll
          for (int c = 0; c < DP; ++c)
            acc[c] = F(agent_nc(D, s, i)) * (D.relax ? Sx[((size_t)tm1 * DP + c) * N + i]
                                                     : Xn[((size_t)(tm1 + 1) * NX + c) * N + i]);
          for_partners(D, s, i, [&](int lp, bool first) {
            const int pair = base + lp;
            F e = smE[pair];
            if (!first) e = -e;
#pragma unroll
            for (int c = 0; c < DP; ++c) acc[c] = fma(e, smA[c * nP + pair], acc[c]);
          });
          F* h = D.h + s.as_off * DP;
#pragma unroll
          for (int c = 0; c < DP; ++c) h[((size_t)tm1 * DP + c) * N + i] = acc[c];
        }
        __syncthreads();
      }
      if (my_m >= 0 && gs.adapt[my_m]) {
        const ScenMeta& s = gs.meta[my_m];
        for (int t = 0; t < s.T; ++t) D.Cm[s.as_off + (size_t)t * s.N + my_i] = 0xFFFF;
      }
      __syncthreads();
      if (tid < G) gs.adapt[tid] = 0;
      __syncthreads();
    }
    xl ^= 1;
    if (!gs.any) break;
  }
  if (my_m >= 0) {
    if (neqp) atomicAdd(&gs.cnt[my_m][0], neqp);
    if (nfact) atomicAdd(&gs.cnt[my_m][1], nfact);
  }
  __syncthreads();
  if (tid < G) {
    if (D.rho_out) {
      D.rho_out[gs.sid[tid]] = gs.rho[tid];
      D.rho_chg[gs.sid[tid]] = gs.rhoc[tid];
    }
    D.eqp[gs.sid[tid]] = gs.cnt[tid][0];
    D.fact[gs.sid[tid]] = gs.cnt[tid][1];
  }
  __syncthreads();
}

}  // namespace tadmm
