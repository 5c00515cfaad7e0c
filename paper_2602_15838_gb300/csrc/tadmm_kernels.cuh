// Kernels and host launchers of the batched ADMM path, templated on the
// arithmetic type F and the dimensions (NX, NU, DP).
#pragma once

#include <algorithm>
#include <cstring>

#include "tadmm_impl.h"

namespace tadmm {

// ---------------------------------------------------------------------------
// Batched persistent kernel: each CTA repeatedly takes the next scenario group
// (same-horizon scenarios of at most 32 agents in total, or one larger
// scenario) from a work queue, largest estimated work first, and runs every
// ADMM iteration of it on-chip, phases separated by CTA barriers.
// ---------------------------------------------------------------------------
// Register-budget variants of the persistent kernel (chosen by the autotuner):
// (max threads per CTA, min resident CTAs per SM) for __launch_bounds__.
// Variant 0, with no register cap, also runs small active-set rounds on lane
// groups (COOP_EQP of run_group); the results are the same bits either way.
template <int V> struct KVariant;
template <> struct KVariant<0> { static constexpr int maxt = 256, minb = 1; };
template <> struct KVariant<1> { static constexpr int maxt = 32, minb = 12; };
template <> struct KVariant<2> { static constexpr int maxt = 64, minb = 8; };
constexpr int kNumVariants = 3;

template <typename F, int NX, int NU, int DP, int V, bool DI>
__global__ void __launch_bounds__(KVariant<V>::maxt, KVariant<V>::minb) k_batched(Dev<F> D) {
  __shared__ Model<F, NX, NU> M;
  __shared__ CtaScratch cs;
  __shared__ GroupSm gs;
  __shared__ GroupStage<F, DP> gst;
  __shared__ int s_q;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  // dynamic shared memory: agent constants [KC][threads], then the pair staging
  F* kcs = (F*)dyn_smem;
  F* sm = D.sm_pairs > 0 ? kcs + AgentConst<NX, NU>::KC * blockDim.x : nullptr;
  load_model<F, NX, NU>(M, D.model);
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_q = atomicAdd(D.queue, 1);
    __syncthreads();
    const int qi = s_q;
    if (qi >= D.n_groups) return;
    const int g = D.order[qi];
    const int b0 = D.goff[g], G = D.goff[g + 1] - b0;
    if (G == 1 && !(D.single_as_group && D.meta[D.gmem[b0]].N <= kGroupMax)) {
      const int sc = D.gmem[b0];
      const ScenMeta s = D.meta[sc];
      run_scenario<F, NX, NU, DP, DI>(D, M, s, sc, cs, sm, D.sm_pairs, kcs);
    } else {
      run_group<F, NX, NU, DP, DI, (V == 0)>(D, M, D.gmem + b0, G, gs, gst, sm, kcs);
    }
  }
}

// ---------------------------------------------------------------------------
// Plain mode: one scenario, one launch per phase, host reads the residuals.
// ---------------------------------------------------------------------------
template <typename F, int NX, int NU, int DP>
__global__ void k_init(Dev<F> D, int sc) {
  const ScenMeta s = D.meta[sc];
  init_phase<F, NX, NU, DP>(D, s, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                            (int64_t)gridDim.x * blockDim.x);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    D.eqp[sc] = 0;
    D.fact[sc] = 0;
  }
}

template <typename F, int NX, int NU, int DP, bool DI, bool HOMO = false>
// One warp per CTA; lanes 0..apw-1 own agents blockIdx.x * apw + lane, the
// other lanes help with their refactorizations.  HOMO: homotopy hot start.
__global__ void __launch_bounds__(32) k_xupdate(Dev<F> D, int sc, int k, int lvl_out, int32_t* flag, int apw) {
  __shared__ Model<F, NX, NU> M;
  __shared__ F kcs[AgentConst<NX, NU>::KC * 32];
  load_model<F, NX, NU>(M, D.model);
  __syncthreads();
  const ScenMeta s = D.meta[sc];
  const bool owns = (int)threadIdx.x < apw;
  const int i = blockIdx.x * apw + threadIdx.x;
  unsigned long long neqp = 0, nfact = 0;
  const int st = xupdate_phase<F, NX, NU, DP, DI, true, HOMO>(D, M, s, owns, k, lvl_out, i, s.N, neqp, nfact, kcs);
  if (st && owns && i < s.N) atomicMax(flag, st);
  if (neqp) atomicAdd(&D.eqp[sc], neqp);
  if (nfact) atomicAdd(&D.fact[sc], nfact);
}

template <typename F, int NX, int NU, int DP>
__global__ void __launch_bounds__(256) k_pair(Dev<F> D, int sc, int xl, int tk, int tkp1, unsigned long long* red1) {
  __shared__ unsigned long long red[32];
  const ScenMeta s = D.meta[sc];
  unsigned long long rb = 0;
  pair_phase<F, NX, NU, DP>(D, s, xl, tk, tkp1, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                            (int64_t)gridDim.x * blockDim.x, rb);
  rb = block_max1(rb, red);
  if (threadIdx.x == 0 && rb) atomicMax(red1, rb);
}

template <typename F, int NX, int NU, int DP>
__global__ void __launch_bounds__(256) k_dual(Dev<F> D, int sc, int xl, int tkm1, int tk, int tkp1,
                                              unsigned long long* red1) {
  __shared__ unsigned long long red[32];
  const ScenMeta s = D.meta[sc];
  unsigned long long sb = 0;
  dual_phase<F, NX, NU, DP>(D, s, xl, tkm1, tk, tkp1, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                            (int64_t)gridDim.x * blockDim.x, sb);
  sb = block_max1(sb, red);
  if (threadIdx.x == 0 && sb) atomicMax(red1, sb);
}

// One warp per (block of 32 agents, step): grid (ceil(N / 32), T), 32 threads.
template <typename F, int NX, int NU, int DP>
__global__ void __launch_bounds__(32) k_gather(Dev<F> D, int sc, int xl_new, int tkp1, int tk) {
  __shared__ GatherTile<F, DP> ts;
  const ScenMeta s = D.meta[sc];
  gather_tile<F, NX, NU, DP>(D, s, xl_new, tkp1, tk, blockIdx.x * 32, blockIdx.y, ts);
}

template <typename F>
__global__ void k_finish(Dev<F> D, int sc, int status, int iters, int cur, double r, double sres) {
  D.status[sc] = status;
  D.iters[sc] = iters;
  D.cur_lvl[sc] = cur;
  D.res[2 * sc] = r;
  D.res[2 * sc + 1] = sres;
}

// ---------------------------------------------------------------------------
// Graph mode: every phase is a grid-wide kernel over all scenarios' units and
// one CUDA graph with a conditional WHILE node repeats the iteration on the
// device until every scenario has stopped (no host round trip per iteration).
// Scenario k's iteration parity fixes its levels: X level (k & 1) holds p^k,
// theta slot k % 3 holds theta^k.
// ---------------------------------------------------------------------------
struct GState {
  int32_t* iter;
  int32_t* active;
  int32_t* need;
  int32_t* fail;
  unsigned long long* rb;
  unsigned long long* sb;
};

__device__ __forceinline__ void scen_max(unsigned long long* arr, int sc, unsigned long long v, bool valid) {
  const unsigned full = __activemask();
  const int lead_sc = __shfl_sync(full, sc, __ffs(full) - 1);
  if (__all_sync(full, valid && sc == lead_sc)) {
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long w = __shfl_xor_sync(full, v, o);
      v = w > v ? w : v;
    }
    if ((threadIdx.x & 31) == __ffs(full) - 1 && v) atomicMax(&arr[sc], v);
  } else if (valid && v) {
    atomicMax(&arr[sc], v);
  }
}

template <typename F, int NX, int NU, int DP>
__global__ void k_g_init(Dev<F> D, GState G) {
  const int sc = blockIdx.x;
  const ScenMeta s = D.meta[sc];
  init_phase<F, NX, NU, DP>(D, s, threadIdx.x, blockDim.x);
  if (threadIdx.x == 0) {
    G.iter[sc] = 0;
    G.active[sc] = 1;
    G.need[sc] = 0;
    G.fail[sc] = 0;
    G.rb[sc] = 0;
    G.sb[sc] = 0;
    D.eqp[sc] = 0;
    D.fact[sc] = 0;
    D.status[sc] = ST_NOT_CONVERGED;
    D.iters[sc] = 0;
  }
}

template <typename F, int NX, int NU, int DP, bool DI, bool HOMO = false>
__global__ void __launch_bounds__(32) k_g_xupdate(Dev<F> D, GState G, const int32_t* __restrict__ agent_scen,
                                                   int64_t tot_agents, int apw) {
  __shared__ Model<F, NX, NU> M;
  __shared__ F kcs[AgentConst<NX, NU>::KC * 32];
  load_model<F, NX, NU>(M, D.model);
  __syncthreads();
  const int64_t ga = (int64_t)blockIdx.x * apw + threadIdx.x;
  // every lane of the warp takes part in the x-update; lanes past apw, past
  // the last agent or of a stopped scenario only help
  const bool owns = (int)threadIdx.x < apw && ga < tot_agents;
  const int sc = owns ? agent_scen[ga] : 0;
  const bool in_scen = owns && G.active[sc];
  const ScenMeta s = D.meta[sc];
  const int i = (int)(ga - s.agent_off), k = G.iter[sc];
  unsigned long long neqp = 0, nfact = 0;
  const int st =
      xupdate_phase<F, NX, NU, DP, DI, true, HOMO>(D, M, s, in_scen, k, (k + 1) & 1, i, s.N, neqp, nfact, kcs);
  if (!in_scen) return;
  if (st) atomicMax(&G.fail[sc], st);
  if (neqp) atomicAdd(&D.eqp[sc], neqp);
  if (nfact) atomicAdd(&D.fact[sc], nfact);
}

template <typename F, int NX, int NU, int DP>
__global__ void __launch_bounds__(128) k_g_pair(Dev<F> D, GState G, const int32_t* __restrict__ pair_scen,
                                                int64_t tot_pairs) {
  const int64_t gp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int tm1 = blockIdx.y;
  int sc = 0;
  bool valid = gp < tot_pairs;
  if (valid) sc = pair_scen[gp];
  ScenMeta s;
  if (valid) {
    s = D.meta[sc];
    valid = tm1 < s.T && G.active[sc] && !G.fail[sc];
  }
  unsigned long long rb = 0;
  if (valid) {
    const int k = G.iter[sc];
    const int64_t q = (int64_t)tm1 * s.P + (gp - s.pair_off);
    pair_phase<F, NX, NU, DP>(D, s, k & 1, k % 3, (k + 1) % 3, q, (int64_t)s.P * s.T, rb);
  }
  scen_max(G.rb, sc, rb, valid);
}

template <typename F>
__global__ void k_g_check1(Dev<F> D, GState G) {
  for (int sc = blockIdx.x * blockDim.x + threadIdx.x; sc < D.n_scen; sc += gridDim.x * blockDim.x) {
    G.need[sc] = 0;
    if (!G.active[sc] || G.fail[sc]) continue;
    const F r = from_bits(G.rb[sc], F(0));
    if (finite_(r) && (r <= F(D.tol) || G.iter[sc] + 1 == D.max_iter)) G.need[sc] = 1;
  }
}

template <typename F, int NX, int NU, int DP>
__global__ void __launch_bounds__(128) k_g_dual(Dev<F> D, GState G, const int32_t* __restrict__ pair_scen,
                                                int64_t tot_pairs) {
  const int64_t gp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int tm1 = blockIdx.y;
  int sc = 0;
  bool valid = gp < tot_pairs;
  if (valid) sc = pair_scen[gp];
  ScenMeta s;
  if (valid) {
    s = D.meta[sc];
    valid = tm1 < s.T && G.need[sc];
  }
  unsigned long long sb = 0;
  if (valid) {
    const int k = G.iter[sc];
    const int64_t q = (int64_t)tm1 * s.P + (gp - s.pair_off);
    dual_phase<F, NX, NU, DP>(D, s, k & 1, (k + 2) % 3, k % 3, (k + 1) % 3, q, (int64_t)s.P * s.T, sb);
  }
  scen_max(G.sb, sc, sb, valid);
}

// Convergence decisions (in the arithmetic type F), then the WHILE condition.
template <typename F>
__global__ void k_g_check2(Dev<F> D, GState G, cudaGraphConditionalHandle cond) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  int mine = 0;
  for (int sc = threadIdx.x; sc < D.n_scen; sc += blockDim.x) {
    if (!G.active[sc]) continue;
    const int k = G.iter[sc];
    const double rho = D.meta[sc].rho;
    int stop = 0, status = ST_NOT_CONVERGED, cur = ((k + 1) & 1) | (((k + 1) % 3) << 1);
    const F r = from_bits(G.rb[sc], F(0));
    if (G.fail[sc]) {
      stop = 1;
      status = G.fail[sc];
      cur = (k & 1) | ((k % 3) << 1);
    } else if (!finite_(r)) {
      stop = 1;
      status = ST_NUMERIC;
    } else if (G.need[sc]) {
      const F sres = F(rho) * from_bits(G.sb[sc], F(0));
      D.res[2 * sc + 1] = double(sres);
      if (!finite_(sres)) { stop = 1; status = ST_NUMERIC; }
      else if (r <= F(D.tol) && sres <= F(D.tol)) { stop = 1; status = ST_CONVERGED; }
      else if (k + 1 == D.max_iter) stop = 1;
    }
    D.res[2 * sc] = double(r);
    D.iters[sc] = k + 1;
    if (stop) {
      G.active[sc] = 0;
      D.status[sc] = status;
      D.cur_lvl[sc] = cur;
    } else {
      G.iter[sc] = k + 1;
      mine = 1;
    }
    G.rb[sc] = 0;
    G.sb[sc] = 0;
  }
  if (mine) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) cudaGraphSetConditional(cond, any ? 1u : 0u);
}

// One warp per (scenario, block of 32 agents, step): blk[b] = (scenario, first agent).
template <typename F, int NX, int NU, int DP>
__global__ void __launch_bounds__(32) k_g_gather(Dev<F> D, GState G, const int2* __restrict__ blk) {
  __shared__ GatherTile<F, DP> ts;
  const int2 b = blk[blockIdx.x];
  const int sc = b.x;
  if (!G.active[sc]) return;
  const ScenMeta s = D.meta[sc];
  const int tm1 = blockIdx.y;
  if (tm1 >= s.T) return;
  const int k1 = G.iter[sc];  // already advanced: levels of iterate k1 = k + 1
  gather_tile<F, NX, NU, DP>(D, s, k1 & 1, k1 % 3, (k1 + 2) % 3, b.y, tm1, ts);
}

// ---------------------------------------------------------------------------
// Import (caller layouts, float64) and export kernels
// ---------------------------------------------------------------------------
template <typename F>
__global__ void k_convert(const double* __restrict__ src, F* __restrict__ dst, int64_t n) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    dst[k] = F(src[k]);
}

// a: caller [pair-step][dp] (pair-major, then t) -> internal [T][DP][P]
template <typename F, int DP>
__global__ void k_import_a(const ScenMeta* __restrict__ meta, const int32_t* __restrict__ pair_scen,
                           const double* __restrict__ src, F* __restrict__ dst, int64_t tot_pairs) {
  for (int64_t gp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gp < tot_pairs;
       gp += (int64_t)gridDim.x * blockDim.x) {
    const ScenMeta s = meta[pair_scen[gp]];
    const int lp = (int)(gp - s.pair_off);
    for (int t = 0; t < s.T; ++t)
#pragma unroll
      for (int c = 0; c < DP; ++c)
        dst[s.ps_off * DP + ((size_t)t * DP + c) * s.P + lp] = F(src[(s.ps_off + (int64_t)lp * s.T + t) * DP + c]);
  }
}

// Re-linearization of the collision constraints around the final iterate of
// the last solve (one outer step of a sequential-QP loop over the halfspace
// linearization of Sec. III): a_ijt = (p_it - p_jt) / |p_it - p_jt| from that iterate's
// positions, unchanged where the two positions coincide.  Formed in float64
// with correctly rounded operations (no contraction), as in the oracle.
template <typename F, int NX, int DP>
__global__ void k_relin_a(Dev<F> D, F* __restrict__ a_out, const int32_t* __restrict__ pair_scen,
                          int64_t tot_pairs, const uint8_t* __restrict__ keep) {
  const int64_t gp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int tm1 = blockIdx.y;
  if (gp >= tot_pairs) return;
  const int sc = pair_scen[gp];
  if (keep && keep[sc]) return;
  const ScenMeta s = D.meta[sc];
  if (tm1 >= s.T) return;
  const int lp = (int)(gp - s.pair_off);
  const int pk = D.pairs[s.pair_off + lp];
  const int i = pk & 0xFFFF, j = pk >> 16;
  const F* X = D.X + (size_t)(D.cur_lvl[sc] & 1) * D.tot_xs * NX + s.xs_off * NX;
  double dd[DP];
#pragma unroll
  for (int c = 0; c < DP; ++c) {
    const size_t ro = ((size_t)(tm1 + 1) * NX + c) * s.N;
    dd[c] = __dadd_rn(double(X[ro + i]), -double(X[ro + j]));
  }
  double n2 = __dmul_rn(dd[0], dd[0]);
#pragma unroll
  for (int c = 1; c < DP; ++c) n2 = __dadd_rn(n2, __dmul_rn(dd[c], dd[c]));
  if (!(n2 > 0.0)) return;
  const double nr = __dsqrt_rn(n2);
#pragma unroll
  for (int c = 0; c < DP; ++c) a_out[s.ps_off * DP + ((size_t)tm1 * DP + c) * s.P + lp] = F(__ddiv_rn(dd[c], nr));
}

// The next solve's initial consensus positions: the final iterate's positions.
template <typename F, int NX, int DP>
__global__ void k_relin_w0(Dev<F> D, F* __restrict__ w0_out, const int32_t* __restrict__ agent_scen,
                           int64_t tot_agents, const uint8_t* __restrict__ keep) {
  const int64_t ga = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (ga >= tot_agents) return;
  const int sc = agent_scen[ga];
  if (keep && keep[sc]) return;
  const ScenMeta s = D.meta[sc];
  const int i = (int)(ga - s.agent_off);
  const F* X = D.X + (size_t)(D.cur_lvl[sc] & 1) * D.tot_xs * NX + s.xs_off * NX;
  for (int tm1 = 0; tm1 < s.T; ++tm1)
#pragma unroll
    for (int c = 0; c < DP; ++c)
      w0_out[s.as_off * DP + ((size_t)tm1 * DP + c) * s.N + i] = X[((size_t)(tm1 + 1) * NX + c) * s.N + i];
}

// Termination test of a sequential-QP loop over the linearization (the rule of
// Sec. V.A: relative objective change and collision-free at every step), one
// CTA per scenario at the final iterate of the last solve: J = the objective of
// Eq. (1), every agent's sum over t < T of (x_t - x_ref)' Q (x_t - x_ref) +
// u_t' R u_t plus (x_T - x_ref)' Q_T (x_T - x_ref), and dmin = the smallest
// |p_it - p_jt| over the coupled pairs and t = 1..T (+inf without pairs).  In
// float64 with a fixed reduction order, so repeated calls agree bit for bit.
template <typename F, int NX, int NU, int DP>
__global__ void __launch_bounds__(256) k_sqp_measure(Dev<F> D, double* __restrict__ J, double* __restrict__ dmin) {
  constexpr int NT = 256;
  __shared__ double rs[NT], rm[NT];
  const int sc = blockIdx.x;
  const ScenMeta s = D.meta[sc];
  const int N = s.N, T = s.T;
  const F* X = D.X + (size_t)(D.cur_lvl[sc] & 1) * D.tot_xs * NX + s.xs_off * NX;
  const F* U = D.U + s.as_off * NU;
  double acc = 0.0;
  for (int64_t e = threadIdx.x; e < (int64_t)N * (T + 1); e += NT) {
    const int i = (int)(e % N), t = (int)(e / N);
    const int64_t ga = s.agent_off + i;
    const F* w = (t < T ? D.Qd : D.Qfd) + ga * NX;
#pragma unroll
    for (int r = 0; r < NX; ++r) {
      const double d = __dadd_rn(double(X[((size_t)t * NX + r) * N + i]), -double(D.x_ref[ga * NX + r]));
      acc = __dadd_rn(acc, __dmul_rn(double(w[r]), __dmul_rn(d, d)));
    }
    if (t < T)
#pragma unroll
      for (int c = 0; c < NU; ++c) {
        const double u = double(U[((size_t)t * NU + c) * N + i]);
        acc = __dadd_rn(acc, __dmul_rn(double(D.Rd[ga * NU + c]), __dmul_rn(u, u)));
      }
  }
  double mn = __longlong_as_double(0x7FF0000000000000ll);  // +inf
  for (int64_t e = threadIdx.x; e < (int64_t)s.P * T; e += NT) {
    const int lp = (int)(e % s.P), tm1 = (int)(e / s.P);
    const int pk = D.pairs[s.pair_off + lp];
    const int i = pk & 0xFFFF, j = pk >> 16;
    double n2 = 0.0;
#pragma unroll
    for (int c = 0; c < DP; ++c) {
      const size_t ro = ((size_t)(tm1 + 1) * NX + c) * N;
      const double d = __dadd_rn(double(X[ro + i]), -double(X[ro + j]));
      n2 = __dadd_rn(n2, __dmul_rn(d, d));
    }
    mn = fmin(mn, __dsqrt_rn(n2));
  }
  rs[threadIdx.x] = acc;
  rm[threadIdx.x] = mn;
  __syncthreads();
  for (int w = NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      rs[threadIdx.x] = __dadd_rn(rs[threadIdx.x], rs[threadIdx.x + w]);
      rm[threadIdx.x] = fmin(rm[threadIdx.x], rm[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    J[sc] = rs[0];
    dmin[sc] = rm[0];
  }
}

// w0: caller [agent-step][dp] (agent-major, then t) -> internal [T][DP][N]
template <typename F, int DP>
__global__ void k_import_w0(const ScenMeta* __restrict__ meta, const int32_t* __restrict__ agent_scen,
                            const double* __restrict__ src, F* __restrict__ dst, int64_t tot_agents) {
  for (int64_t ga = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ga < tot_agents;
       ga += (int64_t)gridDim.x * blockDim.x) {
    const ScenMeta s = meta[agent_scen[ga]];
    const int i = (int)(ga - s.agent_off);
    for (int t = 0; t < s.T; ++t)
#pragma unroll
      for (int c = 0; c < DP; ++c)
        dst[s.as_off * DP + ((size_t)t * DP + c) * s.N + i] = F(src[(s.as_off + (int64_t)i * s.T + t) * DP + c]);
  }
}

template <typename F, int NX, int NU>
__global__ void k_export_agents(Dev<F> D, const int32_t* __restrict__ agent_scen, int64_t tot_agents,
                                double* X, double* U, int8_t* W) {
  for (int64_t ga = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ga < tot_agents;
       ga += (int64_t)gridDim.x * blockDim.x) {
    const int sc = agent_scen[ga];
    const ScenMeta s = D.meta[sc];
    const int i = (int)(ga - s.agent_off), N = s.N, T = s.T;
    const F* Xl = D.X + (size_t)(D.cur_lvl[sc] & 1) * D.tot_xs * NX + s.xs_off * NX;
    if (X)
      for (int t = 0; t <= T; ++t)
#pragma unroll
        for (int r = 0; r < NX; ++r)
          X[(s.xs_off + (int64_t)i * (T + 1) + t) * NX + r] = double(Xl[((size_t)t * NX + r) * N + i]);
    for (int t = 0; t < T; ++t) {
      const uint16_t m = D.Wm[s.as_off + (size_t)t * N + i];
#pragma unroll
      for (int c = 0; c < NU; ++c) {
        const int64_t o = (s.as_off + (int64_t)i * T + t) * NU + c;
        if (U) U[o] = double(D.U[s.as_off * NU + ((size_t)t * NU + c) * N + i]);
        if (W) W[o] = (m & (1u << c)) ? 1 : ((m & (0x100u << c)) ? 2 : 0);
      }
    }
  }
}

template <typename F>
__global__ void k_export_theta(Dev<F> D, const int32_t* __restrict__ pair_scen, int64_t tot_pairs, double* th) {
  for (int64_t gp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gp < tot_pairs;
       gp += (int64_t)gridDim.x * blockDim.x) {
    const int sc = pair_scen[gp];
    const ScenMeta s = D.meta[sc];
    const int lp = (int)(gp - s.pair_off);
    const F* tl = D.theta + (size_t)(D.cur_lvl[sc] >> 1) * D.tot_ps + s.ps_off;
    for (int t = 0; t < s.T; ++t) th[s.ps_off + (int64_t)lp * s.T + t] = double(tl[(size_t)t * s.P + lp]);
  }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
template <typename F>
static Dev<F> make_dev(tadmm_handle* h) {
  Dev<F> D{};
  std::memset(&D, 0, sizeof(D));
  D.meta = h->meta;
  D.pairs = h->pairs;
  D.model = (const F*)h->model;
  D.Qd = (const F*)h->Qd;
  D.Rd = (const F*)h->Rd;
  D.Qfd = (const F*)h->Qfd;
  D.x_init = (const F*)h->x_init;
  D.x_ref = (const F*)h->x_ref;
  D.a = (const F*)h->a;
  D.w0 = (const F*)h->w0;
  D.theta = (F*)h->theta;
  D.X = (F*)h->X;
  D.h = (F*)h->h;
  D.U = (F*)h->U;
  D.Us = (F*)h->Us;
  D.Wm = h->Wm;
  D.Cm = h->Cm;
  D.cache = (F*)h->cache;
  D.tot_ps = h->tot_ps;
  D.tot_xs = h->tot_xs;
  D.n_scen = h->n_scen;
  D.status = h->status;
  D.iters = h->iters;
  D.cur_lvl = h->cur_lvl;
  D.res = h->res;
  D.eqp = h->eqp;
  D.fact = h->fact;
  D.queue = h->queue;
  D.start_mode = h->opt.start_mode;
  D.goff = h->goff;
  D.gmem = h->gmem;
  D.n_groups = h->n_groups;
  D.order = h->gorder;
  D.as_max = h->opt.as_max;
  D.eps_rel = h->opt.eps_rel;
  D.single_as_group = (h->opt.flags & (TADMM_FLAG_NO_GROUPING | TADMM_FLAG_NO_FUSED_PAIR_GATHER)) ? 0 : 1;
  D.coop = (h->opt.flags & TADMM_FLAG_NO_LANE_GROUPS) ? 0 : 1;
  D.adapt_every = h->opt.adapt_every;
  D.adapt_mu = h->opt.adapt_mu;
  D.adapt_tau = h->opt.adapt_tau;
  D.relax = h->opt.relax_alpha != 1.0 ? 1 : 0;
  D.alpha = h->opt.relax_alpha;
  D.phi = (F*)h->phi;
  D.models = (const F*)h->models;
  D.sx = (F*)h->sx;
  D.rho_out = h->rho_out;
  D.rho_chg = h->rho_chg;
  D.deg = h->deg;
  D.adj_ptr = h->adj_ptr;
  D.adj = h->adj;
  D.hprev = (F*)h->hprev;
  D.mu = (F*)h->hmu;
  D.dmu = (F*)h->hdmu;
  return D;
}

// Host decoding of a residual maximum from its bit-ordered key (see ord_bits).
template <typename F>
static double host_decode_bits(unsigned long long b);
template <>
double host_decode_bits<double>(unsigned long long b) {
  double v;
  std::memcpy(&v, &b, 8);
  return v;
}
template <>
double host_decode_bits<float>(unsigned long long b) {
  const uint32_t b32 = (uint32_t)b;
  float v;
  std::memcpy(&v, &b32, 4);
  return v;
}
template <>
double host_decode_bits<df64>(unsigned long long b) {
  const uint32_t h32 = (uint32_t)(b >> 32), k = (uint32_t)b;
  const uint32_t l32 = (k & 0x80000000u) ? (k ^ 0x80000000u) : ~k;
  float hi, lo;
  std::memcpy(&hi, &h32, 4);
  std::memcpy(&lo, &l32, 4);
  return (double)hi + (double)lo;
}

static inline int grid_for(int64_t n, int threads, int cap = 65535) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

template <typename F, int NX, int NU, int DP>
int Impl<F, NX, NU, DP>::import_inputs(tadmm_handle* h, cudaStream_t st) {
  const int nm = NX * NX + NX * NU + 2 * NU;
  k_convert<F><<<1, 128, 0, st>>>(h->st_model, (F*)h->model, nm);
  const int64_t na = h->tot_agents;
  k_convert<F><<<grid_for(na * NX, 256), 256, 0, st>>>(h->st_agent + 0 * na * NX, (F*)h->Qd, na * NX);
  k_convert<F><<<grid_for(na * NU, 256), 256, 0, st>>>(h->st_agent + 1 * na * NX, (F*)h->Rd, na * NU);
  k_convert<F><<<grid_for(na * NX, 256), 256, 0, st>>>(h->st_agent + 1 * na * NX + na * NU, (F*)h->Qfd, na * NX);
  k_convert<F><<<grid_for(na * NX, 256), 256, 0, st>>>(h->st_agent + 2 * na * NX + na * NU, (F*)h->x_init, na * NX);
  k_convert<F><<<grid_for(na * NX, 256), 256, 0, st>>>(h->st_agent + 3 * na * NX + na * NU, (F*)h->x_ref, na * NX);
  if (h->tot_pairs > 0)
    k_import_a<F, DP><<<grid_for(h->tot_pairs, 256), 256, 0, st>>>(h->meta, h->pair_scen, h->st_a, (F*)h->a,
                                                                    h->tot_pairs);
  k_import_w0<F, DP><<<grid_for(na, 128), 128, 0, st>>>(h->meta, h->agent_scen, h->st_w0, (F*)h->w0, na);
  if (h->hetero)
    k_convert<F><<<grid_for(na * nm, 256), 256, 0, st>>>(h->st_models, (F*)h->models, na * nm);
  return cuda_check(cudaGetLastError(), "import kernels");
}

// Conversion of the per-agent cost arrays alone (bit 0 Qd, 1 Rd, 2 Qfd, 3 x_ref)
// from their float64 staging into the arithmetic type.
template <typename F, int NX, int NU, int DP>
int Impl<F, NX, NU, DP>::import_costs(tadmm_handle* h, int which, cudaStream_t st) {
  const int64_t na = h->tot_agents;
  if (which & 1) k_convert<F><<<grid_for(na * NX, 256), 256, 0, st>>>(h->st_agent, (F*)h->Qd, na * NX);
  if (which & 2) k_convert<F><<<grid_for(na * NU, 256), 256, 0, st>>>(h->st_agent + na * NX, (F*)h->Rd, na * NU);
  if (which & 4)
    k_convert<F><<<grid_for(na * NX, 256), 256, 0, st>>>(h->st_agent + na * NX + na * NU, (F*)h->Qfd, na * NX);
  if (which & 8)
    k_convert<F><<<grid_for(na * NX, 256), 256, 0, st>>>(h->st_agent + 3 * na * NX + na * NU, (F*)h->x_ref, na * NX);
  return cuda_check(cudaGetLastError(), "cost import kernels");
}

template <typename F, int NX, int NU, int DP>
int Impl<F, NX, NU, DP>::relinearize(tadmm_handle* h, const uint8_t* keep, cudaStream_t st) {
  Dev<F> D = make_dev<F>(h);
  int tmax = 0;
  for (const ScenMeta& m : h->meta_h) tmax = std::max(tmax, m.T);
  if (h->tot_pairs > 0)
    k_relin_a<F, NX, DP><<<dim3(grid_for(h->tot_pairs, 128, 1 << 30), tmax), 128, 0, st>>>(D, (F*)h->a, h->pair_scen,
                                                                                          h->tot_pairs, keep);
  k_relin_w0<F, NX, DP><<<grid_for(h->tot_agents, 128, 1 << 30), 128, 0, st>>>(D, (F*)h->w0, h->agent_scen,
                                                                              h->tot_agents, keep);
  return cuda_check(cudaGetLastError(), "relinearization kernels");
}

template <typename F, int NX, int NU, int DP>
int Impl<F, NX, NU, DP>::sqp_measure(tadmm_handle* h, double* J, double* dmin, cudaStream_t st) {
  k_sqp_measure<F, NX, NU, DP><<<h->n_scen, 256, 0, st>>>(make_dev<F>(h), J, dmin);
  return cuda_check(cudaGetLastError(), "objective kernel");
}

template <typename F, int NX, int NU, int DP>
static const void* batched_kernel(int v, bool di) {
  if (di) {
    switch (v) {
      case 1: return (const void*)k_batched<F, NX, NU, DP, 1, true>;
      case 2: return (const void*)k_batched<F, NX, NU, DP, 2, true>;
      default: return (const void*)k_batched<F, NX, NU, DP, 0, true>;
    }
  }
  switch (v) {
    case 1: return (const void*)k_batched<F, NX, NU, DP, 1, false>;
    case 2: return (const void*)k_batched<F, NX, NU, DP, 2, false>;
    default: return (const void*)k_batched<F, NX, NU, DP, 0, false>;
  }
}

static int variant_maxt(int v) {
  switch (v) {
    case 1: return KVariant<1>::maxt;
    case 2: return KVariant<2>::maxt;
    default: return KVariant<0>::maxt;
  }
}

// Dynamic shared memory of the fused pair/gather staging: (DP + 1) values per
// pair of the largest scenario, if that fits the per-CTA budget; otherwise per
// pair of the largest group that runs the group path (at most 32 agents), the
// larger scenarios then taking the unfused sweeps.
template <typename F, int DP>
static size_t fused_smem_bytes(const tadmm_handle* h, int* pairs_out) {
  int pmax = h->max_group_pairs;
  for (const ScenMeta& m : h->meta_h) pmax = std::max(pmax, m.P);
  const size_t budget = 96 * 1024;
  if ((size_t)(DP + 1) * pmax * sizeof(F) > budget) pmax = h->max_group_pairs;
  const size_t bytes = (size_t)(DP + 1) * pmax * sizeof(F);
  if ((h->opt.flags & TADMM_FLAG_NO_FUSED_PAIR_GATHER) || pmax == 0 || bytes > budget) {
    if (pairs_out) *pairs_out = 0;
    return 0;
  }
  if (pairs_out) *pairs_out = pmax;
  return bytes;
}

// Dynamic shared memory of the per-thread agent constants.
template <typename F, int NX, int NU>
static size_t agent_const_bytes(int tpc) {
  return (size_t)AgentConst<NX, NU>::KC * tpc * sizeof(F);
}

template <typename F, int NX, int NU, int DP>
int Impl<F, NX, NU, DP>::max_ctas_per_sm(int tpc, int variant, const tadmm_handle* h) {
  int n = 0;
  if (tpc > variant_maxt(variant)) return 0;
  const size_t smem = (h ? fused_smem_bytes<F, DP>(h, nullptr) : 0) + agent_const_bytes<F, NX, NU>(tpc);
  const void* kfn = batched_kernel<F, NX, NU, DP>(variant, h ? h->di != 0 : false);
  if (smem > 48 * 1024) cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kfn, tpc, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <typename F, int NX, int NU, int DP>
int Impl<F, NX, NU, DP>::solve_batched(tadmm_handle* h, double tol, int max_iter, cudaStream_t st) {
  const int var = (h->variant >= 0 && h->variant < kNumVariants) ? h->variant : 0;
  int tpc = h->tpc > 0 ? h->tpc : std::min(128, variant_maxt(var));
  const int occ = max_ctas_per_sm(tpc, var, h);
  if (occ < 1) return set_error(TADMM_EINVAL, "launch shape does not fit the kernel variant");
  int cps = h->cps > 0 ? std::min(h->cps, occ) : occ;
  const int grid = std::max(1, std::min(h->n_groups, h->sm_count * cps));
  if (!h->gexec || h->g_tol != tol || h->g_iter != max_iter || h->g_tpc != tpc || h->g_cps != cps ||
      h->g_var != var) {
    if (h->gexec) {
      cudaGraphExecDestroy(h->gexec);
      h->gexec = nullptr;
    }
    Dev<F> D = make_dev<F>(h);
    D.tol = tol;
    D.max_iter = max_iter;
    int smp = 0;
    const size_t smem = fused_smem_bytes<F, DP>(h, &smp) + agent_const_bytes<F, NX, NU>(tpc);
    D.sm_pairs = smp;
    cudaGraph_t g = nullptr;
    int rc = cuda_check(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (rc) return rc;
    cudaMemsetAsync(h->queue, 0, sizeof(int32_t), h->cap_stream);
    void* args[] = {&D};
    cudaLaunchKernel(batched_kernel<F, NX, NU, DP>(var, h->di != 0), dim3(grid), dim3(tpc), args, smem, h->cap_stream);
    cudaError_t le = cudaGetLastError();
    cudaError_t ee = cudaStreamEndCapture(h->cap_stream, &g);
    if (le != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_check(le, "batched kernel launch"); }
    if ((rc = cuda_check(ee, "end capture"))) return rc;
    rc = cuda_check(cudaGraphInstantiate(&h->gexec, g, 0), "graph instantiate");
    cudaGraphDestroy(g);
    if (rc) return rc;
    h->g_tol = tol;
    h->g_iter = max_iter;
    h->g_tpc = tpc;
    h->g_cps = cps;
    h->g_var = var;
  }
  h->launches = 1;
  return cuda_check(cudaGraphLaunch(h->gexec, st), "graph launch");
}

// Agents per warp of the per-phase x-update kernels: at most one per lane
// group of the cooperative passes (CoopShape<NX>::NG: 8 in 2D, 4 in 3D), and
// fewer, down to one, when there are not enough agents to give every SM four
// warps.  Each of an SM's four sub-partitions issues FP64 instructions at its
// own fixed rate whatever the number of active lanes, so a small agent count
// (one large scenario) is spread over four warps per SM, one per
// sub-partition, rather than packed into fewer warps; every owner can take its
// EQP passes and refactorizations on a lane group.
template <int NX>
static int agents_per_warp(int64_t agents, int sm_count) {
  int apw = CoopShape<NX>::NG;
  while (apw > 1 && (int64_t)apw * sm_count * 4 > agents) apw /= 2;
  return apw;
}

template <typename F, int NX, int NU, int DP>
int Impl<F, NX, NU, DP>::solve_plain(tadmm_handle* h, double tol, int max_iter, cudaStream_t st) {
  Dev<F> D = make_dev<F>(h);
  D.tol = tol;
  D.max_iter = max_iter;
  unsigned long long* hb = (unsigned long long*)h->pinned;  // [0] flag, [1] r bits, [2] s bits
  int64_t launches = 0;
  const bool homo = h->opt.start_mode == TADMM_START_HOMOTOPY;
  for (int sc = 0; sc < h->n_scen; ++sc) {
    const ScenMeta& s = h->meta_h[sc];
    const int64_t PT = (int64_t)s.P * s.T, NT = (int64_t)s.N * s.T;
    const int apw = agents_per_warp<NX>(s.N, h->sm_count);
    k_init<F, NX, NU, DP><<<grid_for(std::max(PT, NT), 256, 4096), 256, 0, st>>>(D, sc);
    ++launches;
    int xl = 0, status = ST_NOT_CONVERGED, iters = 0, tfin = 0;
    double r = 0, sres = 0;
    auto read_bits = [&](unsigned long long b, double rho_scale) -> double {
      return rho_scale * host_decode_bits<F>(b);
    };
    for (int k = 0; k < max_iter; ++k) {
      const int tk = k % 3, tkp1 = (k + 1) % 3, tkm1 = (k + 2) % 3;
      cudaMemsetAsync(h->flag, 0, sizeof(int32_t), st);
      cudaMemsetAsync(h->red2, 0, 2 * sizeof(unsigned long long), st);
      if (h->di)
        if (homo)
          k_xupdate<F, NX, NU, DP, true, true><<<(s.N + apw - 1) / apw, 32, 0, st>>>(D, sc, k, xl ^ 1, h->flag, apw);
        else
          k_xupdate<F, NX, NU, DP, true><<<(s.N + apw - 1) / apw, 32, 0, st>>>(D, sc, k, xl ^ 1, h->flag, apw);
      else
        if (homo)
          k_xupdate<F, NX, NU, DP, false, true><<<(s.N + apw - 1) / apw, 32, 0, st>>>(D, sc, k, xl ^ 1, h->flag, apw);
        else
          k_xupdate<F, NX, NU, DP, false><<<(s.N + apw - 1) / apw, 32, 0, st>>>(D, sc, k, xl ^ 1, h->flag, apw);
      k_pair<F, NX, NU, DP><<<grid_for(PT, 256, h->sm_count * 8), 256, 0, st>>>(D, sc, xl, tk, tkp1, h->red2);
      launches += 2;
      cudaMemcpyAsync(hb, h->flag, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
      cudaMemcpyAsync(hb + 1, h->red2, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
      int rc = cuda_check(cudaStreamSynchronize(st), "plain-mode residual readback");
      if (rc) return rc;
      iters = k + 1;
      const int flag = (int)(*(int32_t*)hb);
      if (flag) { status = flag; tfin = tk; break; }
      // the residual tests are taken in the arithmetic type F
      r = read_bits(hb[1], 1.0);
      tfin = tkp1;
      if (!std::isfinite(r)) { status = ST_NUMERIC; xl ^= 1; break; }
      const bool last = (k + 1 == max_iter);
      const bool r_ok = (sizeof(F) == 8) ? (r <= tol) : (float(r) <= float(tol));  // in the type F
      if (r_ok || last) {
        k_dual<F, NX, NU, DP><<<grid_for(PT, 256, h->sm_count * 8), 256, 0, st>>>(D, sc, xl, tkm1, tk, tkp1,
                                                                                h->red2 + 1);
        ++launches;
        cudaMemcpyAsync(hb + 2, h->red2 + 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
        if ((rc = cuda_check(cudaStreamSynchronize(st), "plain-mode dual residual readback"))) return rc;
        sres = read_bits(hb[2], s.rho);
        if (!std::isfinite(sres)) { status = ST_NUMERIC; xl ^= 1; break; }
        const bool s_ok = (sizeof(F) == 8) ? (sres <= tol) : (float(sres) <= float(tol));
        if (r_ok && s_ok) { status = ST_CONVERGED; xl ^= 1; break; }
        if (last) { xl ^= 1; break; }
      }
      k_gather<F, NX, NU, DP><<<dim3((s.N + 31) / 32, s.T), 32, 0, st>>>(D, sc, xl ^ 1, tkp1, tk);
      ++launches;
      xl ^= 1;
    }
    const int cur = xl | (tfin << 1);
    k_finish<F><<<1, 1, 0, st>>>(D, sc, status, iters, cur, r, sres);
    ++launches;
  }
  h->launches = launches;
  return cuda_check(cudaGetLastError(), "plain-mode launches");
}

template <typename F, int NX, int NU, int DP>
int Impl<F, NX, NU, DP>::solve_graph(tadmm_handle* h, double tol, int max_iter, cudaStream_t st) {
  int rc;
  if (!h->gs_iter) {
    const size_t n = (size_t)h->n_scen;
    if (cudaMalloc(&h->gs_iter, 4 * n) != cudaSuccess || cudaMalloc(&h->gs_active, 4 * n) != cudaSuccess ||
        cudaMalloc(&h->gs_need, 4 * n) != cudaSuccess || cudaMalloc(&h->gs_fail, 4 * n) != cudaSuccess ||
        cudaMalloc(&h->gs_rb, 8 * n) != cudaSuccess || cudaMalloc(&h->gs_sb, 8 * n) != cudaSuccess) {
      cudaGetLastError();
      return set_error(TADMM_ENOMEM, "graph-mode state allocation failed");
    }
  }
  if (!h->gs_blk) {
    // gather blocks: (scenario, first agent) for every 32 agents of every scenario
    std::vector<int32_t> blk;
    for (int sc = 0; sc < h->n_scen; ++sc)
      for (int i0 = 0; i0 < h->meta_h[sc].N; i0 += 32) {
        blk.push_back(sc);
        blk.push_back(i0);
      }
    h->n_gblk = (int)(blk.size() / 2);
    if (cudaMalloc(&h->gs_blk, 4 * std::max<size_t>(blk.size(), 2)) != cudaSuccess) {
      cudaGetLastError();
      return set_error(TADMM_ENOMEM, "graph-mode state allocation failed");
    }
    if ((rc = cuda_check(cudaMemcpy(h->gs_blk, blk.data(), 4 * blk.size(), cudaMemcpyHostToDevice),
                         "graph-mode gather table")))
      return rc;
  }
  GState G{(int32_t*)h->gs_iter, (int32_t*)h->gs_active, (int32_t*)h->gs_need, (int32_t*)h->gs_fail,
           (unsigned long long*)h->gs_rb, (unsigned long long*)h->gs_sb};
  Dev<F> D = make_dev<F>(h);
  const bool homo = h->opt.start_mode == TADMM_START_HOMOTOPY;
  D.tol = tol;
  D.max_iter = max_iter;
  int tmax = 0;
  for (const ScenMeta& m : h->meta_h) tmax = std::max(tmax, m.T);
  if (!h->wexec || h->w_tol != tol || h->w_iter != max_iter) {
    if (h->wexec) {
      cudaGraphExecDestroy(h->wexec);
      h->wexec = nullptr;
    }
    cudaGraph_t g = nullptr;
    if ((rc = cuda_check(cudaGraphCreate(&g, 0), "graph create"))) return rc;
    cudaGraphConditionalHandle cond;
    if ((rc = cuda_check(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault), "cond handle"))) {
      cudaGraphDestroy(g);
      return rc;
    }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if ((rc = cuda_check(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp), "conditional node"))) {
      cudaGraphDestroy(g);
      return rc;
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((rc = cuda_check(cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0,
                                                       cudaStreamCaptureModeThreadLocal), "body capture"))) {
      cudaGraphDestroy(g);
      return rc;
    }
    const int gapw = agents_per_warp<NX>(h->tot_agents, h->sm_count);
    const dim3 gx((unsigned)((h->tot_agents + gapw - 1) / gapw));
    const dim3 gp(grid_for(h->tot_pairs, 128, 1 << 30), tmax);
    const dim3 gg(h->n_gblk, tmax);
    if (h->di)
      if (homo)
        k_g_xupdate<F, NX, NU, DP, true, true><<<gx, 32, 0, h->cap_stream>>>(D, G, h->agent_scen, h->tot_agents, gapw);
      else
        k_g_xupdate<F, NX, NU, DP, true><<<gx, 32, 0, h->cap_stream>>>(D, G, h->agent_scen, h->tot_agents, gapw);
    else
      if (homo)
        k_g_xupdate<F, NX, NU, DP, false, true><<<gx, 32, 0, h->cap_stream>>>(D, G, h->agent_scen, h->tot_agents, gapw);
      else
        k_g_xupdate<F, NX, NU, DP, false><<<gx, 32, 0, h->cap_stream>>>(D, G, h->agent_scen, h->tot_agents, gapw);
    if (h->tot_pairs > 0) k_g_pair<F, NX, NU, DP><<<gp, 128, 0, h->cap_stream>>>(D, G, h->pair_scen, h->tot_pairs);
    k_g_check1<F><<<grid_for(h->n_scen, 128), 128, 0, h->cap_stream>>>(D, G);
    if (h->tot_pairs > 0) k_g_dual<F, NX, NU, DP><<<gp, 128, 0, h->cap_stream>>>(D, G, h->pair_scen, h->tot_pairs);
    k_g_check2<F><<<1, 1024, 0, h->cap_stream>>>(D, G, cond);
    k_g_gather<F, NX, NU, DP><<<gg, 32, 0, h->cap_stream>>>(D, G, (const int2*)h->gs_blk);
    cudaError_t le = cudaGetLastError();
    cudaError_t ee = cudaStreamEndCapture(h->cap_stream, &body);
    if (le != cudaSuccess || ee != cudaSuccess) {
      cudaGraphDestroy(g);
      return cuda_check(le != cudaSuccess ? le : ee, "graph body capture");
    }
    rc = cuda_check(cudaGraphInstantiate(&h->wexec, g, 0), "graph instantiate");
    cudaGraphDestroy(g);
    if (rc) return rc;
    h->w_tol = tol;
    h->w_iter = max_iter;
  }
  k_g_init<F, NX, NU, DP><<<h->n_scen, 128, 0, st>>>(D, G);
  if ((rc = cuda_check(cudaGetLastError(), "graph-mode init"))) return rc;
  h->launches = 1;
  return cuda_check(cudaGraphLaunch(h->wexec, st), "graph launch");
}

template <typename F, int NX, int NU, int DP>
int Impl<F, NX, NU, DP>::export_solution(tadmm_handle* h, double* X, double* U, double* theta, int8_t* W,
                                         cudaStream_t st) {
  Dev<F> D = make_dev<F>(h);
  if (X || U || W)
    k_export_agents<F, NX, NU><<<grid_for(h->tot_agents, 128), 128, 0, st>>>(D, h->agent_scen, h->tot_agents,
                                                                              X, U, W);
  if (theta && h->tot_pairs > 0)
    k_export_theta<F><<<grid_for(h->tot_pairs, 128), 128, 0, st>>>(D, h->pair_scen, h->tot_pairs, theta);
  return cuda_check(cudaGetLastError(), "export kernels");
}


}  // namespace tadmm

#include "tadmm_adjoint.cuh"

namespace tadmm {

// Scratch of the backward pass and the polishing rounds (grown on demand) and
// the device view of it; gX_dev / gout_dev may be null (polishing).
template <typename F, int NX, int NU, int DP>
static int bwd_prepare(tadmm_handle* h, double theta_eps, const double* gX_dev, double* gout_dev, BwdDev<F>& B,
                       std::vector<BwdScen>& bs) {
  const int64_t na = h->tot_agents;
  int tmax = 0;
  for (const ScenMeta& m : h->meta_h) tmax = std::max(tmax, m.T);
  auto grow = [&](void** p, size_t& cap, size_t bytes) -> int {
    if (bytes <= cap && *p) return TADMM_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    cap = 0;
    if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
      cudaGetLastError();
      return set_error(TADMM_ENOMEM, "backward scratch allocation failed");
    }
    cap = bytes;
    return TADMM_OK;
  };
  int64_t psi_total = 0;
  bs.assign(h->n_scen, BwdScen{});
  for (int s = 0; s < h->n_scen; ++s) {
    const ScenMeta& m = h->meta_h[s];
    bs[s].psi_off = psi_total;
    psi_total += (int64_t)m.N * m.T * m.T * DP * DP;
  }
  int rc;
  BwdBufs& b = h->bwd;
  const int64_t ps1 = std::max<int64_t>(h->tot_ps, 1);
  if ((rc = grow(&b.act, b.act_cap, 4 * ps1)) || (rc = grow(&b.piv, b.piv_cap, 4 * ps1)) ||
      (rc = grow(&b.hmask, b.hmask_cap, ps1)) || (rc = grow(&b.Wb, b.Wb_cap, 2 * h->tot_as)) ||
      (rc = grow(&b.pchg, b.pchg_cap, 4 * h->n_scen)) || (rc = grow(&b.ndep, b.ndep_cap, 4 * h->n_scen)) ||
      (rc = grow(&b.cnt, b.cnt_cap, 4 * h->n_scen)) || (rc = grow(&b.amask, b.amask_cap, 8 * na)) ||
      (rc = grow(&b.psi, b.psi_cap, sizeof(F) * std::max<int64_t>(psi_total, 1))) ||
      (rc = grow(&b.kks, b.kks_cap, sizeof(F) * na * DP * tmax * NU)) ||
      (rc = grow(&b.pos0, b.pos0_cap, sizeof(F) * h->tot_as * DP)) ||
      (rc = grow(&b.force, b.force_cap, sizeof(F) * h->tot_as * DP)) ||
      (rc = grow(&b.Xp, b.Xp_cap, sizeof(F) * h->tot_xs * NX)) || (rc = grow(&b.Up, b.Up_cap, sizeof(F) * h->tot_as * NU)) ||
      (rc = grow(&b.Wx, b.Wx_cap, sizeof(F) * h->tot_xs * NX)) || (rc = grow(&b.Wu, b.Wu_cap, sizeof(F) * h->tot_as * NU)) ||
      (rc = grow(&b.bstat, b.bstat_cap, 4 * h->n_scen)) || (rc = grow(&b.bs, b.bs_cap, sizeof(BwdScen) * h->n_scen)))
    return rc;
  std::memset(&B, 0, sizeof(B));
  B.act = (int32_t*)b.act;
  B.act_cnt = (int32_t*)b.cnt;
  B.amask = (unsigned long long*)b.amask;
  B.psi = (F*)b.psi;
  B.kks = (F*)b.kks;
  B.pos0 = (F*)b.pos0;
  B.force = (F*)b.force;
  B.Xp = (F*)b.Xp;
  B.Up = (F*)b.Up;
  B.Wx = (F*)b.Wx;
  B.Wu = (F*)b.Wu;
  B.gX = gX_dev;
  if (gout_dev) {
    B.gQ = gout_dev;
    B.gQf = gout_dev + na * NX;
    B.gR = gout_dev + 2 * na * NX;
    B.gGoal = gout_dev + 2 * na * NX + na * NU;
  }
  B.bstatus = (int32_t*)b.bstat;
  B.piv = (int32_t*)b.piv;
  B.ndep = (int32_t*)b.ndep;
  B.hmask = (uint8_t*)b.hmask;
  B.Wb = (uint16_t*)b.Wb;
  B.pchg = (int32_t*)b.pchg;
  B.theta_eps = theta_eps;
  // pivots of S below this fraction of its largest diagonal entry are rounding
  // noise of an exactly dependent row (about m eps in float64, m eps_32 in float32)
  B.rank_tol = std::is_same<F, float>::value ? 1e-6 : 1e-12;
  B.kk_stride = (int64_t)tmax * NU;
  B.adjoint = 1;
  return TADMM_OK;
}

// Active list of the current set, its sizes, then k_bwd_main (one CTA per scenario).
template <typename F, int NX, int NU, int DP>
static int bwd_solve(tadmm_handle* h, BwdDev<F>& B, std::vector<BwdScen>& bs, cudaStream_t st) {
  Dev<F> D = make_dev<F>(h);
  BwdBufs& b = h->bwd;
  int rc;
  k_bwd_count<F, NX, NU, DP><<<h->n_scen, 32, 0, st>>>(D, B);
  if ((rc = cuda_check(cudaGetLastError(), "backward count launch"))) return rc;
  std::vector<int32_t> cnt(h->n_scen);
  if ((rc = cuda_check(cudaMemcpyAsync(cnt.data(), b.cnt, 4 * h->n_scen, cudaMemcpyDeviceToHost, st), "counts")) ||
      (rc = cuda_check(cudaStreamSynchronize(st), "backward count sync")))
    return rc;
  int64_t s_total = 0, v_total = 0;
  for (int s = 0; s < h->n_scen; ++s) {
    bs[s].m = cnt[s];
    bs[s].s_off = s_total;
    bs[s].v_off = v_total;
    s_total += 2 * (int64_t)cnt[s] * cnt[s];   // S, then the normal matrix of a rank-deficient S
    v_total += 3 * (int64_t)cnt[s];
  }
  auto grow = [&](void** p, size_t& cap, size_t bytes) -> int {
    if (bytes <= cap && *p) return TADMM_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    cap = 0;
    if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
      cudaGetLastError();
      return set_error(TADMM_ENOMEM, "backward scratch allocation failed");
    }
    cap = bytes;
    return TADMM_OK;
  };
  if ((rc = grow(&b.S, b.S_cap, sizeof(F) * std::max<int64_t>(s_total, 1))) ||
      (rc = grow(&b.vec, b.vec_cap, sizeof(F) * std::max<int64_t>(v_total, 1))))
    return rc;
  B.S = (F*)b.S;
  B.vec = (F*)b.vec;
  B.bs = (const BwdScen*)b.bs;
  if ((rc = cuda_check(cudaMemcpyAsync(b.bs, bs.data(), sizeof(BwdScen) * h->n_scen, cudaMemcpyHostToDevice, st),
                       "backward sizes")))
    return rc;
  if (h->di)
    k_bwd_main<F, NX, NU, DP, true><<<h->n_scen, 128, 0, st>>>(D, B);
  else
    k_bwd_main<F, NX, NU, DP, false><<<h->n_scen, 128, 0, st>>>(D, B);
  return cuda_check(cudaGetLastError(), "backward launch");
}

template <typename F, int NX, int NU, int DP>
int Impl<F, NX, NU, DP>::backward(tadmm_handle* h, const double* gX_dev, double theta_eps, double* gout_dev,
                                  double* xpol_dev, cudaStream_t st) {
  BwdDev<F> B;
  std::vector<BwdScen> bs;
  int rc;
  if ((rc = bwd_prepare<F, NX, NU, DP>(h, theta_eps, gX_dev, gout_dev, B, bs))) return rc;
  B.adjoint = gX_dev != nullptr;   // without a loss gradient: the polished point only
  Dev<F> D = make_dev<F>(h);
  if (!h->bwd_polished) {   // the active set of the last solve's final iterate
    k_bwd_init<F, NX, NU, DP><<<h->n_scen, 128, 0, st>>>(D, B);
    if ((rc = cuda_check(cudaGetLastError(), "backward init launch"))) return rc;
  }
  if ((rc = bwd_solve<F, NX, NU, DP>(h, B, bs, st))) return rc;
  if (xpol_dev) k_bwd_export_x<F><<<grid_for(h->tot_xs * NX, 256), 256, 0, st>>>(B.Xp, h->tot_xs * NX, xpol_dev);
  return cuda_check(cudaGetLastError(), "backward export");
}

template <typename F, int NX, int NU, int DP>
int Impl<F, NX, NU, DP>::polish(tadmm_handle* h, double theta_eps, int max_rounds, double kkt_tol, uint8_t* act_dev,
                                int8_t* W_dev, int32_t* status, int32_t* rounds, cudaStream_t st) {
  BwdDev<F> B;
  std::vector<BwdScen> bs;
  int rc;
  if ((rc = bwd_prepare<F, NX, NU, DP>(h, theta_eps, nullptr, nullptr, B, bs))) return rc;
  B.adjoint = 0;
  B.kkt_tol = kkt_tol;
  Dev<F> D = make_dev<F>(h);
  k_bwd_init<F, NX, NU, DP><<<h->n_scen, 128, 0, st>>>(D, B);
  if ((rc = cuda_check(cudaGetLastError(), "polish init launch"))) return rc;
  h->bwd_polished = 1;
  std::vector<int32_t> chg(h->n_scen, 1), bst(h->n_scen, 0);
  int done_rounds = 0;
  for (int r = 0; r < max_rounds; ++r) {
    if ((rc = bwd_solve<F, NX, NU, DP>(h, B, bs, st))) return rc;
    if (h->di)
      k_bwd_polish<F, NX, NU, DP, true><<<h->n_scen, 128, 0, st>>>(D, B);
    else
      k_bwd_polish<F, NX, NU, DP, false><<<h->n_scen, 128, 0, st>>>(D, B);
    if ((rc = cuda_check(cudaGetLastError(), "polish launch"))) return rc;
    if ((rc = cuda_check(cudaMemcpyAsync(chg.data(), h->bwd.pchg, 4 * h->n_scen, cudaMemcpyDeviceToHost, st),
                         "polish flags")) ||
        (rc = cuda_check(cudaMemcpyAsync(bst.data(), h->bwd.bstat, 4 * h->n_scen, cudaMemcpyDeviceToHost, st),
                         "polish status")) ||
        (rc = cuda_check(cudaStreamSynchronize(st), "polish sync")))
      return rc;
    done_rounds = r + 1;
    bool any = false;
    for (int s = 0; s < h->n_scen; ++s) any = any || chg[s];
    if (!any) break;
  }
  if (status)
    for (int s = 0; s < h->n_scen; ++s)
      status[s] = bst[s] == ST_NUMERIC ? ST_NUMERIC : (chg[s] ? ST_NOT_CONVERGED : ST_CONVERGED);
  if (rounds) *rounds = done_rounds;
  if (act_dev || W_dev) {
    k_bwd_export_set<F><<<h->n_scen, 128, 0, st>>>(D, B, NU, act_dev, W_dev);
    if ((rc = cuda_check(cudaGetLastError(), "polish export"))) return rc;
  }
  return TADMM_OK;
}

}  // namespace tadmm
