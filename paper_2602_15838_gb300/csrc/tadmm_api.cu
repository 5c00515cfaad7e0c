// C ABI of libtadmm (declared in include/tadmm.h): validation, device memory,
// input upload, dispatch to the per-precision implementations, results.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "tadmm_impl.h"

namespace tadmm {

static thread_local std::string g_err;

int set_error(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return TADMM_OK;
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return TADMM_ECUDA;
}

}  // namespace tadmm

using tadmm::cuda_check;
using tadmm::set_error;

#define TADMM_DISPATCH(h, CALL)                                                      \
  do {                                                                               \
    if ((h)->prec == 64 && (h)->nx == 4) return tadmm::Impl<double, 4, 2, 2>::CALL;  \
    if ((h)->prec == 64 && (h)->nx == 6) return tadmm::Impl<double, 6, 3, 3>::CALL;  \
    if ((h)->prec == 32 && (h)->nx == 4) return tadmm::Impl<float, 4, 2, 2>::CALL;   \
    if ((h)->prec == 32 && (h)->nx == 6) return tadmm::Impl<float, 6, 3, 3>::CALL;   \
    if ((h)->prec == 128 && (h)->nx == 4) return tadmm::Impl<tadmm::df64, 4, 2, 2>::CALL; \
    return set_error(TADMM_EINVAL, "unsupported precision / dimensions");            \
  } while (0)

// Words of the per-stage factor cache: the layout of the kernels (CacheLayout)
// for the dispatched model sizes.
static int cache_words(int nx, int nu) {
  if (nx == 4 && nu == 2) return tadmm::CacheLayout<4, 2>::E;
  if (nx == 6 && nu == 3) return tadmm::CacheLayout<6, 3>::E;
  return nx * nx + nu * nx + nu * nu + nu + nx * nu + nu;
}

// True when no element is a NaN or an infinity (all exponent bits set).  The
// check runs over chunks with no early exit inside a chunk, on the bit
// patterns, so that the compiler vectorizes it; large arrays are split over a
// few host threads.  It runs on every tadmm_create and tadmm_update (the
// halfspace normals alone are tens of millions of values).
static bool finite_range(const double* p, int64_t n) {
  constexpr uint64_t kExp = 0x7FF0000000000000ull;
  constexpr int64_t kChunk = 4096;
  for (int64_t k0 = 0; k0 < n; k0 += kChunk) {
    const int64_t k1 = std::min(n, k0 + kChunk);
    uint64_t bad = 0;
    for (int64_t k = k0; k < k1; ++k) {
      uint64_t b;
      std::memcpy(&b, p + k, sizeof(b));
      bad |= (uint64_t)((b & kExp) == kExp);
    }
    if (bad) return false;
  }
  return true;
}

static bool finite_all(const double* p, int64_t n) {
  constexpr int64_t kPerThread = (int64_t)1 << 22;
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int nt = (int)std::min<int64_t>(std::min<unsigned>(hw, 8u), (n + kPerThread - 1) / kPerThread);
  if (nt <= 1) return finite_range(p, n);
  std::vector<std::thread> pool;
  std::vector<uint8_t> ok((size_t)nt, 1);
  const int64_t per = (n + nt - 1) / nt;
  for (int t = 0; t < nt; ++t) {
    const int64_t a = t * per, b = std::min(n, a + per);
    pool.emplace_back([&, t, a, b]() { ok[(size_t)t] = b > a ? finite_range(p + a, b - a) : 1; });
  }
  for (auto& th : pool) th.join();
  for (uint8_t v : ok)
    if (!v) return false;
  return true;
}

// Host-side checks that turn bad inputs into TADMM_EINVAL before any launch.
static int validate(const tadmm_batch* b, const tadmm_handle* shape) {
  if (!b) return set_error(TADMM_EINVAL, "batch is NULL");
  if (b->n_scen < 1) return set_error(TADMM_EINVAL, "n_scen must be >= 1");
  const bool dims_ok = (b->nx == 4 && b->nu == 2 && b->dp == 2) || (b->nx == 6 && b->nu == 3 && b->dp == 3);
  if (!dims_ok) return set_error(TADMM_EINVAL, "supported (nx, nu, dp): (4, 2, 2) and (6, 3, 3)");
  if (!b->N || !b->T || !b->A || !b->B || !b->umin || !b->umax || !b->Qd || !b->Rd || !b->Qfd || !b->x_init ||
      !b->x_ref || !b->w0 || !b->d_min || !b->rho)
    return set_error(TADMM_EINVAL, "a required array pointer is NULL");
  int64_t na = 0, nps = 0, nas = 0;
  for (int s = 0; s < b->n_scen; ++s) {
    const int N = b->N[s], T = b->T[s];
    if (N < 1 || N > 32767) return set_error(TADMM_EINVAL, "scenario " + std::to_string(s) + ": N must be in [1, 32767]");
    if (T < 1 || T > 100000) return set_error(TADMM_EINVAL, "scenario " + std::to_string(s) + ": T must be in [1, 100000]");
    // the agent kernels index a scenario's per-stage arrays in 32 bits: the
    // largest is the factor cache, (T + 1) stages x at most 87 words x N agents
    if ((int64_t)(T + 1) * 87 * N >= (int64_t)1 << 31)
      return set_error(TADMM_EINVAL, "scenario " + std::to_string(s) + ": N * (T + 1) too large (per-scenario arrays over 2^31 elements)");
    if (shape && (shape->N[s] != N || shape->T[s] != T))
      return set_error(TADMM_EINVAL, "update: N/T differ from the handle");
    if (!std::isfinite(b->d_min[s])) return set_error(TADMM_EINVAL, "d_min must be finite");
    if (!(b->rho[s] > 0.0) || !std::isfinite(b->rho[s])) return set_error(TADMM_EINVAL, "rho must be > 0");
    na += N;
    nas += (int64_t)N * T;
  }
  if ((b->pair_count == nullptr) != (b->pair_ij == nullptr))
    return set_error(TADMM_EINVAL, "pair_count and pair_ij are both NULL or both set");
  {
    int64_t po = 0;
    std::vector<uint8_t> seen;
    for (int s = 0; s < b->n_scen; ++s) {
      const int64_t N = b->N[s], T = b->T[s];
      int64_t P = N * (N - 1) / 2;
      if (b->pair_count) {
        if (b->pair_count[s] < 0 || b->pair_count[s] > P)
          return set_error(TADMM_EINVAL, "scenario " + std::to_string(s) + ": pair_count out of range");
        P = b->pair_count[s];
        if (shape && shape->pair_count_h.size() && shape->pair_count_h[s] != P)
          return set_error(TADMM_EINVAL, "update: pair lists differ from the handle");
        seen.assign((size_t)(N * N), 0);
        for (int64_t k = 0; k < P; ++k) {
          const int32_t i = b->pair_ij[2 * (po + k)], j = b->pair_ij[2 * (po + k) + 1];
          if (i < 0 || j <= i || j >= N) return set_error(TADMM_EINVAL, "pair_ij entries need 0 <= i < j < N");
          if (seen[(size_t)i * N + j]++) return set_error(TADMM_EINVAL, "pair_ij lists a pair twice");
        }
      }
      po += P;
      nps += P * T;
    }
    if (shape && (shape->pair_count_h.empty() != (b->pair_count == nullptr)))
      return set_error(TADMM_EINVAL, "update: pair lists differ from the handle");
    if (shape && b->pair_ij && !std::equal(b->pair_ij, b->pair_ij + 2 * po, shape->pair_ij_h.begin()))
      return set_error(TADMM_EINVAL, "update: pair lists differ from the handle");
  }
  if (nps > 0 && !b->a) return set_error(TADMM_EINVAL, "a is NULL but the batch has pairs");
  const int nx = b->nx, nu = b->nu, dp = b->dp;
  if ((b->A_agent == nullptr) != (b->B_agent == nullptr))
    return set_error(TADMM_EINVAL, "A_agent and B_agent are both NULL or both set");
  if (shape && (shape->hetero != 0) != (b->A_agent != nullptr))
    return set_error(TADMM_EINVAL, "update: per-agent dynamics differ from the handle");
  if (b->A_agent && (!finite_all(b->A_agent, na * nx * nx) || !finite_all(b->B_agent, na * nx * nu)))
    return set_error(TADMM_EINVAL, "A_agent, B_agent must be finite");
  if (!finite_all(b->A, nx * nx) || !finite_all(b->B, nx * nu)) return set_error(TADMM_EINVAL, "A, B must be finite");
  for (int c = 0; c < nu; ++c)
    if (!std::isfinite(b->umin[c]) || !std::isfinite(b->umax[c]) || b->umin[c] > b->umax[c])
      return set_error(TADMM_EINVAL, "need finite umin <= umax");
  for (int64_t k = 0; k < na * nx; ++k) {
    if (!(b->Qd[k] >= 0.0) || !std::isfinite(b->Qd[k]) || !(b->Qfd[k] >= 0.0) || !std::isfinite(b->Qfd[k]))
      return set_error(TADMM_EINVAL, "Q and Qf diagonals must be finite and >= 0");
  }
  for (int64_t k = 0; k < na * nu; ++k)
    if (!(b->Rd[k] > 0.0) || !std::isfinite(b->Rd[k])) return set_error(TADMM_EINVAL, "R diagonal must be finite and > 0");
  if (!finite_all(b->x_init, na * nx) || !finite_all(b->x_ref, na * nx))
    return set_error(TADMM_EINVAL, "x_init and x_ref must be finite");
  if (!finite_all(b->w0, nas * dp)) return set_error(TADMM_EINVAL, "w0 must be finite");
  if (nps > 0 && !finite_all(b->a, nps * dp)) return set_error(TADMM_EINVAL, "a must be finite");
  return TADMM_OK;
}

// True when A = [[I, dt I], [0, I]] and B = [[b1 I], [b2 I]] exactly, the
// pattern the structured kernel path assumes.
static bool is_double_integrator(const tadmm_batch* b) {
  const int nx = b->nx, nu = b->nu, H = nx / 2;
  if (nu != H) return false;
  const double dt = b->A[0 * nx + H], b1 = b->B[0], b2 = b->B[H * nu + 0];
  for (int r = 0; r < nx; ++r)
    for (int c = 0; c < nx; ++c) {
      double want = (r == c) ? 1.0 : 0.0;
      if (r < H && c == r + H) want = dt;
      if (b->A[r * nx + c] != want) return false;
    }
  for (int r = 0; r < nx; ++r)
    for (int c = 0; c < nu; ++c) {
      double want = 0.0;
      if (r < H && c == r) want = b1;
      if (r >= H && c == r - H) want = b2;
      if (b->B[r * nu + c] != want) return false;
    }
  return true;
}

static void free_all(tadmm_handle* h) {
  if (!h) return;
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->wexec) cudaGraphExecDestroy(h->wexec);
  void* gptrs[] = {h->gs_iter, h->gs_active, h->gs_need, h->gs_fail, h->gs_rb, h->gs_sb, h->gs_blk};
  for (void* p : gptrs)
    if (p) cudaFree(p);
  void* ptrs0[] = {h->goff, h->gmem, h->gorder};
  for (void* p : ptrs0)
    if (p) cudaFree(p);
  void* ptrs[] = {h->meta,   h->order, h->pairs, h->deg, h->adj_ptr, h->adj, h->pair_scen, h->agent_scen, h->model, h->Qd,     h->Rd,
                  h->Qfd,    h->x_init, h->x_ref, h->a,        h->w0,         h->theta, h->phi, h->sx, h->models, h->st_models, h->X, h->h,
                  h->U,      h->Us,    h->cache, h->Wm,        h->Cm,         h->status, h->iters, h->cur_lvl,
                  h->res,    h->eqp,   h->fact,  h->rho_out, h->rho_chg, h->queue,     h->st_model,   h->st_agent, h->st_a, h->st_w0,
                  h->ex_buf, h->flag,  h->red2, h->hprev, h->hmu, h->hdmu, h->st_costs, h->cost_flag, h->sqp_buf};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  void* bptrs[] = {h->bwd.act, h->bwd.cnt, h->bwd.amask, h->bwd.psi, h->bwd.kks, h->bwd.pos0, h->bwd.force,
                   h->bwd.Xp,  h->bwd.Up,  h->bwd.Wx,    h->bwd.Wu,  h->bwd.bstat, h->bwd.bs, h->bwd.S,
                   h->bwd.vec, h->bwd.gX,  h->bwd.gout,  h->bwd.xpol, h->bwd.piv, h->bwd.ndep, h->bwd.hmask,
                   h->bwd.Wb,  h->bwd.pchg, h->bwd.set_act, h->bwd.set_W};
  for (void* p : bptrs)
    if (p) cudaFree(p);
  if (h->pinned) cudaFreeHost(h->pinned);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
}

template <typename P>
static int dmalloc(P** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return set_error(TADMM_ENOMEM, std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes failed");
  }
  return TADMM_OK;
}

// Copies the caller's float64 arrays into staging and converts them to the
// internal layouts on `st`.
static int upload_inputs(tadmm_handle* h, const tadmm_batch* b, cudaStream_t st) {
  const int nx = h->nx, nu = h->nu, dp = h->dp;
  const int64_t na = h->tot_agents;
  for (int s = 0; s < h->n_scen; ++s) {
    h->meta_h[s].d = b->d_min[s];
    h->meta_h[s].rho = b->rho[s];
  }
  int rc;
  if ((rc = cuda_check(cudaMemcpyAsync(h->meta, h->meta_h.data(), sizeof(tadmm::ScenMeta) * h->n_scen,
                                       cudaMemcpyHostToDevice, st), "copy scenario table")))
    return rc;
  double* m = h->st_model;
  cudaMemcpyAsync(m, b->A, sizeof(double) * nx * nx, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(m + nx * nx, b->B, sizeof(double) * nx * nu, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(m + nx * nx + nx * nu, b->umin, sizeof(double) * nu, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(m + nx * nx + nx * nu + nu, b->umax, sizeof(double) * nu, cudaMemcpyHostToDevice, st);
  double* ag = h->st_agent;
  cudaMemcpyAsync(ag, b->Qd, sizeof(double) * na * nx, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(ag + na * nx, b->Rd, sizeof(double) * na * nu, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(ag + na * nx + na * nu, b->Qfd, sizeof(double) * na * nx, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(ag + 2 * na * nx + na * nu, b->x_init, sizeof(double) * na * nx, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(ag + 3 * na * nx + na * nu, b->x_ref, sizeof(double) * na * nx, cudaMemcpyHostToDevice, st);
  if (h->tot_ps > 0) cudaMemcpyAsync(h->st_a, b->a, sizeof(double) * h->tot_ps * dp, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(h->st_w0, b->w0, sizeof(double) * h->tot_as * dp, cudaMemcpyHostToDevice, st);
  if (h->hetero) {
    // per-agent models in the device layout [agent][A, B, umin, umax]
    const int nm = nx * nx + nx * nu + 2 * nu;
    cudaStreamSynchronize(st);  // the host packing may still feed an earlier copy
    h->models_h.resize((size_t)na * nm);
    for (int64_t i = 0; i < na; ++i) {
      double* d = h->models_h.data() + (size_t)i * nm;
      std::copy(b->A_agent + i * nx * nx, b->A_agent + (i + 1) * nx * nx, d);
      std::copy(b->B_agent + i * nx * nu, b->B_agent + (i + 1) * nx * nu, d + nx * nx);
      std::copy(b->umin, b->umin + nu, d + nx * nx + nx * nu);
      std::copy(b->umax, b->umax + nu, d + nx * nx + nx * nu + nu);
    }
    cudaMemcpyAsync(h->st_models, h->models_h.data(), sizeof(double) * na * nm, cudaMemcpyHostToDevice, st);
  }
  if ((rc = cuda_check(cudaGetLastError(), "input copies"))) return rc;
  TADMM_DISPATCH(h, import_inputs(h, st));
}

extern "C" int tadmm_create(const tadmm_batch* b, const tadmm_options* opt, tadmm_handle** out) {
  if (!out) return set_error(TADMM_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = validate(b, nullptr);
  if (rc) return rc;
  tadmm_options o{};
  o.precision = 64;
  o.start_mode = TADMM_START_TURBO;
  o.mode = TADMM_MODE_BATCHED;
  if (opt) o = *opt;
  if (o.precision != 64 && o.precision != 32) return set_error(TADMM_EINVAL, "precision must be 64 or 32");
  if (o.start_mode < 0 || o.start_mode > 3) return set_error(TADMM_EINVAL, "start_mode must be 0, 1, 2 or 3");
  if (o.start_mode == TADMM_START_HOMOTOPY && o.mode == TADMM_MODE_BATCHED)
    return set_error(TADMM_EINVAL, "the homotopy hot start runs in the plain and graph modes");
  if (o.start_mode == TADMM_START_HOMOTOPY && (o.flags & TADMM_FLAG_DOUBLE_FLOAT))
    return set_error(TADMM_EINVAL, "the homotopy hot start does not take TADMM_FLAG_DOUBLE_FLOAT");
  if (o.mode != TADMM_MODE_BATCHED && o.mode != TADMM_MODE_PLAIN && o.mode != TADMM_MODE_GRAPH)
    return set_error(TADMM_EINVAL, "bad mode");
  if (o.as_max < 0 || o.eps_rel < 0 || !std::isfinite(o.eps_rel)) return set_error(TADMM_EINVAL, "bad as_max / eps_rel");
  if (o.threads_per_cta != 0 && (o.threads_per_cta < 32 || o.threads_per_cta > 256 || o.threads_per_cta % 32))
    return set_error(TADMM_EINVAL, "threads_per_cta must be 0 or a multiple of 32 in [32, 256]");
  if (o.ctas_per_sm < 0) return set_error(TADMM_EINVAL, "ctas_per_sm must be >= 0");
  if (o.kernel_variant < 0 || o.kernel_variant > 2) return set_error(TADMM_EINVAL, "kernel_variant must be in 0..2");

  if (o.adapt_every < 0) return set_error(TADMM_EINVAL, "adapt_every must be >= 0");
  if (o.adapt_every > 0) {
    if (!(o.adapt_mu > 1.0) || !(o.adapt_tau > 1.0) || !std::isfinite(o.adapt_mu) || !std::isfinite(o.adapt_tau))
      return set_error(TADMM_EINVAL, "residual balancing needs finite adapt_mu > 1 and adapt_tau > 1");
    if (o.mode != TADMM_MODE_BATCHED)
      return set_error(TADMM_EINVAL, "residual balancing runs in the batched mode");
    if (o.flags & (TADMM_FLAG_NO_GROUPING | TADMM_FLAG_NO_FUSED_PAIR_GATHER))
      return set_error(TADMM_EINVAL, "residual balancing runs on the group path (no NO_GROUPING / NO_FUSED flags)");
    for (int s2 = 0; s2 < b->n_scen; ++s2)
      if (b->N[s2] > 32) return set_error(TADMM_EINVAL, "residual balancing supports scenarios of at most 32 agents");
  }
  if (o.relax_alpha == 0.0) o.relax_alpha = 1.0;
  if (!(o.relax_alpha > 0.0 && o.relax_alpha < 2.0))
    return set_error(TADMM_EINVAL, "relax_alpha must be 0 (off) or in (0, 2)");
  if (o.relax_alpha != 1.0) {
    if (o.mode != TADMM_MODE_BATCHED) return set_error(TADMM_EINVAL, "over-relaxation runs in the batched mode");
    if (o.flags & (TADMM_FLAG_NO_GROUPING | TADMM_FLAG_NO_FUSED_PAIR_GATHER))
      return set_error(TADMM_EINVAL, "over-relaxation runs on the group path (no NO_GROUPING / NO_FUSED flags)");
    for (int s2 = 0; s2 < b->n_scen; ++s2)
      if (b->N[s2] > 32) return set_error(TADMM_EINVAL, "over-relaxation supports scenarios of at most 32 agents");
  }
  if ((o.flags & TADMM_FLAG_DOUBLE_FLOAT) && b->A_agent)
    return set_error(TADMM_EINVAL, "TADMM_FLAG_DOUBLE_FLOAT does not take per-agent dynamics");
  if ((o.flags & TADMM_FLAG_DOUBLE_FLOAT) && (o.precision != 64 || b->nx != 4))
    return set_error(TADMM_EINVAL, "TADMM_FLAG_DOUBLE_FLOAT needs precision 64 and (nx, nu, dp) = (4, 2, 2)");
  tadmm_handle* h = new tadmm_handle();
  h->prec = (o.flags & TADMM_FLAG_DOUBLE_FLOAT) ? 128 : o.precision;
  h->nx = b->nx;
  h->nu = b->nu;
  h->dp = b->dp;
  h->n_scen = b->n_scen;
  h->opt = o;
  h->tpc = o.threads_per_cta;
  h->cps = o.ctas_per_sm;
  h->variant = o.kernel_variant;
  h->hetero = b->A_agent ? 1 : 0;
  h->di = (!(o.flags & TADMM_FLAG_NO_STRUCTURE) && !h->hetero && is_double_integrator(b)) ? 1 : 0;
  h->N.assign(b->N, b->N + b->n_scen);
  h->T.assign(b->T, b->T + b->n_scen);
  h->meta_h.resize(b->n_scen);
  std::vector<int32_t> pairs, pair_scen, agent_scen, deg, adj_ptr, adj;
  if (b->pair_count) {
    h->pair_count_h.assign(b->pair_count, b->pair_count + b->n_scen);
    int64_t tp = 0;
    for (int s = 0; s < b->n_scen; ++s) tp += b->pair_count[s];
    h->pair_ij_h.assign(b->pair_ij, b->pair_ij + 2 * tp);
  }
  adj_ptr.push_back(0);
  int64_t lpo = 0;  // offset of the scenario's listed pairs
  for (int s = 0; s < b->n_scen; ++s) {
    tadmm::ScenMeta& m = h->meta_h[s];
    m.N = h->N[s];
    m.T = h->T[s];
    m.P = b->pair_count ? b->pair_count[s] : m.N * (m.N - 1) / 2;
    m.sparse = b->pair_count ? 1 : 0;
    m.agent_off = h->tot_agents;
    m.as_off = h->tot_as;
    m.ps_off = h->tot_ps;
    m.xs_off = h->tot_xs;
    m.pair_off = h->tot_pairs;
    m.d = b->d_min[s];
    m.rho = b->rho[s];
    h->tot_agents += m.N;
    h->tot_as += (int64_t)m.N * m.T;
    h->tot_ps += (int64_t)m.P * m.T;
    h->tot_xs += (int64_t)m.N * (m.T + 1);
    h->tot_pairs += m.P;
    if (!m.sparse) {
      for (int i = 0; i < m.N; ++i) {
        agent_scen.push_back(s);
        deg.push_back(m.N - 1);
        adj_ptr.push_back((int32_t)adj.size());
        for (int j = i + 1; j < m.N; ++j) {
          pairs.push_back(i | (j << 16));
          pair_scen.push_back(s);
        }
      }
    } else {
      // listed pairs; per agent, its pairs by increasing partner (sign bit: the
      // agent is the second of the pair)
      std::vector<std::vector<std::pair<int, int32_t>>> inc(m.N);
      for (int k = 0; k < m.P; ++k) {
        const int i = b->pair_ij[2 * (lpo + k)], j = b->pair_ij[2 * (lpo + k) + 1];
        pairs.push_back(i | (j << 16));
        pair_scen.push_back(s);
        inc[i].push_back({j, (int32_t)k});
        inc[j].push_back({i, (int32_t)(k | 0x80000000u)});
      }
      for (int i = 0; i < m.N; ++i) {
        agent_scen.push_back(s);
        std::sort(inc[i].begin(), inc[i].end());
        deg.push_back((int32_t)inc[i].size());
        for (const auto& e : inc[i]) adj.push_back(e.second);
        adj_ptr.push_back((int32_t)adj.size());
      }
      lpo += m.P;
    }
  }
  // processing order of the persistent kernel: largest estimated work first
  std::vector<int32_t> order(b->n_scen);
  std::iota(order.begin(), order.end(), 0);
  std::vector<double> work(b->n_scen);
  for (int s = 0; s < b->n_scen; ++s)
    work[s] = double(h->meta_h[s].P) * h->meta_h[s].T * 30.0 + double(h->meta_h[s].N) * h->meta_h[s].T * 400.0;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });

  // Scenario groups for the persistent kernel: scenarios of equal horizon packed
  // first-fit-decreasing into groups of at most 32 agents (one lane per agent);
  // scenarios with more than 32 agents stay alone.  Groups run largest work first.
  std::vector<int32_t> goff, gmem;
  {
    const bool group = !(o.flags & (TADMM_FLAG_NO_GROUPING | TADMM_FLAG_NO_FUSED_PAIR_GATHER));
    std::vector<int32_t> idx(b->n_scen);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
      if (h->T[x] != h->T[y]) return h->T[x] > h->T[y];
      return h->N[x] > h->N[y];
    });
    std::vector<std::vector<int32_t>> groups;
    std::vector<int> load;
    size_t first_open = 0;
    int cur_T = -1;
    for (int sc : idx) {
      const int n = h->N[sc];
      if (h->T[sc] != cur_T) {
        cur_T = h->T[sc];
        first_open = groups.size();
      }
      int placed = -1;
      if (group && n <= 32)
        for (size_t g = first_open; g < groups.size(); ++g)
          if (load[g] + n <= 32 && load[g] > 0 && h->N[groups[g][0]] <= 32) { placed = (int)g; break; }
      if (placed < 0) {
        groups.push_back({});
        load.push_back(0);
        placed = (int)groups.size() - 1;
      }
      groups[placed].push_back(sc);
      load[placed] += n;
    }
    std::vector<double> gw(groups.size());
    for (size_t g = 0; g < groups.size(); ++g) {
      double pairs = 0;
      int gp = 0;
      for (int sc : groups[g]) {
        pairs += h->meta_h[sc].P;
        gp += h->meta_h[sc].P;
      }
      // groups that run the group path: several scenarios, or one of <= 32 agents
      if (groups[g].size() > 1 || h->N[groups[g][0]] <= 32) h->max_group_pairs = std::max(h->max_group_pairs, gp);
      gw[g] = double(h->T[groups[g][0]]) * (600.0 + 30.0 * pairs / 32.0);
    }
    std::vector<int32_t> gord(groups.size());
    std::iota(gord.begin(), gord.end(), 0);
    std::stable_sort(gord.begin(), gord.end(), [&](int x, int y) { return gw[x] > gw[y]; });
    goff.push_back(0);
    for (size_t g = 0; g < groups.size(); ++g) {
      for (int sc : groups[g]) gmem.push_back(sc);
      goff.push_back((int32_t)gmem.size());
    }
    h->n_groups = (int)groups.size();
    order = gord;
  }

  cudaGetDevice(&h->device);
  cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
  const size_t fs = h->prec == 32 ? 4 : 8;
  const int nx = h->nx, nu = h->nu, dp = h->dp;
  const int64_t na = h->tot_agents;
  const size_t ex_doubles = (size_t)std::max<int64_t>({h->tot_xs * nx, h->tot_as * nu, h->tot_ps, 1});
  h->ex_bytes = ex_doubles * sizeof(double);
  if ((rc = dmalloc(&h->goff, 4 * goff.size())) || (rc = dmalloc(&h->gmem, 4 * gmem.size())) ||
      (rc = dmalloc(&h->gorder, 4 * order.size())) ||
      (rc = dmalloc(&h->meta, sizeof(tadmm::ScenMeta) * h->n_scen)) || (rc = dmalloc(&h->order, 4 * order.size())) ||
      (rc = dmalloc(&h->pairs, 4 * pairs.size())) || (rc = dmalloc(&h->deg, 4 * deg.size())) ||
      (rc = dmalloc(&h->adj_ptr, 4 * adj_ptr.size())) || (rc = dmalloc(&h->adj, 4 * std::max<size_t>(adj.size(), 1))) || (rc = dmalloc(&h->pair_scen, 4 * pair_scen.size())) ||
      (rc = dmalloc(&h->agent_scen, 4 * agent_scen.size())) ||
      (rc = dmalloc(&h->model, fs * (nx * nx + nx * nu + 2 * nu))) || (rc = dmalloc(&h->Qd, fs * na * nx)) ||
      (rc = dmalloc(&h->Rd, fs * na * nu)) || (rc = dmalloc(&h->Qfd, fs * na * nx)) ||
      (rc = dmalloc(&h->x_init, fs * na * nx)) || (rc = dmalloc(&h->x_ref, fs * na * nx)) ||
      (rc = dmalloc(&h->a, fs * h->tot_ps * dp)) || (rc = dmalloc(&h->w0, fs * h->tot_as * dp)) ||
      (rc = dmalloc(&h->theta, fs * 3 * h->tot_ps)) || (rc = dmalloc(&h->X, fs * 2 * h->tot_xs * nx)) ||
      (rc = dmalloc(&h->h, fs * h->tot_as * dp)) || (rc = dmalloc(&h->U, fs * h->tot_as * nu)) ||
      (rc = dmalloc(&h->Us, fs * h->tot_as * nu)) ||
      (rc = dmalloc(&h->cache, fs * h->tot_xs * cache_words(nx, nu))) ||
      (rc = dmalloc(&h->Wm, 2 * h->tot_as)) || (rc = dmalloc(&h->Cm, 2 * h->tot_as)) ||
      (rc = dmalloc(&h->status, 4 * h->n_scen)) || (rc = dmalloc(&h->iters, 4 * h->n_scen)) ||
      (rc = dmalloc(&h->cur_lvl, 4 * h->n_scen)) || (rc = dmalloc(&h->res, 16 * h->n_scen)) ||
      (rc = dmalloc(&h->eqp, 8 * h->n_scen)) || (rc = dmalloc(&h->fact, 8 * h->n_scen)) ||
      (rc = dmalloc(&h->rho_out, 8 * h->n_scen)) || (rc = dmalloc(&h->rho_chg, 4 * h->n_scen)) ||
      (rc = dmalloc(&h->queue, 16)) ||
      (rc = dmalloc(&h->st_model, 8 * (nx * nx + nx * nu + 2 * nu))) ||
      (rc = dmalloc(&h->st_agent, 8 * na * (4 * nx + nu))) || (rc = dmalloc(&h->st_a, 8 * h->tot_ps * dp)) ||
      (rc = dmalloc(&h->st_w0, 8 * h->tot_as * dp)) || (rc = dmalloc(&h->ex_buf, h->ex_bytes + h->tot_as * nu + 16)) ||
      (rc = dmalloc(&h->flag, 16)) || (rc = dmalloc(&h->red2, 16)) ||
      (o.relax_alpha != 1.0 && ((rc = dmalloc(&h->phi, fs * h->tot_ps)) || (rc = dmalloc(&h->sx, fs * h->tot_as * dp)))) ||
      (o.start_mode == TADMM_START_HOMOTOPY &&
       ((rc = dmalloc(&h->hprev, fs * h->tot_as * dp)) || (rc = dmalloc(&h->hmu, fs * h->tot_as * nu)) ||
        (rc = dmalloc(&h->hdmu, fs * h->tot_as * nu)))) ||
      (h->hetero && ((rc = dmalloc(&h->models, fs * na * (nx * nx + nx * nu + 2 * nu))) ||
                     (rc = dmalloc(&h->st_models, 8 * na * (nx * nx + nx * nu + 2 * nu)))))) {
    free_all(h);
    return rc;
  }
  if (cudaMallocHost(&h->pinned, 64) != cudaSuccess) {
    free_all(h);
    return set_error(TADMM_ENOMEM, "cudaMallocHost failed");
  }
  if ((rc = cuda_check(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking), "stream create"))) {
    free_all(h);
    return rc;
  }
  cudaStream_t st = h->cap_stream;
  cudaMemcpyAsync(h->order, order.data(), 4 * order.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(h->gorder, order.data(), 4 * order.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(h->goff, goff.data(), 4 * goff.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(h->gmem, gmem.data(), 4 * gmem.size(), cudaMemcpyHostToDevice, st);
  if (!pairs.empty()) {
    cudaMemcpyAsync(h->pairs, pairs.data(), 4 * pairs.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(h->deg, deg.data(), 4 * deg.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(h->adj_ptr, adj_ptr.data(), 4 * adj_ptr.size(), cudaMemcpyHostToDevice, st);
    if (!adj.empty()) cudaMemcpyAsync(h->adj, adj.data(), 4 * adj.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(h->pair_scen, pair_scen.data(), 4 * pair_scen.size(), cudaMemcpyHostToDevice, st);
  }
  cudaMemcpyAsync(h->agent_scen, agent_scen.data(), 4 * agent_scen.size(), cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(h->status, 0xFF, 4 * h->n_scen, st);
  cudaMemsetAsync(h->iters, 0, 4 * h->n_scen, st);
  cudaMemsetAsync(h->cur_lvl, 0, 4 * h->n_scen, st);
  cudaMemsetAsync(h->res, 0, 16 * h->n_scen, st);
  cudaMemsetAsync(h->eqp, 0, 8 * h->n_scen, st);
  cudaMemsetAsync(h->fact, 0, 8 * h->n_scen, st);
  if ((rc = upload_inputs(h, b, st)) || (rc = cuda_check(cudaStreamSynchronize(st), "create: upload"))) {
    free_all(h);
    return rc;
  }
  *out = h;
  return TADMM_OK;
}

extern "C" int tadmm_update(tadmm_handle* h, const tadmm_batch* b, void* stream) {
  if (!h) return set_error(TADMM_EINVAL, "handle is NULL");
  if (!b || b->n_scen != h->n_scen || b->nx != h->nx || b->nu != h->nu || b->dp != h->dp)
    return set_error(TADMM_EINVAL, "update: batch shape differs from the handle");
  int rc = validate(b, h);
  if (rc) return rc;
  return upload_inputs(h, b, (cudaStream_t)stream);
}

// Device-side checks of new cost values (float64): finite Q, Qf >= 0, finite
// x_ref, finite R > 0.  Any violation sets *bad.
__global__ void k_check_costs(const double* Qd, const double* Rd, const double* Qfd, const double* xr, int64_t nq,
                              int64_t nr, int32_t* bad) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
  bool ok = true;
  for (int64_t k = tid; k < nq; k += nt) {
    if (Qd) ok = ok && isfinite(Qd[k]) && Qd[k] >= 0.0;
    if (Qfd) ok = ok && isfinite(Qfd[k]) && Qfd[k] >= 0.0;
    if (xr) ok = ok && isfinite(xr[k]);
  }
  if (Rd)
    for (int64_t k = tid; k < nr; k += nt) ok = ok && isfinite(Rd[k]) && Rd[k] > 0.0;
  if (!ok) atomicOr(bad, 1);
}

extern "C" int tadmm_update_costs(tadmm_handle* h, const double* Qd, const double* Rd, const double* Qfd,
                                  const double* x_ref, void* stream) {
  if (!h) return set_error(TADMM_EINVAL, "handle is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t na = h->tot_agents, nq = na * h->nx, nr = na * h->nu;
  int rc;
  if (!h->st_costs) {
    if ((rc = dmalloc(&h->st_costs, sizeof(double) * (size_t)(3 * nq + nr))) || (rc = dmalloc(&h->cost_flag, 16)))
      return rc;
  }
  // scratch blocks Qd | Rd | Qfd | x_ref, then the staging blocks of the same arrays
  double* sc[4] = {h->st_costs, h->st_costs + nq, h->st_costs + nq + nr, h->st_costs + 2 * nq + nr};
  double* sg[4] = {h->st_agent, h->st_agent + nq, h->st_agent + nq + nr, h->st_agent + 3 * nq + nr};
  const double* src[4] = {Qd, Rd, Qfd, x_ref};
  const int64_t n[4] = {nq, nr, nq, nq};
  int which = 0;
  for (int k = 0; k < 4; ++k) {
    if (!src[k]) continue;
    which |= 1 << k;
    if ((rc = cuda_check(cudaMemcpyAsync(sc[k], src[k], sizeof(double) * n[k], cudaMemcpyDefault, st), "cost copy")))
      return rc;
  }
  if (!which) return TADMM_OK;
  if ((rc = cuda_check(cudaMemsetAsync(h->cost_flag, 0, sizeof(int32_t), st), "cost flag")))
    return rc;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(1024, (std::max(nq, nr) + 255) / 256));
  k_check_costs<<<grid, 256, 0, st>>>(
      Qd ? sc[0] : nullptr, Rd ? sc[1] : nullptr, Qfd ? sc[2] : nullptr, x_ref ? sc[3] : nullptr, nq, nr, h->cost_flag);
  int32_t* flag_h = (int32_t*)h->pinned;
  if ((rc = cuda_check(cudaGetLastError(), "cost check")) ||
      (rc = cuda_check(cudaMemcpyAsync(flag_h, h->cost_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, st), "cost flag")) ||
      (rc = cuda_check(cudaStreamSynchronize(st), "cost check sync")))
    return rc;
  if (*flag_h) return set_error(TADMM_EINVAL, "update_costs: Q and Qf diagonals must be finite and >= 0, R finite and > 0, x_ref finite");
  for (int k = 0; k < 4; ++k)
    if ((which >> k) & 1 &&
        (rc = cuda_check(cudaMemcpyAsync(sg[k], sc[k], sizeof(double) * n[k], cudaMemcpyDeviceToDevice, st), "cost stage")))
      return rc;
  TADMM_DISPATCH(h, import_costs(h, which, st));
}

extern "C" int tadmm_solve(tadmm_handle* h, double tol, int32_t max_iter, void* stream) {
  if (!h) return set_error(TADMM_EINVAL, "handle is NULL");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return set_error(TADMM_EINVAL, "tol must be finite and >= 0");
  if (max_iter < 1) return set_error(TADMM_EINVAL, "max_iter must be >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  int rc;
  if (h->opt.mode == TADMM_MODE_PLAIN) {
    auto run = [&]() -> int { TADMM_DISPATCH(h, solve_plain(h, tol, max_iter, st)); };
    rc = run();
  } else if (h->opt.mode == TADMM_MODE_GRAPH) {
    auto run = [&]() -> int { TADMM_DISPATCH(h, solve_graph(h, tol, max_iter, st)); };
    rc = run();
  } else {
    auto run = [&]() -> int { TADMM_DISPATCH(h, solve_batched(h, tol, max_iter, st)); };
    rc = run();
  }
  if (rc == TADMM_OK) h->solved = 1;
  h->bwd_polished = 0;
  return rc;
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

extern "C" int tadmm_get_solution(tadmm_handle* h, double* X, double* U, double* theta, int8_t* W, int32_t* status,
                                  int32_t* iters, double* res, void* stream) {
  if (!h) return set_error(TADMM_EINVAL, "handle is NULL");
  if (!h->solved) return set_error(TADMM_ESTATE, "get_solution before solve");
  cudaStream_t st = (cudaStream_t)stream;
  const int nx = h->nx, nu = h->nu;
  auto export_one = [&](double* Xd, double* Ud, double* Td, int8_t* Wd) -> int {
    TADMM_DISPATCH(h, export_solution(h, Xd, Ud, Td, Wd, st));
  };
  int rc;
  double* ex = h->ex_buf;
  int8_t* exw = (int8_t*)((char*)h->ex_buf + h->ex_bytes);
  struct Item { void* dst; size_t bytes; int kind; };
  const Item items[4] = {{X, sizeof(double) * h->tot_xs * nx, 0},
                         {U, sizeof(double) * h->tot_as * nu, 1},
                         {theta, sizeof(double) * h->tot_ps, 2},
                         {W, (size_t)h->tot_as * nu, 3}};
  for (const Item& it : items) {
    if (!it.dst || it.bytes == 0) continue;
    const bool dev = is_device_ptr(it.dst);
    void* tgt = dev ? it.dst : (it.kind == 3 ? (void*)exw : (void*)ex);
    rc = export_one(it.kind == 0 ? (double*)tgt : nullptr, it.kind == 1 ? (double*)tgt : nullptr,
                    it.kind == 2 ? (double*)tgt : nullptr, it.kind == 3 ? (int8_t*)tgt : nullptr);
    if (rc) return rc;
    if (!dev && (rc = cuda_check(cudaMemcpyAsync(it.dst, tgt, it.bytes, cudaMemcpyDefault, st), "copy result")))
      return rc;
  }
  if (status && (rc = cuda_check(cudaMemcpyAsync(status, h->status, 4 * h->n_scen, cudaMemcpyDefault, st), "status")))
    return rc;
  if (iters && (rc = cuda_check(cudaMemcpyAsync(iters, h->iters, 4 * h->n_scen, cudaMemcpyDefault, st), "iters")))
    return rc;
  if (res && (rc = cuda_check(cudaMemcpyAsync(res, h->res, 16 * h->n_scen, cudaMemcpyDefault, st), "res")))
    return rc;
  return cuda_check(cudaStreamSynchronize(st), "get_solution sync");
}

extern "C" int tadmm_get_counters(tadmm_handle* h, int64_t* eqp, int64_t* fact, int64_t* pairsteps) {
  if (!h) return set_error(TADMM_EINVAL, "handle is NULL");
  if (!h->solved) return set_error(TADMM_ESTATE, "get_counters before solve");
  int rc;
  if ((rc = cuda_check(cudaDeviceSynchronize(), "counters sync"))) return rc;
  if (eqp && (rc = cuda_check(cudaMemcpy(eqp, h->eqp, 8 * h->n_scen, cudaMemcpyDeviceToHost), "eqp"))) return rc;
  if (fact && (rc = cuda_check(cudaMemcpy(fact, h->fact, 8 * h->n_scen, cudaMemcpyDeviceToHost), "fact"))) return rc;
  if (pairsteps) {
    std::vector<int32_t> it(h->n_scen);
    if ((rc = cuda_check(cudaMemcpy(it.data(), h->iters, 4 * h->n_scen, cudaMemcpyDeviceToHost), "iters"))) return rc;
    for (int s = 0; s < h->n_scen; ++s) pairsteps[s] = (int64_t)it[s] * h->meta_h[s].P * h->meta_h[s].T;
  }
  return TADMM_OK;
}

extern "C" int tadmm_relinearize(tadmm_handle* h, void* stream) {
  if (!h) return set_error(TADMM_EINVAL, "handle is NULL");
  if (!h->solved) return set_error(TADMM_ESTATE, "relinearize before solve");
  cudaStream_t st = (cudaStream_t)stream;
  TADMM_DISPATCH(h, relinearize(h, nullptr, st));
}

extern "C" int tadmm_sqp(tadmm_handle* h, double tol, int32_t max_iter, int32_t max_outer, double obj_rtol,
                         double dist_tol, int32_t* outer, int32_t* sqp_status, double* objective, double* min_dist,
                         void* stream) {
  if (!h) return set_error(TADMM_EINVAL, "handle is NULL");
  if (max_outer < 1) return set_error(TADMM_EINVAL, "max_outer must be >= 1");
  if (!(obj_rtol >= 0.0) || !std::isfinite(obj_rtol)) return set_error(TADMM_EINVAL, "obj_rtol must be finite and >= 0");
  if (std::isnan(dist_tol) || std::isinf(dist_tol)) return set_error(TADMM_EINVAL, "dist_tol must be finite");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return set_error(TADMM_EINVAL, "tol must be finite and >= 0");
  if (max_iter < 1) return set_error(TADMM_EINVAL, "max_iter must be >= 1");
  if (dist_tol < 0.0) dist_tol = 2.0 * std::sqrt((double)h->dp) * tol;
  cudaStream_t st = (cudaStream_t)stream;
  const int n = h->n_scen;
  int rc;
  if (!h->sqp_buf && (rc = dmalloc(&h->sqp_buf, sizeof(double) * 2 * n + n + 16))) return rc;
  double* J_dev = h->sqp_buf;
  double* D_dev = h->sqp_buf + n;
  uint8_t* keep_dev = (uint8_t*)(h->sqp_buf + 2 * n);
  std::vector<double> J(n), D(n), Jp(n, 0.0), Jout(n, 0.0), Dout(n, 0.0);
  std::vector<int32_t> stat(n), steps(n, 0);
  std::vector<uint8_t> done(n, 0);
  int n_done = 0;
  for (int m = 1; m <= max_outer; ++m) {
    if ((rc = tadmm_solve(h, tol, max_iter, stream))) return rc;
    auto measure = [&]() -> int { TADMM_DISPATCH(h, sqp_measure(h, J_dev, D_dev, st)); };
    if ((rc = measure()) ||
        (rc = cuda_check(cudaMemcpyAsync(J.data(), J_dev, sizeof(double) * n, cudaMemcpyDeviceToHost, st), "objective")) ||
        (rc = cuda_check(cudaMemcpyAsync(D.data(), D_dev, sizeof(double) * n, cudaMemcpyDeviceToHost, st), "distance")) ||
        (rc = cuda_check(cudaMemcpyAsync(stat.data(), h->status, 4 * n, cudaMemcpyDeviceToHost, st), "status")) ||
        (rc = cuda_check(cudaStreamSynchronize(st), "sqp sync")))
      return rc;
    for (int s = 0; s < n; ++s) {
      if (done[s]) continue;
      steps[s] = m;
      Jout[s] = J[s];
      Dout[s] = D[s];
      if (stat[s] == TADMM_CONVERGED && m >= 2 && std::fabs(J[s] - Jp[s]) <= obj_rtol * std::fabs(Jp[s]) &&
          D[s] >= h->meta_h[s].d - dist_tol) {
        done[s] = 1;
        ++n_done;
      }
      Jp[s] = J[s];
    }
    if (n_done == n || m == max_outer) break;
    // Scenarios that met the rule keep their linearization (their re-solve in
    // the next step reproduces their solution bit for bit); the others are
    // re-linearized at their solution.
    auto relin = [&]() -> int { TADMM_DISPATCH(h, relinearize(h, keep_dev, st)); };
    if ((rc = cuda_check(cudaMemcpyAsync(keep_dev, done.data(), n, cudaMemcpyHostToDevice, st), "sqp mask")) ||
        (rc = relin()) || (rc = cuda_check(cudaStreamSynchronize(st), "sqp mask sync")))
      return rc;
  }
  for (int s = 0; s < n; ++s) {
    if (outer) outer[s] = steps[s];
    if (sqp_status) sqp_status[s] = done[s] ? TADMM_CONVERGED : TADMM_NOT_CONVERGED;
    if (objective) objective[s] = Jout[s];
    if (min_dist) min_dist[s] = Dout[s];
  }
  return TADMM_OK;
}

extern "C" int tadmm_get_penalty(tadmm_handle* h, double* rho_final, int32_t* rho_changes) {
  if (!h) return set_error(TADMM_EINVAL, "handle is NULL");
  if (!h->solved) return set_error(TADMM_ESTATE, "get_penalty before solve");
  int rc;
  if ((rc = cuda_check(cudaDeviceSynchronize(), "penalty sync"))) return rc;
  if (h->opt.mode == TADMM_MODE_BATCHED) {
    if (rho_final && (rc = cuda_check(cudaMemcpy(rho_final, h->rho_out, 8 * h->n_scen, cudaMemcpyDeviceToHost), "rho")))
      return rc;
    if (rho_changes &&
        (rc = cuda_check(cudaMemcpy(rho_changes, h->rho_chg, 4 * h->n_scen, cudaMemcpyDeviceToHost), "rho changes")))
      return rc;
  } else {
    for (int s = 0; s < h->n_scen; ++s) {
      if (rho_final) rho_final[s] = h->meta_h[s].rho;
      if (rho_changes) rho_changes[s] = 0;
    }
  }
  return TADMM_OK;
}

extern "C" int tadmm_autotune(tadmm_handle* h, int32_t probe_iter, void* stream, int32_t* threads_out,
                              int32_t* ctas_out, int32_t* variant_out) {
  if (!h) return set_error(TADMM_EINVAL, "handle is NULL");
  if (probe_iter < 1) return set_error(TADMM_EINVAL, "probe_iter must be >= 1");
  if (h->opt.mode != TADMM_MODE_BATCHED) return set_error(TADMM_EINVAL, "autotune applies to the batched mode");
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int keep_t = h->tpc, keep_c = h->cps, keep_v = h->variant;
  struct Shape { int v, tpc, cps; float ms; };
  // device time of the last of `reps` solves of `iters` iterations (tol 0) in shape sh
  auto time_shape = [&](const Shape& sh, int iters, int reps, float& ms) -> int {
    h->variant = sh.v;
    h->tpc = sh.tpc;
    h->cps = sh.cps;
    int rc = TADMM_OK;
    for (int rep = 0; rep < reps && rc == TADMM_OK; ++rep) {
      cudaEventRecord(e0, st);
      rc = tadmm_solve(h, 0.0, iters, stream);
      cudaEventRecord(e1, st);
      if (rc == TADMM_OK) rc = cuda_check(cudaEventSynchronize(e1), "autotune sync");
      if (rc == TADMM_OK) cudaEventElapsedTime(&ms, e0, e1);
    }
    return rc;
  };
  struct Cand { int v, tpc; };
  const Cand cands[] = {{0, 32}, {0, 64}, {0, 128}, {1, 32}, {2, 64}};
  std::vector<Shape> probed;
  int rc = TADMM_OK;
  // stage 1: every candidate shape over probe_iter iterations
  for (const Cand& cd : cands) {
    const int tpc = cd.tpc;
    auto occ = [&]() -> int { TADMM_DISPATCH(h, max_ctas_per_sm(tpc, cd.v, h)); };
    const int maxc = occ();
    if (maxc < 1) continue;
    std::vector<int> cps_list = {maxc};
    if (maxc >= 4) cps_list.push_back(maxc / 2);
    for (int cps : cps_list) {
      Shape sh{cd.v, tpc, cps, 0.0f};
      if ((rc = time_shape(sh, probe_iter, 2, sh.ms))) break;
      probed.push_back(sh);
    }
    if (rc) break;
  }
  // stage 2: the three fastest again over 4 x probe_iter iterations, since the
  // ranking of close shapes can change once the active-set transient of the
  // first iterations has passed
  Shape best{0, 128, 0, 1e30f};
  if (rc == TADMM_OK && !probed.empty()) {
    std::stable_sort(probed.begin(), probed.end(), [](const Shape& a, const Shape& b) { return a.ms < b.ms; });
    best = probed[0];
    const size_t nfin = std::min<size_t>(3, probed.size());
    if (nfin > 1) {
      best.ms = 1e30f;
      for (size_t k = 0; k < nfin && rc == TADMM_OK; ++k) {
        Shape sh = probed[k];
        if ((rc = time_shape(sh, probe_iter > (1 << 28) ? probe_iter : 4 * probe_iter, 1, sh.ms))) break;
        if (sh.ms < best.ms) best = sh;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc || probed.empty()) {
    h->tpc = keep_t;
    h->cps = keep_c;
    h->variant = keep_v;
    return rc ? rc : set_error(TADMM_EINVAL, "no launch shape fits this batch");
  }
  h->tpc = best.tpc;
  h->cps = best.cps;
  h->variant = best.v;
  if (threads_out) *threads_out = best.tpc;
  if (ctas_out) *ctas_out = best.cps;
  if (variant_out) *variant_out = best.v;
  return TADMM_OK;
}

extern "C" int tadmm_backward(tadmm_handle* h, const double* grad_X, double theta_eps, double* gQ, double* gQf,
                              double* gR, double* gGoal, double* X_polished, int32_t* status, int32_t* n_dependent,
                              void* stream) {
  if (!h) return set_error(TADMM_EINVAL, "handle is NULL");
  if (!h->solved) return set_error(TADMM_ESTATE, "backward before solve");
  if (!(theta_eps >= 0.0) || !std::isfinite(theta_eps)) return set_error(TADMM_EINVAL, "theta_eps must be >= 0");
  for (const auto& m : h->meta_h)
    if (m.T > 64) return set_error(TADMM_EINVAL, "backward supports horizons T <= 64");
  cudaStream_t st = (cudaStream_t)stream;
  const int nx = h->nx, nu = h->nu;
  const int64_t na = h->tot_agents;
  auto grow = [&](void** p, size_t& cap, size_t bytes) -> int {
    if (bytes <= cap && *p) return TADMM_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    cap = 0;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return set_error(TADMM_ENOMEM, "backward staging allocation failed");
    }
    cap = bytes;
    return TADMM_OK;
  };
  int rc;
  const size_t gx_bytes = sizeof(double) * h->tot_xs * nx;
  const size_t gout_n = (size_t)na * (3 * nx + nu);
  if ((rc = grow(&h->bwd.gX, h->bwd.gX_cap, gx_bytes)) ||
      (rc = grow(&h->bwd.gout, h->bwd.gout_cap, sizeof(double) * gout_n)) ||
      (rc = grow(&h->bwd.xpol, h->bwd.xpol_cap, gx_bytes)))
    return rc;
  if (grad_X && (rc = cuda_check(cudaMemcpyAsync(h->bwd.gX, grad_X, gx_bytes, cudaMemcpyDefault, st), "grad_X copy")))
    return rc;
  double* gout = (double*)h->bwd.gout;
  auto run = [&]() -> int {
    TADMM_DISPATCH(h, backward(h, grad_X ? (const double*)h->bwd.gX : nullptr, theta_eps, gout,
                               X_polished ? (double*)h->bwd.xpol : nullptr, st));
  };
  if ((rc = run())) return rc;
  struct Out { void* dst; size_t off, n; };
  const Out outs[4] = {{gQ, 0, (size_t)na * nx}, {gQf, (size_t)na * nx, (size_t)na * nx},
                       {gR, 2 * (size_t)na * nx, (size_t)na * nu}, {gGoal, 2 * (size_t)na * nx + na * nu, (size_t)na * nx}};
  for (const Out& o : outs)
    if (grad_X && o.dst && (rc = cuda_check(cudaMemcpyAsync(o.dst, gout + o.off, sizeof(double) * o.n, cudaMemcpyDefault, st),
                                  "gradient copy")))
      return rc;
  if (X_polished && (rc = cuda_check(cudaMemcpyAsync(X_polished, h->bwd.xpol, gx_bytes, cudaMemcpyDefault, st),
                                     "polished X copy")))
    return rc;
  if (status && (rc = cuda_check(cudaMemcpyAsync(status, h->bwd.bstat, 4 * h->n_scen, cudaMemcpyDefault, st),
                                 "backward status copy")))
    return rc;
  if (n_dependent && (rc = cuda_check(cudaMemcpyAsync(n_dependent, h->bwd.ndep, 4 * h->n_scen, cudaMemcpyDefault, st),
                                      "backward rank copy")))
    return rc;
  return cuda_check(cudaStreamSynchronize(st), "backward sync");
}

extern "C" int tadmm_polish(tadmm_handle* h, double theta_eps, int32_t max_rounds, double kkt_tol, uint8_t* act,
                            int8_t* W, int32_t* status, int32_t* rounds, void* stream) {
  if (!h) return set_error(TADMM_EINVAL, "handle is NULL");
  if (!h->solved) return set_error(TADMM_ESTATE, "polish before solve");
  if (!(theta_eps >= 0.0) || !std::isfinite(theta_eps)) return set_error(TADMM_EINVAL, "theta_eps must be >= 0");
  if (max_rounds < 1) return set_error(TADMM_EINVAL, "max_rounds must be >= 1");
  if (!(kkt_tol >= 0.0) || !std::isfinite(kkt_tol)) return set_error(TADMM_EINVAL, "kkt_tol must be >= 0");
  if (kkt_tol == 0.0) kkt_tol = h->prec == 32 ? 1e-5 : 1e-9;
  for (const auto& m : h->meta_h)
    if (m.T > 64) return set_error(TADMM_EINVAL, "polish supports horizons T <= 64");
  cudaStream_t st = (cudaStream_t)stream;
  auto grow = [&](void** p, size_t& cap, size_t bytes) -> int {
    if (bytes <= cap && *p) return TADMM_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    cap = 0;
    if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
      cudaGetLastError();
      return set_error(TADMM_ENOMEM, "polish staging allocation failed");
    }
    cap = bytes;
    return TADMM_OK;
  };
  int rc;
  const size_t act_bytes = (size_t)std::max<int64_t>(h->tot_ps, 1), w_bytes = (size_t)h->tot_as * h->nu;
  if ((act && (rc = grow(&h->bwd.set_act, h->bwd.set_act_cap, act_bytes))) ||
      (W && (rc = grow(&h->bwd.set_W, h->bwd.set_W_cap, w_bytes))))
    return rc;
  uint8_t* act_dev = act ? (uint8_t*)h->bwd.set_act : nullptr;
  int8_t* W_dev = W ? (int8_t*)h->bwd.set_W : nullptr;
  std::vector<int32_t> stat(h->n_scen);
  int32_t nr = 0;
  auto run = [&]() -> int {
    TADMM_DISPATCH(h, polish(h, theta_eps, max_rounds, kkt_tol, act_dev, W_dev, stat.data(), &nr, st));
  };
  if ((rc = run())) return rc;
  if (act && h->tot_ps > 0 &&
      (rc = cuda_check(cudaMemcpyAsync(act, act_dev, (size_t)h->tot_ps, cudaMemcpyDefault, st), "active set copy")))
    return rc;
  if (W && (rc = cuda_check(cudaMemcpyAsync(W, W_dev, w_bytes, cudaMemcpyDefault, st), "working set copy")))
    return rc;
  if ((rc = cuda_check(cudaStreamSynchronize(st), "polish sync"))) return rc;
  if (status) std::memcpy(status, stat.data(), 4 * h->n_scen);
  if (rounds) *rounds = nr;
  return TADMM_OK;
}

extern "C" void tadmm_destroy(tadmm_handle* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  free_all(h);
}

extern "C" const char* tadmm_last_error(void) { return tadmm::g_err.c_str(); }

extern "C" const char* tadmm_version(void) { return "tadmm 0.1 (sm_103a)"; }
