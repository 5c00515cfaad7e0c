// tadmm_solve_noalloc: one scenario solved without any device allocation.
//
// Some callers cannot call cudaMalloc once they are running: a real-time
// control loop that is only allowed to allocate during start-up (an allocation
// costs unpredictable time and may synchronize the whole device), or a host
// program whose device memory is owned by an outside allocator that forbids
// raw allocations.  This entry point serves them: inputs and outputs are device
// buffers the caller already owns, and all working memory of the solver lives
// in one fixed-size array in device global memory that the library reserves
// when it is loaded (TADMM_NOALLOC_SCRATCH_BYTES on every GPU that loads it,
// held until the process exits).
//
// The array is shared by every call: each call re-initializes all the state it
// reads, and two calls whose work overlaps on the GPU (different streams, or
// different host threads, on the same device) race on it and corrupt each
// other.  Callers must serialize them.
//
// Input values are checked on the device (the caller's arrays are device
// memory) by the rules tadmm_create applies on the host; a scenario that
// breaks one is reported through status TADMM_INVALID_INPUT and not solved.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "tadmm_kernels.cuh"

namespace tadmm {

static __device__ __align__(256) unsigned char g_noalloc_scratch[TADMM_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The name of the
// array is only a host-side stand-in, so the address is looked up with that
// device current: on every call made outside stream capture (which also picks
// up a new address after a device reset), and from the last lookup during a
// capture.  With lazy module loading the first call on a device also loads the
// library's module there (an allocation by the driver), so it belongs to the
// caller's start-up, before any capture.
int scratch_address(void** out, cudaStream_t st) {
  int dev = 0;
  int rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (rc) return rc;
  if (dev < 0 || dev >= kMaxDevices) return set_error(TADMM_EINVAL, "device ordinal out of range");
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if ((rc = cuda_check(cudaStreamIsCapturing(st, &cap), "cudaStreamIsCapturing"))) return rc;
  std::lock_guard<std::mutex> lk(g_mu);
  if (cap == cudaStreamCaptureStatusNone || !g_scratch_addr[dev]) {
    void* p = nullptr;
    rc = cuda_check(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(scratch)");
    if (rc) return rc;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return TADMM_OK;
}

struct Carve {
  char* base;
  size_t off = 0;
  template <typename P>
  P* take(size_t bytes) {
    off = (off + 255) & ~size_t(255);
    P* p = base ? (P*)(base + off) : nullptr;
    off += bytes ? bytes : 16;
    return p;
  }
};

}  // namespace

// Scenario table, processing order, pair table, zeroed bookkeeping.
__global__ void k_noalloc_setup(ScenMeta* meta, int32_t* order, int32_t* pairs, int32_t* pair_scen,
                                int32_t* agent_scen, int32_t* queue, int N, int T, double d, double rho) {
  const int P = N * (N - 1) / 2;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  if (tid == 0) {
    ScenMeta m;
    m.N = N; m.T = T; m.P = P; m.sparse = 0;
    m.agent_off = 0; m.as_off = 0; m.ps_off = 0; m.xs_off = 0; m.pair_off = 0;
    m.d = d; m.rho = rho;
    *meta = m;
    order[0] = 0;
    *queue = 0;
  }
  for (int i = tid; i < N; i += nt) {
    agent_scen[i] = 0;
    const int base = i * N - (i * (i + 1)) / 2;
    for (int j = i + 1; j < N; ++j) {
      pairs[base + (j - i - 1)] = i | (j << 16);
      pair_scen[base + (j - i - 1)] = 0;
    }
  }
}

// Input values by the rules of tadmm_create (host checks there, device checks
// here, since the inputs are device memory): finite A, B, x_init, x_ref, w0,
// a; finite umin <= umax; finite Q, Qf >= 0; finite R > 0.  Any violation
// marks the scenario TADMM_INVALID_INPUT (bad = 1), which the solve skips.
template <int NX, int NU, int DP>
__global__ void k_noalloc_validate(const double* model, const double* Qd, const double* Rd, const double* Qfd,
                                   const double* x_init, const double* x_ref, const double* a, const double* w0,
                                   int N, int64_t P, int T, int32_t* bad) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
  bool ok = true;
  for (int64_t k = tid; k < NX * NX + NX * NU; k += nt) ok = ok && isfinite(model[k]);
  if (tid < NU) {
    const double lo = model[NX * NX + NX * NU + tid], hi = model[NX * NX + NX * NU + NU + tid];
    ok = ok && isfinite(lo) && isfinite(hi) && lo <= hi;
  }
  for (int64_t k = tid; k < (int64_t)N * NX; k += nt)
    ok = ok && isfinite(Qd[k]) && Qd[k] >= 0.0 && isfinite(Qfd[k]) && Qfd[k] >= 0.0 && isfinite(x_init[k]) &&
         isfinite(x_ref[k]);
  for (int64_t k = tid; k < (int64_t)N * NU; k += nt) ok = ok && isfinite(Rd[k]) && Rd[k] > 0.0;
  for (int64_t k = tid; k < (int64_t)N * T * DP; k += nt) ok = ok && isfinite(w0[k]);
  for (int64_t k = tid; k < P * T * DP; k += nt) ok = ok && isfinite(a[k]);
  if (!ok) atomicOr(bad, 1);
}

// The single scenario's ADMM run: the same phases as the batched persistent
// kernel, in one CTA.
template <typename F, int NX, int NU, int DP>
__global__ void __launch_bounds__(64) k_noalloc_solve(Dev<F> D, const int32_t* bad) {
  if (*bad) return;
  __shared__ Model<F, NX, NU> M;
  __shared__ CtaScratch cs;
  __shared__ F kcs[AgentConst<NX, NU>::KC * 64];
  load_model<F, NX, NU>(M, D.model);
  __syncthreads();
  const ScenMeta s = D.meta[0];
  run_scenario<F, NX, NU, DP, false>(D, M, s, 0, cs, nullptr, 0, kcs);
}

__global__ void k_noalloc_results(const int32_t* status, const int32_t* iters, const double* res,
                                  const int32_t* bad, int32_t* status_iters, double* res_out) {
  if (status_iters) {
    status_iters[0] = *bad ? TADMM_INVALID_INPUT : status[0];
    status_iters[1] = *bad ? 0 : iters[0];
  }
  if (res_out) {
    res_out[0] = *bad ? CUDART_NAN : res[0];
    res_out[1] = *bad ? CUDART_NAN : res[1];
  }
}

template <int NX, int NU, int DP>
static int noalloc_run(const tadmm_scenario_dev* sc, int start_mode, double tol, int max_iter, double* X,
                       double* U, double* theta, int32_t* status_iters, double* res, cudaStream_t st) {
  using F = double;
  constexpr int E = CacheLayout<NX, NU>::E;
  const int N = sc->N, T = sc->T;
  const int64_t P = (int64_t)N * (N - 1) / 2;
  const int64_t PT = P * T, NT = (int64_t)N * T, XS = (int64_t)N * (T + 1);
  const int nm = NX * NX + NX * NU + 2 * NU;

  void* base = nullptr;
  Carve cv{nullptr};
  // first pass sizes the layout, second pass places it in the scratch array
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
      if (cv.off > (size_t)TADMM_NOALLOC_SCRATCH_BYTES)
        return set_error(TADMM_EINVAL, "scenario needs " + std::to_string(cv.off) +
                                           " bytes of solver state; the static scratch of tadmm_solve_noalloc holds " +
                                           std::to_string((size_t)TADMM_NOALLOC_SCRATCH_BYTES) + " bytes");
      int rc = scratch_address(&base, st);
      if (rc) return rc;
    }
    cv = Carve{(char*)base};
    Dev<F> D{};  // fields not set below stay zero (no residual balancing, no penalty output)
    std::memset(&D, 0, sizeof(D));
    ScenMeta* meta = cv.take<ScenMeta>(sizeof(ScenMeta));
    int32_t* order = cv.take<int32_t>(4);
    int32_t* pairs = cv.take<int32_t>(4 * P);
    int32_t* pair_scen = cv.take<int32_t>(4 * P);
    int32_t* agent_scen = cv.take<int32_t>(4 * N);
    F* model = cv.take<F>(sizeof(F) * nm);
    F* Qd = cv.take<F>(sizeof(F) * N * NX);
    F* Rd = cv.take<F>(sizeof(F) * N * NU);
    F* Qfd = cv.take<F>(sizeof(F) * N * NX);
    F* x_init = cv.take<F>(sizeof(F) * N * NX);
    F* x_ref = cv.take<F>(sizeof(F) * N * NX);
    F* a = cv.take<F>(sizeof(F) * PT * DP);
    F* w0 = cv.take<F>(sizeof(F) * NT * DP);
    F* th = cv.take<F>(sizeof(F) * 3 * PT);
    F* Xs = cv.take<F>(sizeof(F) * 2 * XS * NX);
    F* h = cv.take<F>(sizeof(F) * NT * DP);
    F* Us = cv.take<F>(sizeof(F) * NT * NU);
    F* Uss = cv.take<F>(sizeof(F) * NT * NU);
    F* cache = cv.take<F>(sizeof(F) * XS * E);
    uint16_t* Wm = cv.take<uint16_t>(2 * NT);
    uint16_t* Cm = cv.take<uint16_t>(2 * NT);
    int32_t* status = cv.take<int32_t>(4);
    int32_t* iters = cv.take<int32_t>(4);
    int32_t* cur_lvl = cv.take<int32_t>(4);
    double* resd = cv.take<double>(16);
    unsigned long long* eqp = cv.take<unsigned long long>(8);
    unsigned long long* fact = cv.take<unsigned long long>(8);
    int32_t* queue = cv.take<int32_t>(4);
    int32_t* bad = cv.take<int32_t>(4);
    if (pass == 0) continue;

    int rc0 = cuda_check(cudaMemsetAsync(bad, 0, sizeof(int32_t), st), "clear input flag");
    if (rc0) return rc0;

    k_noalloc_setup<<<grid_for(N, 64, 1024), 64, 0, st>>>(meta, order, pairs, pair_scen, agent_scen, queue, N, T,
                                                          sc->d_min, sc->rho);
    k_convert<F><<<1, 64, 0, st>>>(sc->A, model, NX * NX);
    k_convert<F><<<1, 64, 0, st>>>(sc->B, model + NX * NX, NX * NU);
    k_convert<F><<<1, 64, 0, st>>>(sc->umin, model + NX * NX + NX * NU, NU);
    k_convert<F><<<1, 64, 0, st>>>(sc->umax, model + NX * NX + NX * NU + NU, NU);
    k_convert<F><<<grid_for(N * NX, 128), 128, 0, st>>>(sc->Qd, Qd, (int64_t)N * NX);
    k_convert<F><<<grid_for(N * NU, 128), 128, 0, st>>>(sc->Rd, Rd, (int64_t)N * NU);
    k_convert<F><<<grid_for(N * NX, 128), 128, 0, st>>>(sc->Qfd, Qfd, (int64_t)N * NX);
    k_convert<F><<<grid_for(N * NX, 128), 128, 0, st>>>(sc->x_init, x_init, (int64_t)N * NX);
    k_convert<F><<<grid_for(N * NX, 128), 128, 0, st>>>(sc->x_ref, x_ref, (int64_t)N * NX);
    if (P > 0) k_import_a<F, DP><<<grid_for(P, 128), 128, 0, st>>>(meta, pair_scen, sc->a, a, P);
    k_import_w0<F, DP><<<grid_for(N, 128), 128, 0, st>>>(meta, agent_scen, sc->w0, w0, N);
    k_noalloc_validate<NX, NU, DP><<<grid_for(std::max<int64_t>(PT * DP, (int64_t)N * T * DP), 128, 1024), 128, 0, st>>>(
        model, Qd, Rd, Qfd, x_init, x_ref, a, w0, N, P, T, bad);

    D.meta = meta; D.order = order; D.pairs = pairs; D.model = model;
    D.Qd = Qd; D.Rd = Rd; D.Qfd = Qfd; D.x_init = x_init; D.x_ref = x_ref; D.a = a; D.w0 = w0;
    D.theta = th; D.X = Xs; D.h = h; D.U = Us; D.Us = Uss; D.Wm = Wm; D.Cm = Cm; D.cache = cache;
    D.tot_ps = PT; D.tot_xs = XS; D.n_scen = 1;
    D.status = status; D.iters = iters; D.cur_lvl = cur_lvl; D.res = resd; D.eqp = eqp; D.fact = fact;
    D.queue = queue;
    D.tol = tol; D.max_iter = max_iter; D.start_mode = start_mode; D.as_max = 0; D.eps_rel = 0.0;
    k_noalloc_solve<F, NX, NU, DP><<<1, 64, 0, st>>>(D, bad);
    if (X || U)
      k_export_agents<F, NX, NU><<<grid_for(N, 128), 128, 0, st>>>(D, agent_scen, N, X, U, nullptr);
    if (theta && P > 0) k_export_theta<F><<<grid_for(P, 128), 128, 0, st>>>(D, pair_scen, P, theta);
    k_noalloc_results<<<1, 1, 0, st>>>(status, iters, resd, bad, status_iters, res);
  }
  return cuda_check(cudaGetLastError(), "tadmm_solve_noalloc launches");
}

}  // namespace tadmm

extern "C" int tadmm_solve_noalloc(const tadmm_scenario_dev* sc, int32_t start_mode, double tol, int32_t max_iter,
                                   double* X, double* U, double* theta, int32_t* status_iters, double* res,
                                   void* stream) {
  using tadmm::set_error;
  if (!sc) return set_error(TADMM_EINVAL, "scenario is NULL");
  const bool d2 = sc->nx == 4 && sc->nu == 2 && sc->dp == 2;
  const bool d3 = sc->nx == 6 && sc->nu == 3 && sc->dp == 3;
  if (!d2 && !d3) return set_error(TADMM_EINVAL, "supported (nx, nu, dp): (4, 2, 2) and (6, 3, 3)");
  if (sc->N < 1 || sc->N > 32767 || sc->T < 1) return set_error(TADMM_EINVAL, "need 1 <= N <= 32767 and T >= 1");
  if (!sc->A || !sc->B || !sc->umin || !sc->umax || !sc->Qd || !sc->Rd || !sc->Qfd || !sc->x_init || !sc->x_ref ||
      !sc->w0 || (sc->N > 1 && !sc->a))
    return set_error(TADMM_EINVAL, "a required input pointer is NULL");
  if (!(sc->rho > 0.0) || !std::isfinite(sc->rho) || !std::isfinite(sc->d_min))
    return set_error(TADMM_EINVAL, "need rho > 0 and finite d_min");
  if (start_mode < 0 || start_mode > 2) return set_error(TADMM_EINVAL, "start_mode must be 0, 1 or 2");
  if (!(tol >= 0.0) || !std::isfinite(tol) || max_iter < 1) return set_error(TADMM_EINVAL, "need tol >= 0, max_iter >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  if (d2) return tadmm::noalloc_run<4, 2, 2>(sc, start_mode, tol, max_iter, X, U, theta, status_iters, res, st);
  return tadmm::noalloc_run<6, 3, 3>(sc, start_mode, tol, max_iter, X, U, theta, status_iters, res, st);
}
