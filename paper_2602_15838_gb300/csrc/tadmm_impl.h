// Host-side state of a tadmm handle and the per-precision / per-dimension
// implementation entry points (explicitly instantiated in tadmm_f64.cu and
// tadmm_f32.cu).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/tadmm.h"
#include "tadmm_device.cuh"

// Scratch of the implicit-KKT backward pass (grown on demand).
struct BwdBufs {
  void *act = nullptr, *cnt = nullptr, *amask = nullptr, *psi = nullptr, *kks = nullptr, *pos0 = nullptr,
       *force = nullptr, *Xp = nullptr, *Up = nullptr, *Wx = nullptr, *Wu = nullptr, *bstat = nullptr,
       *bs = nullptr, *S = nullptr, *vec = nullptr, *gX = nullptr, *gout = nullptr, *xpol = nullptr,
       *piv = nullptr, *ndep = nullptr, *hmask = nullptr, *Wb = nullptr, *pchg = nullptr, *set_act = nullptr,
       *set_W = nullptr;
  size_t act_cap = 0, cnt_cap = 0, amask_cap = 0, psi_cap = 0, kks_cap = 0, pos0_cap = 0, force_cap = 0,
         Xp_cap = 0, Up_cap = 0, Wx_cap = 0, Wu_cap = 0, bstat_cap = 0, bs_cap = 0, S_cap = 0, vec_cap = 0,
         gX_cap = 0, gout_cap = 0, xpol_cap = 0, piv_cap = 0, ndep_cap = 0, hmask_cap = 0, Wb_cap = 0,
         pchg_cap = 0, set_act_cap = 0, set_W_cap = 0;
};

struct tadmm_handle {
  int prec = 64, nx = 0, nu = 0, dp = 0, n_scen = 0;
  int64_t tot_agents = 0, tot_as = 0, tot_ps = 0, tot_xs = 0, tot_pairs = 0;
  tadmm_options opt{};
  std::vector<int32_t> N, T;
  std::vector<tadmm::ScenMeta> meta_h;
  int device = 0, sm_count = 0;

  // device state
  tadmm::ScenMeta* meta = nullptr;
  int32_t* order = nullptr;
  int32_t* goff = nullptr;      // scenario groups of the persistent kernel
  int32_t* gmem = nullptr;
  int32_t* gorder = nullptr;
  int n_groups = 0;
  int max_group_pairs = 0;
  int32_t* pairs = nullptr;
  int32_t* deg = nullptr;       // [tot_agents] copies per agent
  int32_t* adj_ptr = nullptr;   // [tot_agents + 1]
  int32_t* adj = nullptr;       // listed-pair adjacency (sparse scenarios)
  std::vector<int32_t> pair_count_h, pair_ij_h;  // caller's pair lists (empty: all pairs)
  int32_t* pair_scen = nullptr;
  int32_t* agent_scen = nullptr;
  void* model = nullptr;
  void* Qd = nullptr;
  void* Rd = nullptr;
  void* Qfd = nullptr;
  void* x_init = nullptr;
  void* x_ref = nullptr;
  void* a = nullptr;
  void* w0 = nullptr;
  void* theta = nullptr;
  void* models = nullptr;        // heterogeneous agents: [tot_agents] per-agent model (A, B, umin, umax)
  double* st_models = nullptr;   // their float64 staging
  std::vector<double> models_h;  // host packing of the caller's per-agent A, B (kept for async copies)
  int hetero = 0;                // 1: per-agent dynamics
  void* phi = nullptr;           // over-relaxation: [tot_ps] pair part of the consensus copies
  void* sx = nullptr;            // over-relaxation: [tot_as][dp] agent part of the consensus copies
  void* hprev = nullptr;         // homotopy hot start: [tot_as][dp] previous coupling terms
  void* hmu = nullptr;           //   [tot_as][nu] bound multipliers of the previous optimum
  void* hdmu = nullptr;          //   [tot_as][nu] their segment direction
  void* X = nullptr;
  void* h = nullptr;
  void* U = nullptr;
  void* Us = nullptr;
  void* cache = nullptr;
  uint16_t* Wm = nullptr;
  uint16_t* Cm = nullptr;
  int32_t* status = nullptr;
  int32_t* iters = nullptr;
  int32_t* cur_lvl = nullptr;
  double* res = nullptr;
  unsigned long long* eqp = nullptr;
  unsigned long long* fact = nullptr;
  double* rho_out = nullptr;     // [n_scen] penalty at the end of the last solve
  int32_t* rho_chg = nullptr;    // [n_scen] residual-balancing changes of the last solve
  int32_t* queue = nullptr;

  // float64 staging in the caller's layouts (imports and exports)
  double* st_model = nullptr;   // A, B, umin, umax
  double* st_agent = nullptr;   // Qd, Rd, Qfd, x_init, x_ref (5 blocks)
  double* st_a = nullptr;       // [tot_ps][dp]
  double* st_w0 = nullptr;      // [tot_as][dp]
  double* ex_buf = nullptr;     // export scratch
  double* st_costs = nullptr;   // tadmm_update_costs: float64 staging of Qd, Rd, Qfd, x_ref before validation
  int32_t* cost_flag = nullptr; //   its device-side validation flag
  double* sqp_buf = nullptr;     // tadmm_sqp: [n_scen] objective | [n_scen] min distance | [n_scen] uint8 keep mask
  size_t ex_bytes = 0;

  // plain mode
  int32_t* flag = nullptr;               // device: agent QP failure code
  unsigned long long* red2 = nullptr;    // device: residual maxima bits
  void* pinned = nullptr;                // host pinned readback buffer

  // batched mode launch shape and captured graph
  int tpc = 0, cps = 0, variant = 0;
  int di = 0;               // model is an exact double integrator (structured kernel path)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  double g_tol = -1.0;
  int g_iter = -1, g_tpc = -1, g_cps = -1, g_var = -1;
  int solved = 0;
  int bwd_polished = 0;     // the backward active set was refined by tadmm_polish after the last solve
  int64_t launches = 0;   // kernel launches enqueued by the last solve
  BwdBufs bwd;

  // graph mode (conditional WHILE node over the per-iteration phase kernels)
  void *gs_iter = nullptr, *gs_active = nullptr, *gs_need = nullptr, *gs_fail = nullptr, *gs_rb = nullptr,
       *gs_sb = nullptr;
  void* gs_blk = nullptr;   // int2 (scenario, first agent) per 32-agent gather block
  int n_gblk = 0;
  cudaGraphExec_t wexec = nullptr;
  double w_tol = -1.0;
  int w_iter = -1;
};

namespace tadmm {

int set_error(int code, const std::string& msg);
int cuda_check(cudaError_t e, const char* what);

template <typename F, int NX, int NU, int DP>
struct Impl {
  static int import_inputs(tadmm_handle* h, cudaStream_t st);
  static int solve_batched(tadmm_handle* h, double tol, int max_iter, cudaStream_t st);
  static int solve_plain(tadmm_handle* h, double tol, int max_iter, cudaStream_t st);
  static int solve_graph(tadmm_handle* h, double tol, int max_iter, cudaStream_t st);
  static int export_solution(tadmm_handle* h, double* X, double* U, double* theta, int8_t* W,
                             cudaStream_t st);
  static int max_ctas_per_sm(int tpc, int variant, const tadmm_handle* h);
  static int backward(tadmm_handle* h, const double* gX_dev, double theta_eps, double* gout_dev, double* xpol_dev,
                      cudaStream_t st);
  static int relinearize(tadmm_handle* h, const uint8_t* keep, cudaStream_t st);
  static int sqp_measure(tadmm_handle* h, double* J, double* dmin, cudaStream_t st);
  static int import_costs(tadmm_handle* h, int which, cudaStream_t st);
  static int polish(tadmm_handle* h, double theta_eps, int max_rounds, double kkt_tol, uint8_t* act_dev, int8_t* W_dev,
                    int32_t* status, int32_t* rounds, cudaStream_t st);
};

}  // namespace tadmm
