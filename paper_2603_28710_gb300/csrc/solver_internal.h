// The solver handle (shared by the single-solver C ABI in host.cu and the batched solver
// in batch_host.cu) and the helpers that build per-stage kernel arguments.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/adg.h"
#include "adg_internal.h"

struct adg_solver {
  adg_mesh mesh{};
  int dim = 2, degree = 1, N = 2, ND = 4, NF = 2, NV = 4;
  int64_t ne = 0, ndof = 0;
  int P[3] = {1, 1, 1};
  int max_delay = 0;
  adg_flux flux = ADG_FLUX_SYNC;
  adg_options opt{};
  int np = 1;
  int stages = 0;
  bool rk2n = false;
  double rka[8] = {0}, rkb[8] = {0}, rkc[8] = {0};
  double h[3] = {1, 1, 1};
  double J = 1.0;
  int prec = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // device memory
  double* w = nullptr;
  void* x = nullptr;         // 2R: r ; 2N: q (operator storage type)
  void* tr = nullptr;        // traces of the current stage input
  void* tr_alt = nullptr;    // fused and element paths: traces of the next stage input (swapped with tr)
  void* fl = nullptr;        // face fluxes
  void* ring = nullptr;      // delayed-flux history
  int32_t* pe_slot = nullptr;
  int32_t* pe_iface = nullptr;
  adg::OpTables* tab_dev = nullptr;
  double* red_partial = nullptr;
  double* red_out = nullptr;
  int* flag = nullptr;
  double* tmp_u = nullptr;
  double* tmp_k = nullptr;
  int red_blocks = 0;
  adg::OpTables tab{};
  adg::MeshArgs margs{};
  int64_t npe = 0;
  int depth = 0, head = -1, n_iface = 0;
  // run state
  bool has_state = false, traces_valid = false;
  int64_t step = 0;
  double t = 0.0, dt = 0.0;
  std::string err;
  // learned ghost-trace predictor and trace logging
  int32_t* pe_face_d = nullptr;   // [slot] direction of the PE face
  int32_t* pe_face_e = nullptr;   // [slot] element on its low side
  uint16_t* mlp = nullptr;        // BF16 parameters (device)
  void* lw_E = nullptr;           // learned-mode per-channel work buffers
  double* lw_s = nullptr;
  float* lw_x = nullptr;
  float* lw_y = nullptr;
  float trust = 1.0f;
  double* log = nullptr;          // caller's device buffer of PE-face trace records
  int64_t log_cap = 0, log_count = 0;
  // fused per-stage kernel (ADG_PATH_FUSED)
  bool fused = false;          // adg_step takes the fused path
  bool faces = false;          // adg_step takes the element path (ADG_PATH_ELEMENT)
  bool traces_partial = false; // tr holds only tile-boundary traces (after fused stages)
  int tile[3] = {1, 1, 1}, ntile[3] = {1, 1, 1};
  int tma = 0;                 // tiles staged by TMA tensor copies
  CUtensorMap tm_w{}, tm_x{};  // tensor maps of w and x: [var][z][y][x * nodes]
  int* kerr = nullptr;         // device error code of bounded waits
  // kernel timing (adg_set_profiling)
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_kind;  // kind of each recorded pair
  size_t ev_used = 0;
  double prof_ms[2] = {0.0, 0.0};  // totals folded from the pool when it filled up
  int64_t prof_n[2] = {0, 0};
};

namespace adg {
// (hi, lo) FP32 pair of a value
float2 split2(long double v);
// Flux-kernel arguments of RK stage m with every static field set (AT weights for all
// delays the schedule can produce); the per-step fields (store, head, delay, step) are 0.
FluxArgs stage_flux_args(const adg_solver* s, int m);
// Volume-kernel arguments of RK stage m (needs the time step, i.e. a state was set).
VolArgs stage_vol_args(const adg_solver* s, int m);
}  // namespace adg
