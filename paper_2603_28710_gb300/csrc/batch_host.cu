// Batched solver: many independent instances (different meshes, degrees and delays)
// advanced together.  Instances of the same dimension and degree form a group; per RK
// stage every group runs one persistent flux launch and one persistent volume launch over
// all of its instances.  A whole step (schedule kernel + all stage launches) is captured
// once into a CUDA graph and replayed; an autotuner picks each group's element tile.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/adg.h"
#include "batch.cuh"
#include "solver_internal.h"

namespace adg {
cudaError_t batch_vol_fp64(int, int, int, const VolArgs*, const FluxArgs*, int, int, const BatchGroupArgs&, int, cudaStream_t, int*);
cudaError_t batch_vol_fp32(int, int, int, const VolArgs*, const FluxArgs*, int, int, const BatchGroupArgs&, int, cudaStream_t, int*);
cudaError_t batch_vol_df64(int, int, int, const VolArgs*, const FluxArgs*, int, int, const BatchGroupArgs&, int, cudaStream_t, int*);
cudaError_t batch_flux_fp64(int, int, const FluxArgs*, int, int, const BatchGroupArgs&, int, cudaStream_t, int*);
cudaError_t batch_flux_fp32(int, int, const FluxArgs*, int, int, const BatchGroupArgs&, int, cudaStream_t, int*);
cudaError_t batch_flux_df64(int, int, const FluxArgs*, int, int, const BatchGroupArgs&, int, cudaStream_t, int*);
void noalloc_set_error(const char* msg);

namespace {

// One thread per instance: communication flag, delay counter and ring head of the step
// about to run (closed forms of Algorithms 2 and 3), written into every stage's flux
// arguments; then the step counter advances.
__global__ void batch_schedule_kernel(BatchSched* sc, FluxArgs* fa, int nstages, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  BatchSched s = sc[i];
  const long long step = s.step;
  int comm = 1, k = 0;
  if (!s.random && s.pe) {
    if (s.flux_kind == 1) {
      k = (int)(step % s.L);
      comm = (k == 0);
    } else if (s.flux_kind >= 2) {
      const long long cyc = (long long)s.L + s.np + 1;
      const int ph = (int)(step % cyc);
      comm = ph < s.np + 1;
      k = comm ? 0 : ph - s.np;
    }
  }
  const int store = s.pe && (s.random || comm);
  if (store) s.head = (s.head + 1) % s.depth;
  for (int m = 0; m < nstages; ++m) {
    FluxArgs& A = fa[i * nstages + m];
    A.store = (store && m == 0) ? 1 : 0;
    A.head = s.head < 0 ? 0 : s.head;
    A.uniform_delay = s.random ? 0 : (comm ? 0 : k);
    A.step = step;
  }
  s.step = step + 1;
  sc[i] = s;
}

// occ != nullptr: no launch, *occ = resident blocks per SM of the kernel; fa != nullptr:
// the element-path kernel (face fluxes evaluated in the volume launch)
cudaError_t vol_launch(int prec, int dim, int N, int tt, const VolArgs* va, const FluxArgs* fa,
                       int ns, int st, const BatchGroupArgs& g, int grid, cudaStream_t s,
                       int* occ = nullptr) {
  switch (prec) {
    case 0: return batch_vol_fp64(dim, N, tt, va, fa, ns, st, g, grid, s, occ);
    case 1: return batch_vol_fp32(dim, N, tt, va, fa, ns, st, g, grid, s, occ);
    case 2: return batch_vol_df64(dim, N, tt, va, fa, ns, st, g, grid, s, occ);
  }
  return cudaErrorInvalidValue;
}

cudaError_t flux_launch(int prec, int dim, int N, const FluxArgs* fa, int ns, int st,
                        const BatchGroupArgs& g, int grid, cudaStream_t s, int* occ = nullptr) {
  switch (prec) {
    case 0: return batch_flux_fp64(dim, N, fa, ns, st, g, grid, s, occ);
    case 1: return batch_flux_fp32(dim, N, fa, ns, st, g, grid, s, occ);
    case 2: return batch_flux_df64(dim, N, fa, ns, st, g, grid, s, occ);
  }
  return cudaErrorInvalidValue;
}

int ipow(int b, int e) {
  int r = 1;
  while (e-- > 0) r *= b;
  return r;
}

}  // namespace
}  // namespace adg

using namespace adg;

struct adg_batch {
  std::vector<adg_solver*> inst;
  int n = 0, prec = 0, stages = 0, dim = 2;
  cudaStream_t stream = nullptr;
  VolArgs* va_dev = nullptr;
  FluxArgs* fa_dev = nullptr;
  BatchSched* sc_dev = nullptr;
  std::vector<VolArgs> va_host;
  std::vector<FluxArgs> fa_host;
  std::vector<BatchSched> sc_host;
  std::vector<char> has_state;
  std::vector<int64_t> inst_steps;  // steps taken since each instance's state was set
  // element path (FP32 operator): one volume launch per group and stage, every element
  // evaluating the fluxes on its own faces; no face-flux launch.  Traces cycle through the
  // instance's two trace buffers and, for an odd stage count, a third one (tr3), so that
  // every step ends with the current traces in the instance's own buffer again and the
  // graph's per-stage arguments stay fixed.
  bool faces = false;
  std::vector<void*> tr3;
  struct Group {
    int N = 0, tt = 128;
    std::vector<int> inst;   // all instances of the degree
    std::vector<int> finst;  // instances in the graph's face-flux launch
    std::vector<int> vinst;  // instances in the persistent volume launch
    std::vector<int> solo;   // instances with a volume launch of their own
    std::vector<int> handles;  // instances stepped as separate handles, outside the graph
    int* inst_dev = nullptr;  // the flux launch's instances (finst)
    int* vinst_dev = nullptr;
    int* voff_dev = nullptr;
    int* foff_dev = nullptr;
    int vtotal = 0, ftotal = 0;
    int vgrid = 0, fgrid = 0;
    int vpersist = 1, fpersist = 1;  // one resident wave looping over tiles, or a block per tile
    int solo_waves = 4;  // instances filling the GPU this many times get a volume launch of
                         // their own (0: none do)
    int handle_waves = 0;  // instances filling the GPU this many times are stepped as
                           // separate handles (0: none are)
  };
  std::vector<Group> groups;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  int64_t steps = 0;
  std::string err;
};

namespace {

adg_status bfail(adg_batch* b, adg_status st, const std::string& m) {
  if (b) b->err = m;
  else noalloc_set_error(m.c_str());
  return st;
}

#define BCUDA(B, call)                                                                        \
  do {                                                                                        \
    cudaError_t e__ = (call);                                                                 \
    if (e__ != cudaSuccess)                                                                   \
      return bfail((B), e__ == cudaErrorMemoryAllocation ? ADG_ERR_OOM : ADG_ERR_CUDA,        \
                   std::string(#call) + ": " + cudaGetErrorString(e__));                      \
  } while (0)

void drop_graph(adg_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

void free_batch(adg_batch* b) {
  drop_graph(b);
  for (auto& g : b->groups) {
    if (g.inst_dev) cudaFree(g.inst_dev);
    if (g.vinst_dev) cudaFree(g.vinst_dev);
    if (g.voff_dev) cudaFree(g.voff_dev);
    if (g.foff_dev) cudaFree(g.foff_dev);
  }
  for (void* p : b->tr3)
    if (p) cudaFree(p);
  if (b->va_dev) cudaFree(b->va_dev);
  if (b->fa_dev) cudaFree(b->fa_dev);
  if (b->sc_dev) cudaFree(b->sc_dev);
  for (adg_solver* s : b->inst) adg_destroy(s);
}

// persistent grid: one wave of resident blocks (per_sm from the occupancy calculator), never
// more blocks than virtual blocks; a second partial wave would run a share of the work at
// low occupancy after the first wave ends
int persistent_grid(int total, int per_sm) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(1, std::min(total, sms * per_sm));
}

// An instance whose volume tiles fill the GPU solo_waves times over (default 4; the
// autotuner also tries 1 and never) gets a volume launch of its own -- the single-handle
// kernel, arguments in the kernel's parameter bank -- instead of a share of the persistent
// launch: a persistent block reads its instance's arguments from shared memory, which costs
// registers and hence occupancy, while small instances gain more from sharing one launch.

// Split of a group into batched and solo volume work, and virtual-block offsets, for the
// chosen tile and launch shapes.
adg_status layout_group(adg_batch* b, adg_batch::Group& g) {
  const int nd = ipow(g.N, b->dim), nf = nd / g.N;
  const int epb = std::max(1, g.tt / nd);
  int vocc = 0, focc = 0, dev = 0, sms = 152;
  // (a non-null flux pointer selects the element-path kernel; nothing is launched)
  BCUDA(b, vol_launch(b->prec, b->dim, g.N, g.tt, nullptr, b->faces ? b->fa_dev : nullptr, 0, 0,
                      BatchGroupArgs{}, 0, 0, &vocc));
  BCUDA(b, flux_launch(b->prec, b->dim, g.N, nullptr, 0, 0, BatchGroupArgs{}, 0, 0, &focc));
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t wave = (int64_t)sms * std::max(1, vocc);
  g.vinst.clear();
  g.solo.clear();
  g.finst.clear();
  g.handles.clear();
  for (int i : g.inst) {
    const int64_t tiles = (b->inst[i]->ne + epb - 1) / epb;
    if (g.handle_waves > 0 && tiles >= g.handle_waves * wave) {
      g.handles.push_back(i);
      continue;
    }
    g.finst.push_back(i);
    // (the element path has no solo launches: its face rules live in device memory)
    (!b->faces && g.solo_waves > 0 && tiles >= g.solo_waves * wave ? g.solo : g.vinst).push_back(i);
  }
  std::vector<int> voff(g.vinst.size() + 1), foff(g.finst.size() + 1);
  voff[0] = foff[0] = 0;
  for (size_t k = 0; k < g.vinst.size(); ++k)
    voff[k + 1] = voff[k] + (int)((b->inst[g.vinst[k]]->ne + epb - 1) / epb);
  for (size_t k = 0; k < g.finst.size(); ++k)
    foff[k + 1] = foff[k] + b->dim * (int)((b->inst[g.finst[k]]->ne * nf + 255) / 256);
  g.vtotal = voff.back();
  g.ftotal = foff.back();
  g.vgrid = g.vpersist ? persistent_grid(g.vtotal, std::max(1, vocc)) : g.vtotal;
  g.fgrid = g.fpersist ? persistent_grid(g.ftotal, std::max(1, focc)) : g.ftotal;
  if (!g.vinst.empty())
    BCUDA(b, cudaMemcpy(g.vinst_dev, g.vinst.data(), g.vinst.size() * sizeof(int),
                        cudaMemcpyHostToDevice));
  if (!g.finst.empty())
    BCUDA(b, cudaMemcpy(g.inst_dev, g.finst.data(), g.finst.size() * sizeof(int),
                        cudaMemcpyHostToDevice));
  BCUDA(b, cudaMemcpy(g.voff_dev, voff.data(), voff.size() * sizeof(int), cudaMemcpyHostToDevice));
  BCUDA(b, cudaMemcpy(g.foff_dev, foff.data(), foff.size() * sizeof(int), cudaMemcpyHostToDevice));
  return ADG_OK;
}

BatchGroupArgs group_args(const adg_batch::Group& g, bool vol) {
  BatchGroupArgs a;
  a.inst = vol ? g.vinst_dev : g.inst_dev;
  a.off = vol ? g.voff_dev : g.foff_dev;
  a.n = (int)(vol ? g.vinst.size() : g.finst.size());
  a.total = vol ? g.vtotal : g.ftotal;
  return a;
}

// volume work of a group at stage m: the persistent launch and the solo launches
adg_status vol_group(adg_batch* b, adg_batch::Group& g, int m, cudaStream_t s) {
  if (!g.vinst.empty())
    BCUDA(b, vol_launch(b->prec, b->dim, g.N, g.tt, b->va_dev, b->faces ? b->fa_dev : nullptr,
                        b->stages, m, group_args(g, true), g.vgrid, s));
  for (int i : g.solo)
    BCUDA(b, launch_vol(b->prec, b->dim, g.N, b->va_host[i * b->stages + m], s));
  return ADG_OK;
}

// enqueue one full step: schedule kernel, then flux and volume launches of every group
adg_status enqueue_step(adg_batch* b, cudaStream_t s) {
  batch_schedule_kernel<<<(b->n + 127) / 128, 128, 0, s>>>(b->sc_dev, b->fa_dev, b->stages, b->n);
  BCUDA(b, cudaGetLastError());
  for (int m = 0; m < b->stages; ++m) {
    for (auto& g : b->groups)
      if (!g.finst.empty() && !b->faces)
        BCUDA(b, flux_launch(b->prec, b->dim, g.N, b->fa_dev, b->stages, m, group_args(g, false),
                             g.fgrid, s));
    for (auto& g : b->groups) {
      adg_status st = vol_group(b, g, m, s);
      if (st != ADG_OK) return st;
    }
  }
  return ADG_OK;
}

// The step is captured on a private stream (the legacy default stream cannot be captured);
// the instantiated graph is then launched on the caller's stream.
adg_status build_graph(adg_batch* b) {
  drop_graph(b);
  cudaStream_t cap = nullptr;
  BCUDA(b, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cap);
    BCUDA(b, e);
  }
  adg_status st = enqueue_step(b, cap);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(cap, &g);
  cudaStreamDestroy(cap);
  if (st != ADG_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  BCUDA(b, e);
  b->graph = g;
  BCUDA(b, cudaGraphInstantiate(&b->exec, g, 0));
  return ADG_OK;
}

adg_status refresh_instance(adg_batch* b, int i) {
  adg_solver* s = b->inst[i];
  for (int m = 0; m < b->stages; ++m) {
    b->va_host[i * b->stages + m] = stage_vol_args(s, m);
    b->fa_host[i * b->stages + m] = stage_flux_args(s, m);
  }
  if (b->faces) {
    // stage m reads the traces in X[in(m)] and writes the next stage's into X[out(m)]:
    // X0 -> X1 -> X0 -> ... and, for an odd stage count, X1 -> X2 -> X0 at the end
    void* X[3] = {s->tr, s->tr_alt, b->tr3[i]};
    const int S = b->stages;
    for (int m = 0; m < S; ++m) {
      int in = m & 1, out = (m + 1) & 1;
      if (S & 1) {
        if (m == S - 2) out = 2;
        if (m == S - 1) {
          in = 2;
          out = 0;
        }
      }
      b->fa_host[i * S + m].tr = X[in];
      b->va_host[i * S + m].tr = X[out];
    }
  }
  BatchSched sc;
  std::memset(&sc, 0, sizeof(sc));
  sc.random = s->opt.delay_mode == ADG_DELAY_RANDOM;
  sc.pe = (s->flux != ADG_FLUX_SYNC && s->npe > 0) ? 1 : 0;
  sc.flux_kind = (int)s->flux;
  sc.L = s->max_delay;
  sc.np = s->np;
  sc.depth = s->depth;
  sc.head = -1;
  sc.step = 0;
  b->sc_host[i] = sc;
  BCUDA(b, cudaMemcpyAsync(b->va_dev + i * b->stages, &b->va_host[i * b->stages],
                           sizeof(VolArgs) * b->stages, cudaMemcpyHostToDevice, b->stream));
  BCUDA(b, cudaMemcpyAsync(b->fa_dev + i * b->stages, &b->fa_host[i * b->stages],
                           sizeof(FluxArgs) * b->stages, cudaMemcpyHostToDevice, b->stream));
  BCUDA(b, cudaMemcpyAsync(b->sc_dev + i, &b->sc_host[i], sizeof(BatchSched),
                           cudaMemcpyHostToDevice, b->stream));
  BCUDA(b, cudaStreamSynchronize(b->stream));
  drop_graph(b);  // solo volume launches hold the instance's arguments by value
  b->has_state[i] = 1;
  b->inst_steps[i] = 0;
  return ADG_OK;
}

// one step of the instances stepped as separate handles (their own host schedule and
// single-handle launches, on the batch's stream after the graph's work)
adg_status step_handles(adg_batch* b) {
  for (auto& g : b->groups)
    for (int i : g.handles) {
      adg_status st = adg_step(b->inst[i], 1);
      if (st != ADG_OK) return bfail(b, st, adg_last_error(b->inst[i]));
    }
  return ADG_OK;
}

}  // namespace

extern "C" {

adg_status adg_batch_create(int n, const adg_mesh* meshes, const int* degrees, const int* P,
                            const int* max_delay, adg_flux flux, const adg_options* opt,
                            adg_batch** out) {
  if (!out) return bfail(nullptr, ADG_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (n < 1 || !meshes || !degrees || !P || !max_delay)
    return bfail(nullptr, ADG_ERR_INVALID, "need n >= 1 and non-NULL meshes, degrees, P, max_delay");
  if (flux == ADG_FLUX_LEARNED)
    return bfail(nullptr, ADG_ERR_UNSUPPORTED, "the learned flux is not available in batches");
  adg_options o;
  if (opt) o = *opt;
  else adg_default_options(&o);
  // the batched kernels run the split path's element code; the instances the batch steps
  // as separate handles take the split or element path (both give the split path's bits),
  // so results equal separate split-path handles bit for bit
  if (o.kernel_path == ADG_PATH_FUSED) o.kernel_path = ADG_PATH_SPLIT;
  adg_batch* b = new (std::nothrow) adg_batch();
  if (!b) return bfail(nullptr, ADG_ERR_OOM, "host allocation failed");
  b->n = n;
  b->prec = (int)o.precision;
  b->stream = (cudaStream_t)o.cuda_stream;
  b->dim = meshes[0].dim;
  for (int i = 0; i < n; ++i) {
    if (meshes[i].dim != b->dim) {
      free_batch(b);
      delete b;
      return bfail(nullptr, ADG_ERR_INVALID, "all instances must have the same dimension");
    }
    adg_solver* s = nullptr;
    adg_status st = adg_create(&meshes[i], degrees[i], &P[3 * i], max_delay[i], flux, &o, &s);
    if (st != ADG_OK) {
      std::string msg = std::string("instance ") + std::to_string(i) + ": " + adg_last_error(nullptr);
      free_batch(b);
      delete b;
      return bfail(nullptr, st, msg);
    }
    b->inst.push_back(s);
  }
  b->stages = b->inst[0]->stages;
  // the FP32 operator takes the element path unless the split path was asked for (the
  // instance handles then hold their second trace buffer)
  b->faces = o.precision == ADG_PREC_FP32 && o.kernel_path != ADG_PATH_SPLIT;
  b->tr3.assign(n, nullptr);
  b->va_host.resize((size_t)n * b->stages);
  b->fa_host.resize((size_t)n * b->stages);
  b->sc_host.resize(n);
  b->has_state.assign(n, 0);
  b->inst_steps.assign(n, 0);
  std::map<int, std::vector<int>> by_n;
  for (int i = 0; i < n; ++i) by_n[b->inst[i]->N].push_back(i);
  cudaError_t ce = cudaMalloc((void**)&b->va_dev, sizeof(VolArgs) * n * b->stages);
  if (ce == cudaSuccess) ce = cudaMalloc((void**)&b->fa_dev, sizeof(FluxArgs) * n * b->stages);
  if (ce == cudaSuccess) ce = cudaMalloc((void**)&b->sc_dev, sizeof(BatchSched) * n);
  for (int i = 0; i < n && ce == cudaSuccess && b->faces && (b->stages & 1); ++i) {
    const adg_solver* si = b->inst[i];
    const size_t ntr = (size_t)2 * si->dim * si->NV * si->ne * si->NF;
    ce = cudaMalloc(&b->tr3[i], ntr * storage_bytes(b->prec));
  }
  for (auto& kv : by_n) {
    adg_batch::Group g;
    g.N = kv.first;
    g.inst = kv.second;
    const size_t k = g.inst.size();
    if (ce == cudaSuccess) ce = cudaMalloc((void**)&g.inst_dev, k * sizeof(int));
    if (ce == cudaSuccess) ce = cudaMalloc((void**)&g.vinst_dev, k * sizeof(int));
    if (ce == cudaSuccess) ce = cudaMalloc((void**)&g.voff_dev, (k + 1) * sizeof(int));
    if (ce == cudaSuccess) ce = cudaMalloc((void**)&g.foff_dev, (k + 1) * sizeof(int));
    b->groups.push_back(g);
  }
  if (ce != cudaSuccess) {
    std::string msg = std::string("adg_batch_create: ") + cudaGetErrorString(ce);
    free_batch(b);
    delete b;
    return bfail(nullptr, ce == cudaErrorMemoryAllocation ? ADG_ERR_OOM : ADG_ERR_CUDA, msg);
  }
  for (auto& g : b->groups) {
    adg_status st = layout_group(b, g);
    if (st != ADG_OK) {
      std::string msg = b->err;
      free_batch(b);
      delete b;
      return bfail(nullptr, st, msg);
    }
  }
  *out = b;
  return ADG_OK;
}

adg_status adg_batch_init_vortex(adg_batch* b, int i, double beta, double x0, double y0) {
  if (!b) return bfail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  if (i < 0 || i >= b->n) return bfail(b, ADG_ERR_INVALID, "instance index out of range");
  adg_status st = adg_init_vortex(b->inst[i], 0.0, beta, x0, y0);
  if (st != ADG_OK) return bfail(b, st, adg_last_error(b->inst[i]));
  return refresh_instance(b, i);
}

adg_status adg_batch_set_state(adg_batch* b, int i, const double* u, int64_t count, int on_device) {
  if (!b) return bfail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  if (i < 0 || i >= b->n) return bfail(b, ADG_ERR_INVALID, "instance index out of range");
  adg_status st = adg_set_state(b->inst[i], u, count, on_device);
  if (st != ADG_OK) return bfail(b, st, adg_last_error(b->inst[i]));
  return refresh_instance(b, i);
}

adg_status adg_batch_step(adg_batch* b, int n_steps) {
  if (!b) return bfail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  if (n_steps < 0) return bfail(b, ADG_ERR_INVALID, "n_steps must be >= 0");
  for (int i = 0; i < b->n; ++i)
    if (!b->has_state[i]) return bfail(b, ADG_ERR_STATE, "instance " + std::to_string(i) + " has no state");
  if (!b->exec) {
    adg_status st = build_graph(b);
    if (st != ADG_OK) return st;
  }
  bool graph_work = false;
  for (auto& g : b->groups) graph_work = graph_work || !g.finst.empty();
  for (int it = 0; it < n_steps; ++it) {
    if (graph_work) BCUDA(b, cudaGraphLaunch(b->exec, b->stream));
    adg_status st = step_handles(b);
    if (st != ADG_OK) return st;
  }
  b->steps += n_steps;
  for (int i = 0; i < b->n; ++i) b->inst_steps[i] += n_steps;
  return ADG_OK;
}

adg_status adg_batch_autotune(adg_batch* b, int trials, int* tile_threads) {
  if (!b) return bfail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  if (trials < 1) trials = 3;
  // uniform flow in every instance: the tuner times real launches on real buffers
  for (int i = 0; i < b->n; ++i) {
    adg_solver* s = b->inst[i];
    std::vector<double> u((size_t)s->ndof);
    const int64_t per = s->ne * s->ND;
    for (int v = 0; v < s->NV; ++v)
      for (int64_t q = 0; q < per; ++q)
        u[v * per + q] = (v == 0) ? 1.0 : (v == s->NV - 1 ? 2.5 : 0.0);
    adg_status st = adg_set_state(s, u.data(), s->ndof, 0);
    if (st != ADG_OK) return bfail(b, st, adg_last_error(s));
    st = refresh_instance(b, i);
    if (st != ADG_OK) return st;
  }
  drop_graph(b);
  cudaEvent_t e0, e1;
  BCUDA(b, cudaEventCreate(&e0));
  BCUDA(b, cudaEventCreate(&e1));
  // time `trials` launches (after one warm-up) of the group's volume work at stage 0 (it
  // reads only the solution, never the RK register: the persistent launch and the solo
  // launches of its split for the tile) or of its face-flux kernel
  auto time_group = [&](adg_batch::Group& g, bool vol, float* ms) -> adg_status {
    for (int t = 0; t <= trials; ++t) {
      if (t == 1) BCUDA(b, cudaEventRecord(e0, b->stream));
      if (vol) {
        adg_status st = vol_group(b, g, 0, b->stream);
        if (st != ADG_OK) return st;
      } else
        BCUDA(b, flux_launch(b->prec, b->dim, g.N, b->fa_dev, b->stages, 0,
                             group_args(g, false), g.fgrid, b->stream));
    }
    BCUDA(b, cudaEventRecord(e1, b->stream));
    BCUDA(b, cudaEventSynchronize(e1));
    BCUDA(b, cudaEventElapsedTime(ms, e0, e1));
    return ADG_OK;
  };
  const int cand[3] = {64, 128, 256};
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    auto& g = b->groups[gi];
    float best = 1e30f, ms = 0.f;
    int best_tt = 128, best_vp = 1, best_fp = 1, best_sw = 4;
    // volume kernel: tile size x launch shape x which instances run the single-handle
    // launch (those filling the GPU 1 or 4 times over, or none)
    const int solo_cand[3] = {4, 1, 0};
    const int nsolo = b->faces ? 1 : 3;  // the element path has no solo launches
    for (int tt : cand)
      for (int vp = 1; vp >= 0; --vp)
        for (int si = 0; si < nsolo; ++si) {
          const int sw = solo_cand[si];
          g.tt = tt;
          g.vpersist = vp;
          g.solo_waves = sw;
          adg_status st = layout_group(b, g);
          if (st == ADG_OK) st = time_group(g, true, &ms);
          if (st != ADG_OK) return st;
          if (ms < best) {
            best = ms;
            best_tt = tt;
            best_vp = vp;
            best_sw = sw;
          }
        }
    g.tt = best_tt;
    g.vpersist = best_vp;
    g.solo_waves = best_sw;
    // face-flux kernel: launch shape (none on the element path)
    best = 1e30f;
    for (int fp = 1; fp >= 0 && !b->faces; --fp) {
      g.fpersist = fp;
      adg_status st = layout_group(b, g);
      if (st == ADG_OK) st = time_group(g, false, &ms);
      if (st != ADG_OK) return st;
      if (ms < best) {
        best = ms;
        best_fp = fp;
      }
    }
    g.fpersist = best_fp;
    adg_status st = layout_group(b, g);
    if (st != ADG_OK) return st;
    if (tile_threads) tile_threads[gi] = best_tt;
  }
  // whole steps: the instances that fill the GPU once over either stay in the graph or are
  // stepped as separate handles (their single-handle launches with host-side schedules),
  // whichever is faster -- so a batch never runs them slower than separate handles would
  auto time_steps = [&](float* ms) -> adg_status {
    drop_graph(b);
    for (int t = 0; t <= std::max(trials, 5); ++t) {
      if (t == 1) BCUDA(b, cudaEventRecord(e0, b->stream));
      adg_status st = adg_batch_step(b, 1);
      if (st != ADG_OK) return st;
    }
    BCUDA(b, cudaEventRecord(e1, b->stream));
    BCUDA(b, cudaEventSynchronize(e1));
    BCUDA(b, cudaEventElapsedTime(ms, e0, e1));
    return ADG_OK;
  };
  for (auto& g : b->groups) {
    float ms_graph = 0.f, ms_handles = 0.f;
    g.handle_waves = 0;
    adg_status st = layout_group(b, g);
    if (st == ADG_OK) st = time_steps(&ms_graph);
    if (st != ADG_OK) return st;
    g.handle_waves = 1;
    st = layout_group(b, g);
    if (st != ADG_OK) return st;
    if (g.handles.empty()) {
      g.handle_waves = 0;
    } else {
      st = time_steps(&ms_handles);
      if (st != ADG_OK) return st;
      // the graph keeps them only when it is clearly faster (timing noise would otherwise
      // flip the choice toward a slower shape about half the time)
      if (ms_graph < 0.99f * ms_handles) g.handle_waves = 0;
    }
    st = layout_group(b, g);
    if (st != ADG_OK) return st;
  }
  drop_graph(b);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the tuning launches advanced the uniform flow; states must be set again
  for (int i = 0; i < b->n; ++i) b->has_state[i] = 0;
  return ADG_OK;
}

adg_status adg_batch_get_state(adg_batch* b, int i, double* u, int64_t count, int on_device) {
  if (!b) return bfail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  if (i < 0 || i >= b->n) return bfail(b, ADG_ERR_INVALID, "instance index out of range");
  adg_status st = adg_get_state(b->inst[i], u, count, on_device);
  if (st != ADG_OK) return bfail(b, st, adg_last_error(b->inst[i]));
  return ADG_OK;
}

adg_status adg_batch_info(const adg_batch* b, int i, double* t, int64_t* step, double* dt,
                          int64_t* n_dof, int* degree) {
  if (!b) return bfail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  if (i < 0 || i >= b->n) return bfail(const_cast<adg_batch*>(b), ADG_ERR_INVALID, "instance index out of range");
  const adg_solver* s = b->inst[i];
  if (step) *step = b->inst_steps[i];
  if (dt) *dt = s->dt;
  if (t) *t = s->dt * (double)b->inst_steps[i];
  if (n_dof) *n_dof = s->ndof;
  if (degree) *degree = s->degree;
  return ADG_OK;
}

adg_status adg_batch_l2_error_vortex(adg_batch* b, int i, double t, double beta, double x0,
                                     double y0, double* err3) {
  if (!b) return bfail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  if (i < 0 || i >= b->n) return bfail(b, ADG_ERR_INVALID, "instance index out of range");
  adg_status st = adg_l2_error_vortex(b->inst[i], t, beta, x0, y0, err3);
  if (st != ADG_OK) return bfail(b, st, adg_last_error(b->inst[i]));
  return ADG_OK;
}

int adg_batch_num_groups(const adg_batch* b) { return b ? (int)b->groups.size() : -1; }

const char* adg_batch_last_error(const adg_batch* b) { return b ? b->err.c_str() : adg_last_error(nullptr); }

void adg_batch_destroy(adg_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  free_batch(b);
  delete b;
}

}  // extern "C"
