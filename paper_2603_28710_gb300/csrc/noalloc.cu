// adg_rhs_noalloc: the FP64 DG operator without any device allocation (see include/adg.h).
//
// The operator's scratch (operator tables, face traces, face fluxes) lives in one
// file-scope device array.  Host code cannot use the array's name as a device address
// (in host code it names a host-side shadow), so each device's address is fetched once
// with cudaGetSymbolAddress while that device is current, and that address is what the
// kernels receive.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "../../include/adg.h"
#include "adg_internal.h"

namespace adg {
// defined in host.cu
void noalloc_build_tables(int N, const double* h, OpTables* T);
void noalloc_set_error(const char* msg);
}

namespace {

constexpr size_t kScratchBytes = (size_t)ADG_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {nullptr};

adg_status noalloc_fail(adg_status st, const std::string& m) {
  adg::noalloc_set_error(m.c_str());
  return st;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// The operator tables travel as a kernel argument (kernel arguments may hold up to 32 KB;
// the tables take about 9 KB) and a one-block kernel stores them into the scratch array:
// the launch copies the argument when it is enqueued, so no host memory is read after the
// call returns and no host-to-device copy waits for the stream.
struct TableBlob {
  unsigned long long v[sizeof(adg::OpTables) / 8];
};
static_assert(sizeof(adg::OpTables) % 8 == 0, "tables are a whole number of 8-byte words");
static_assert(sizeof(TableBlob) <= 30 * 1024, "tables must fit in a kernel argument");

__global__ void store_tables_kernel(const TableBlob T, unsigned long long* dst) {
  for (int i = threadIdx.x; i < (int)(sizeof(TableBlob) / 8); i += blockDim.x) dst[i] = T.v[i];
}

}  // namespace

extern "C" adg_status adg_rhs_noalloc(const adg_mesh* mesh, int degree, double gamma,
                                      const double* u, double* k, int64_t count,
                                      void* cuda_stream) {
  using namespace adg;
  if (!mesh || !u || !k) return noalloc_fail(ADG_ERR_INVALID, "mesh, u or k is NULL");
  const int dim = mesh->dim;
  if (dim != 2 && dim != 3) return noalloc_fail(ADG_ERR_INVALID, "dim must be 2 or 3");
  if (degree < 1 || degree > (dim == 2 ? 7 : 5))
    return noalloc_fail(ADG_ERR_INVALID, "degree must be 1..7 (2D) or 1..5 (3D)");
  if (!(gamma > 1.0)) return noalloc_fail(ADG_ERR_INVALID, "gamma must exceed 1");
  const int N = degree + 1, NV = dim + 2;
  const int ND = dim == 3 ? N * N * N : N * N, NF = ND / N;
  int64_t ne = 1;
  double h[3] = {1.0, 1.0, 1.0};
  for (int d = 0; d < dim; ++d) {
    if (mesh->n_elem[d] < 1) return noalloc_fail(ADG_ERR_INVALID, "n_elem must be >= 1");
    if (!(mesh->hi[d] > mesh->lo[d])) return noalloc_fail(ADG_ERR_INVALID, "hi must exceed lo");
    ne *= mesh->n_elem[d];
    h[d] = (mesh->hi[d] - mesh->lo[d]) / mesh->n_elem[d];
  }
  if (count != (int64_t)NV * ne * ND) return noalloc_fail(ADG_ERR_INVALID, "count does not match the mesh");
  // scratch layout: tables | traces [d][side][v][e][j] | fluxes [d][v][e][j]
  const size_t tab_bytes = align256(sizeof(OpTables));
  const size_t tr_bytes = align256((size_t)2 * dim * NV * ne * NF * sizeof(double));
  const size_t fl_bytes = align256((size_t)dim * NV * ne * NF * sizeof(double));
  const size_t need = tab_bytes + tr_bytes + fl_bytes;
  if (need > kScratchBytes)
    return noalloc_fail(ADG_ERR_INVALID,
                        "mesh too large for the built-in scratch: needs " + std::to_string(need) +
                            " bytes, the limit is " + std::to_string(kScratchBytes));

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(ADG_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(ADG_ERR_UNSUPPORTED, "device index too large");
  unsigned char* base = nullptr;
  {
    // one-time set-up per device, with that device current
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess)
        return noalloc_fail(ADG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_dev[dev] = p;
    }
    base = static_cast<unsigned char*>(g_scratch_dev[dev]);
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;

  OpTables tab;
  std::memset(&tab, 0, sizeof(tab));
  noalloc_build_tables(N, h, &tab);
  OpTables* tab_dev = reinterpret_cast<OpTables*>(base);
  void* tr = base + tab_bytes;
  void* fl = base + tab_bytes + tr_bytes;
  TableBlob blob;
  std::memcpy(blob.v, &tab, sizeof(OpTables));
  store_tables_kernel<<<1, 128, 0, s>>>(blob, reinterpret_cast<unsigned long long*>(tab_dev));
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(ADG_ERR_CUDA, std::string("table store: ") + cudaGetErrorString(e));

  MeshArgs m;
  std::memset(&m, 0, sizeof(m));
  m.n[0] = mesh->n_elem[0];
  m.n[1] = mesh->n_elem[1];
  m.n[2] = dim == 3 ? mesh->n_elem[2] : 1;
  m.ne = ne;
  mesh_finish(m);

  TraceArgs ta;
  std::memset(&ta, 0, sizeof(ta));
  ta.m = m;
  ta.tab = tab_dev;
  ta.u = u;
  ta.tr = tr;
  e = launch_trace(0, dim, N, ta, s);
  if (e != cudaSuccess) return noalloc_fail(ADG_ERR_CUDA, std::string("trace kernel: ") + cudaGetErrorString(e));

  FluxArgs fa;
  std::memset(&fa, 0, sizeof(fa));
  fa.m = m;
  fa.gamma = gamma;
  fa.gm1 = gamma - 1.0;
  fa.tr = tr;
  fa.fl = fl;
  fa.pe_mode = 0;
  e = launch_flux(0, dim, N, fa, s);
  if (e != cudaSuccess) return noalloc_fail(ADG_ERR_CUDA, std::string("flux kernel: ") + cudaGetErrorString(e));

  VolArgs va;
  std::memset(&va, 0, sizeof(va));
  va.m = m;
  va.tab = tab_dev;
  va.gamma = gamma;
  va.gm1 = gamma - 1.0;
  va.mode = kModeRHS;
  va.w_in = u;
  va.kout = k;
  va.fl = fl;
  va.tr = tr;
  va.write_traces = 0;
  e = launch_vol(0, dim, N, va, s);
  if (e != cudaSuccess) return noalloc_fail(ADG_ERR_CUDA, std::string("volume kernel: ") + cudaGetErrorString(e));
  return ADG_OK;
}
