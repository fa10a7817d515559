// Host side of the ADG library: the C ABI of include/adg.h, the FP64 operator tables, the
// delay schedules and the per-stage launch sequence.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/adg.h"
#include "adg_internal.h"
#include "solver_internal.h"

using namespace adg;

namespace {
constexpr size_t kMlpParamCount = 4545;  // parameters of the learned predictor (mlp.cuh)
}

namespace adg {
// (hi, lo) FP32 pair of a value: hi = RN(v), lo = RN(v - hi)
float2 split2(long double v) {
  float hi = (float)v;
  float lo = (float)(v - (long double)hi);
  return make_float2(hi, lo);
}
}  // namespace adg

namespace {

thread_local std::string g_err;

adg_status fail(adg_solver* s, adg_status st, const std::string& msg) {
  if (s) s->err = msg;
  else g_err = msg;
  return st;
}

adg_status cuda_fail(adg_solver* s, cudaError_t e, const char* what) {
  return fail(s, e == cudaErrorMemoryAllocation ? ADG_ERR_OOM : ADG_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define ADG_CUDA(S, call)                                    \
  do {                                                       \
    cudaError_t e__ = (call);                                \
    if (e__ != cudaSuccess) return cuda_fail((S), e__, #call); \
  } while (0)

// ---- basis (Gauss-Legendre, Lagrange, barycentric derivative) -----------------------

// Legendre P_n and P_n' by the three-term recurrence and P_k' = k P_{k-1} + x P_{k-1}'.
void legendre_ld(int n, long double x, long double* p, long double* dp) {
  long double pm1 = 1.0L, dpm1 = 0.0L, pk = x, dpk = 1.0L;
  if (n == 0) { *p = 1.0L; *dp = 0.0L; return; }
  for (int k = 2; k <= n; ++k) {
    long double pn = ((2 * k - 1) * x * pk - (k - 1) * pm1) / k;
    long double dpn = k * pk + x * dpk;
    pm1 = pk; dpm1 = dpk;
    pk = pn; dpk = dpn;
  }
  (void)dpm1;
  *p = pk;
  *dp = dpk;
}

void gauss_legendre(int n, double* xo, double* wo) {
  const long double pi = 3.141592653589793238462643383279502884L;
  long double xs[16], ws[16];
  for (int i = 1; i <= n; ++i) {
    // Tricomi's asymptotic first guess of the i-th largest root
    long double th = pi * (4.0L * i - 1.0L) / (4.0L * n + 2.0L);
    long double z = (1.0L - 1.0L / (8.0L * n * n) + 1.0L / (8.0L * n * n * n)) * cosl(th);
    long double p, dp;
    for (int it = 0; it < 60; ++it) {
      legendre_ld(n, z, &p, &dp);
      long double dz = p / dp;
      z -= dz;
      if (fabsl(dz) < 1e-19L) break;
    }
    legendre_ld(n, z, &p, &dp);
    xs[n - i] = z;
    ws[n - i] = 2.0L / ((1.0L - z * z) * dp * dp);
  }
  for (int i = 0; i < n; ++i) {
    xo[i] = (double)xs[i];
    wo[i] = (double)ws[i];
  }
}

void bary_weights(int n, const long double* x, long double* lam) {
  for (int j = 0; j < n; ++j) {
    long double p = 1.0L;
    for (int k = 0; k < n; ++k)
      if (k != j) p *= (x[j] - x[k]);
    lam[j] = 1.0L / p;
  }
}

// l_j(y) for all j by the second barycentric formula
void lagrange_at(int n, const long double* x, const long double* lam, long double y,
                 long double* out) {
  for (int j = 0; j < n; ++j)
    if (y == x[j]) {
      for (int k = 0; k < n; ++k) out[k] = (k == j) ? 1.0L : 0.0L;
      return;
    }
  long double den = 0.0L;
  for (int j = 0; j < n; ++j) den += lam[j] / (y - x[j]);
  for (int j = 0; j < n; ++j) out[j] = (lam[j] / (y - x[j])) / den;
}

void build_tables(adg_solver* s) {
  const int N = s->N;
  OpTables& T = s->tab;
  std::memset(&T, 0, sizeof(T));
  double xd[16], wd[16];
  gauss_legendre(N, xd, wd);
  long double x[16], lam[16];
  for (int i = 0; i < N; ++i) {
    x[i] = xd[i];
    T.xi[i] = xd[i];
    T.wq[i] = wd[i];
  }
  bary_weights(N, x, lam);
  // differentiation matrix Dm[a][i] = l_i'(x_a)
  long double Dm[16][16];
  for (int a = 0; a < N; ++a) {
    long double diag = 0.0L;
    for (int i = 0; i < N; ++i) {
      if (i == a) continue;
      Dm[a][i] = (lam[i] / lam[a]) / (x[a] - x[i]);
      diag -= Dm[a][i];
    }
    Dm[a][a] = diag;
  }
  long double lp[16], lm[16];
  lagrange_at(N, x, lam, 1.0L, lp);
  lagrange_at(N, x, lam, -1.0L, lm);
  for (int d = 0; d < 3; ++d) {
    long double sc = 2.0L / (long double)s->h[d];
    for (int i = 0; i < N; ++i) {
      for (int a = 0; a < N; ++a) {
        long double q = sc * (long double)wd[a] * Dm[a][i] / (long double)wd[i];
        T.Q[d][i * N + a] = (double)q;
        T.Qf[d][i * N + a] = split2(q);
      }
      // lift coefficients (2/h) l_i(+-1) / omega_i, halved: the face-flux kernel stores
      // twice the numerical flux
      long double vp = 0.5L * sc * lp[i] / (long double)wd[i];
      long double vm = 0.5L * sc * lm[i] / (long double)wd[i];
      T.Lp[d][i] = (double)vp;
      T.Lm[d][i] = (double)vm;
      T.Lpf[d][i] = split2(vp);
      T.Lmf[d][i] = split2(vm);
    }
  }
  for (int a = 0; a < N; ++a) {
    T.Tp[a] = (double)lp[a];
    T.Tm[a] = (double)lm[a];
    T.Tpf[a] = split2(lp[a]);
    T.Tmf[a] = split2(lm[a]);
  }
  double xe[16], we[16];
  gauss_legendre(N + 1, xe, we);
  for (int p = 0; p < N + 1; ++p) {
    T.xe[p] = xe[p];
    T.we[p] = we[p];
    long double l[16];
    lagrange_at(N, x, lam, (long double)xe[p], l);
    for (int a = 0; a < N; ++a) T.Le[p * N + a] = (double)l[a];
  }
}

// ---- AT weights: Lagrange extrapolation to the stage time from levels -(km + l) ------
void at_weights_ld(int np, long double km, long double* c) {
  for (int l = 0; l <= np; ++l) {
    long double v = 1.0L;
    for (int j = 0; j <= np; ++j)
      if (j != l) v *= (km + j) / (long double)(j - l);
    c[l] = v;
  }
}

void at_weights(int np, double km, double* c) {
  long double t[kMaxN];
  at_weights_ld(np, km, t);
  for (int l = 0; l <= np; ++l) c[l] = (double)t[l];
}

// ---- Runge-Kutta coefficients ---------------------------------------------------------
int rk_coeffs(adg_rk scheme, double* a, double* b, double* c) {
  int s = 0;
  bool two_n = false;
  if (scheme == ADG_RK_2R_22) {
    s = 2;
    a[0] = 1.0; a[1] = 0.0;
    b[0] = 0.5; b[1] = 0.5;
  } else if (scheme == ADG_RK_2R_33) {
    s = 3;
    a[0] = 0.755726352; a[1] = 0.386954477; a[2] = 0.0;
    b[0] = 0.245170287; b[1] = 0.184896052; b[2] = 0.569933661;
  } else if (scheme == ADG_RK_2N_CK45) {
    s = 5;
    two_n = true;
    const double A[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                         -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
    const double B[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                         1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                         2277821191437.0 / 14882151754819.0};
    for (int i = 0; i < 5; ++i) { a[i] = A[i]; b[i] = B[i]; }
  } else {
    return 0;
  }
  // Stage abscissae: run the scheme on y' = 1 from y = 0 with dt = 1; the input of
  // stage m then equals c_m.
  long double y = 0.0L, q = 0.0L, r = 0.0L;
  for (int m = 0; m < s; ++m) {
    c[m] = (double)(two_n ? y : r);
    if (two_n) {
      q = (long double)a[m] * q + 1.0L;
      y += (long double)b[m] * q;
    } else {
      long double y0 = y;
      r = y0 + (long double)a[m];
      y = y0 + (long double)b[m];
    }
  }
  return s;
}

uint64_t splitmix64_host(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int num_interfaces(int dim, const int* P) {
  int nsub = 1, dirs = 0;
  for (int d = 0; d < dim; ++d) {
    nsub *= P[d];
    if (P[d] > 1) ++dirs;
  }
  return nsub * dirs;
}

// Schedule of one step n: communication flag and delay counter in closed form.
void caa_step(adg_flux flux, int L, int np, int64_t n, int* comm, int* k) {
  if (flux == ADG_FLUX_SYNC) {
    *comm = 1;
    *k = 0;
  } else if (flux == ADG_FLUX_STD_DELAYED) {
    *k = (int)(n % L);
    *comm = (*k == 0);
  } else {
    const int64_t cyc = (int64_t)L + np + 1;
    const int ph = (int)(n % cyc);
    *comm = ph < np + 1;
    *k = *comm ? 0 : ph - np;
  }
}

int random_delay(adg_flux flux, int np, uint64_t seed, int dmax, int64_t n, int nif, int f) {
  if (flux == ADG_FLUX_SYNC) return 0;
  int kt = (int)(splitmix64_host(seed ^ ((uint64_t)n * (uint64_t)nif + (uint64_t)f)) %
                 (uint64_t)(dmax + 1));
  int64_t need = (flux == ADG_FLUX_STD_DELAYED) ? kt : (int64_t)kt + np;
  return (n - need < 0) ? 0 : kt;
}

adg_status schedule_impl(adg_flux flux, adg_delay_mode mode, int L, int np, int dim,
                         const int* P, uint64_t seed, int dmax, int64_t n0, int n, int32_t* comm,
                         int32_t* k, int32_t* iface_delay) {
  const int nif = num_interfaces(dim, P);
  for (int i = 0; i < n; ++i) {
    const int64_t step = n0 + i;
    if (mode == ADG_DELAY_RANDOM) {
      int kmax = 0;
      for (int f = 0; f < nif; ++f) {
        int kt = random_delay(flux, np, seed, dmax, step, nif, f);
        if (iface_delay) iface_delay[(int64_t)i * nif + f] = kt;
        kmax = kt > kmax ? kt : kmax;
      }
      if (comm) comm[i] = kmax == 0;
      if (k) k[i] = kmax;
    } else {
      int c, kk;
      caa_step(flux, L, np, step, &c, &kk);
      if (comm) comm[i] = c;
      if (k) k[i] = kk;
      if (iface_delay)
        for (int f = 0; f < nif; ++f) iface_delay[(int64_t)i * nif + f] = kk;
    }
  }
  return ADG_OK;
}

bool valid_degree(int dim, int degree) {
  return degree >= 1 && (dim == 2 ? degree <= 7 : degree <= 5);
}

size_t prec_bytes(int prec) { return storage_bytes(prec); }

// cuTensorMapEncodeTiled from the driver, through the runtime's entry-point query (no link
// against the driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;  // handles may be created from several host threads
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// Tensor map of one state-shaped array (elem_bytes per value, layout [var][elem][node]) seen
// as [var][z][y][x * nodes], with boxes of one element tile.  false when the layout breaks
// a TMA rule (row strides and the box row must be whole 16-byte units, box extents <= 256).
bool encode_state_map(adg_solver* s, CUtensorMap* map, void* base, int elem_bytes) {
  EncodeTiledFn fn = encode_tiled_fn();
  if (!fn || !base) return false;
  const int D = s->dim;
  const uint64_t rowlen = (uint64_t)s->ND * s->margs.n[0];
  if ((rowlen * elem_bytes) % 16 != 0) return false;
  if (((uint64_t)s->tile[0] * s->ND * elem_bytes) % 16 != 0) return false;
  if ((uint64_t)s->tile[0] * s->ND > 256 || s->NV > 256 || s->tile[1] > 256 || s->tile[2] > 256)
    return false;
  cuuint64_t gdim[4], gstride[3];
  cuuint32_t box[4], estr[4] = {1, 1, 1, 1};
  gdim[0] = rowlen;
  gdim[1] = (cuuint64_t)s->margs.n[1];
  box[0] = (cuuint32_t)(s->tile[0] * s->ND);
  box[1] = (cuuint32_t)s->tile[1];
  gstride[0] = rowlen * elem_bytes;
  if (D == 3) {
    gdim[2] = (cuuint64_t)s->margs.n[2];
    gdim[3] = (cuuint64_t)s->NV;
    box[2] = (cuuint32_t)s->tile[2];
    box[3] = (cuuint32_t)s->NV;
    gstride[1] = gstride[0] * s->margs.n[1];
    gstride[2] = gstride[1] * s->margs.n[2];
  } else {
    gdim[2] = (cuuint64_t)s->NV;
    box[2] = (cuuint32_t)s->NV;
    gstride[1] = gstride[0] * s->margs.n[1];
  }
  const CUresult r = fn(map, elem_bytes == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                        (cuuint32_t)(D + 1), base, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Folds the recorded event pairs into the per-kind totals and empties the pool (waits
// for the solver's stream).
cudaError_t prof_fold(adg_solver* s) {
  cudaError_t err = cudaStreamSynchronize(s->stream);
  if (err != cudaSuccess) return err;
  for (size_t i = 0; i + 1 < s->ev_used; i += 2) {
    float t = 0.f;
    err = cudaEventElapsedTime(&t, s->ev_pool[i], s->ev_pool[i + 1]);
    if (err != cudaSuccess) return err;
    const int kind = s->ev_kind[i / 2];
    s->prof_ms[kind] += t;
    s->prof_n[kind] += 1;
  }
  s->ev_used = 0;
  return cudaSuccess;
}

// Event pair around one launch (profiling only).  The pool holds at most kMaxProfEvents
// events: when it is full the recorded pairs are folded into running totals (one wait
// for the stream), so a long profiled run keeps a bounded number of CUDA events.
constexpr size_t kMaxProfEvents = 2048;
cudaError_t prof_begin(adg_solver* s, int kind) {
  if (!s->profiling) return cudaSuccess;
  if (s->ev_used + 2 > kMaxProfEvents) {
    cudaError_t err = prof_fold(s);
    if (err != cudaSuccess) return err;
  }
  if (s->ev_used + 2 > s->ev_pool.size()) {
    for (int i = 0; i < 64; ++i) {
      cudaEvent_t e;
      cudaError_t err = cudaEventCreate(&e);
      if (err != cudaSuccess) return err;
      s->ev_pool.push_back(e);
    }
  }
  if (s->ev_kind.size() < s->ev_pool.size() / 2) s->ev_kind.resize(s->ev_pool.size() / 2);
  s->ev_kind[s->ev_used / 2] = kind;
  return cudaEventRecord(s->ev_pool[s->ev_used], s->stream);
}

cudaError_t prof_end(adg_solver* s) {
  if (!s->profiling) return cudaSuccess;
  cudaError_t err = cudaEventRecord(s->ev_pool[s->ev_used + 1], s->stream);
  s->ev_used += 2;
  return err;
}

void free_all(adg_solver* s) {
  for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
  s->ev_pool.clear();
  void* ptrs[] = {s->w, s->x, s->tr, s->fl, s->ring, s->pe_slot, s->pe_iface, s->tab_dev,
                  s->red_partial, s->red_out, s->flag, s->tmp_u, s->tmp_k, s->pe_face_d,
                  s->pe_face_e, s->mlp, s->lw_E, s->lw_s, s->lw_x, s->lw_y, s->tr_alt,
                  s->kerr};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
}

adg_status launch_traces_of(adg_solver* s, const double* u) {
  TraceArgs ta{};
  ta.m = s->margs;
  ta.tab = s->tab_dev;
  ta.u = u;
  ta.tr = s->tr;
  ADG_CUDA(s, launch_trace(s->prec, s->dim, s->N, ta, s->stream));
  return ADG_OK;
}

FluxArgs base_flux_args(adg_solver* s) {
  FluxArgs fa;
  std::memset(&fa, 0, sizeof(fa));
  fa.m = s->margs;
  fa.gamma = s->opt.gamma;
  fa.gammaf = split2(s->opt.gamma);
  fa.gm1 = s->opt.gamma - 1.0;
  fa.gm1f = split2(s->opt.gamma - 1.0);
  fa.tr = s->tr;
  fa.fl = s->fl;
  fa.flux_kind = (int)s->flux;
  fa.pe_slot = s->pe_slot;
  fa.pe_iface = s->pe_iface;
  fa.npe = s->npe;
  fa.ring = s->ring;
  fa.depth = s->depth;
  fa.seed = s->opt.seed;
  fa.n_iface = s->n_iface;
  fa.dmax = s->opt.random_delay_max;
  fa.np = s->np;
  fa.nterms = (s->flux == ADG_FLUX_STD_DELAYED) ? 1 : s->np + 1;
  return fa;
}

adg_status upload_dt_tables(adg_solver* s);

adg_status after_state_set(adg_solver* s) {
  s->has_state = true;
  s->step = 0;
  s->t = 0.0;
  s->head = -1;
  if (s->opt.dt > 0) {
    s->dt = s->opt.dt;
  } else {
    ADG_CUDA(s, launch_max_speed(s->dim, s->N, s->margs, s->opt.gamma, s->w, s->red_partial,
                                 s->red_out, s->red_blocks, s->stream));
    double smax = 0;
    ADG_CUDA(s, cudaMemcpyAsync(&smax, s->red_out, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    ADG_CUDA(s, cudaStreamSynchronize(s->stream));
    if (!(smax > 0) || !std::isfinite(smax))
      return fail(s, ADG_ERR_NONFINITE, "state has no finite positive signal speed");
    double hmin = s->h[0];
    for (int d = 1; d < s->dim; ++d) hmin = s->h[d] < hmin ? s->h[d] : hmin;
    double dt = s->opt.cfl * hmin / ((2.0 * s->degree + 1.0) * smax);
    if (s->opt.t_end > 0) dt = s->opt.t_end / std::ceil(s->opt.t_end / dt);
    s->dt = dt;
  }
  adg_status st = upload_dt_tables(s);
  if (st != ADG_OK) return st;
  st = launch_traces_of(s, s->w);
  if (st != ADG_OK) return st;
  s->traces_valid = true;
  s->traces_partial = false;
  if (s->kerr) ADG_CUDA(s, cudaMemsetAsync(s->kerr, 0, sizeof(int), s->stream));
  return ADG_OK;
}

// dt-scaled operator tables for the 2N update, uploaded with the others
adg_status upload_dt_tables(adg_solver* s) {
  for (int d = 0; d < 3; ++d) {
    for (int i = 0; i < s->N * s->N; ++i) {
      s->tab.Qs[d][i] = s->tab.Q[d][i] * s->dt;
      s->tab.Qsf[d][i] = split2((long double)s->tab.Q[d][i] * s->dt);
    }
    for (int i = 0; i < s->N; ++i) {
      s->tab.Lps[d][i] = s->tab.Lp[d][i] * s->dt;
      s->tab.Lms[d][i] = s->tab.Lm[d][i] * s->dt;
      s->tab.Lpsf[d][i] = split2((long double)s->tab.Lp[d][i] * s->dt);
      s->tab.Lmsf[d][i] = split2((long double)s->tab.Lm[d][i] * s->dt);
    }
  }
  ADG_CUDA(s, cudaMemcpyAsync(s->tab_dev, &s->tab, sizeof(OpTables), cudaMemcpyHostToDevice, s->stream));
  return ADG_OK;
}

// Checkpoint layout: this header, then the solution (FP64), the traces and the ring
// (operator storage type).
struct CkptHeader {
  char magic[8];
  int32_t version, dim, degree, prec, flux, rk, delay_mode, max_delay, np, depth, rdmax;
  int32_t P[3], n_elem[3], head;
  int64_t ndof, n_tr, n_ring, step;
  uint64_t seed;
  double t, dt, lo[3], hi[3], gamma;
};
constexpr char kCkptMagic[8] = {'A', 'D', 'G', 'C', 'K', 'P', 'T', '1'};

int64_t ckpt_tr_values(const adg_solver* s) { return (int64_t)2 * s->dim * s->NV * s->ne * s->NF; }
int64_t ckpt_ring_values(const adg_solver* s) {
  if (!s->ring) return 0;
  return (int64_t)s->depth * (s->flux >= ADG_FLUX_AT_TRACE ? 2 : 1) * s->NV * s->npe * s->NF;
}

CkptHeader ckpt_header(const adg_solver* s) {
  CkptHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, kCkptMagic, 8);
  h.version = 1;
  h.dim = s->dim;
  h.degree = s->degree;
  h.prec = s->prec;
  h.flux = (int32_t)s->flux;
  h.rk = (int32_t)s->opt.rk;
  h.delay_mode = (int32_t)s->opt.delay_mode;
  h.max_delay = s->max_delay;
  h.np = s->np;
  h.depth = s->depth;
  h.rdmax = s->opt.random_delay_max;
  for (int d = 0; d < 3; ++d) {
    h.P[d] = s->P[d];
    h.n_elem[d] = s->mesh.n_elem[d];
    h.lo[d] = s->mesh.lo[d];
    h.hi[d] = s->mesh.hi[d];
  }
  h.head = s->head;
  h.ndof = s->ndof;
  h.n_tr = ckpt_tr_values(s);
  h.n_ring = ckpt_ring_values(s);
  h.step = s->step;
  h.seed = s->opt.seed;
  h.t = s->t;
  h.dt = s->dt;
  h.gamma = s->opt.gamma;
  return h;
}

int64_t ckpt_bytes(const adg_solver* s) {
  const int64_t sb = (int64_t)prec_bytes(s->prec);
  return (int64_t)sizeof(CkptHeader) + s->ndof * 8 + (ckpt_tr_values(s) + ckpt_ring_values(s)) * sb;
}

}  // namespace

namespace adg {
FluxArgs stage_flux_args(const adg_solver* s, int m) {
  FluxArgs fa = base_flux_args(const_cast<adg_solver*>(s));
  const bool pe = s->flux != ADG_FLUX_SYNC && s->npe > 0;
  const bool random = s->opt.delay_mode == ADG_DELAY_RANDOM;
  fa.pe_mode = pe ? 1 : 0;
  fa.random = random ? 1 : 0;
  if (pe) {
    const int kmax = random ? s->opt.random_delay_max : s->max_delay;
    for (int kt = 0; kt <= kmax && kt < kMaxCoefDelay; ++kt) {
      if (s->flux == ADG_FLUX_STD_DELAYED) {
        fa.ctab[kt][0] = 1.0;
        fa.ctabf[kt][0] = make_float2(1.0f, 0.0f);
      } else {
        long double c[kMaxN];
        at_weights_ld(s->np, (long double)kt + s->rkc[m], c);
        for (int l = 0; l <= s->np; ++l) {
          fa.ctab[kt][l] = (double)c[l];
          fa.ctabf[kt][l] = split2(c[l]);
        }
      }
    }
  }
  return fa;
}

VolArgs stage_vol_args(const adg_solver* s, int m) {
  VolArgs va;
  std::memset(&va, 0, sizeof(va));
  va.m = s->margs;
  va.tab = s->tab_dev;
  va.gamma = s->opt.gamma;
  va.gammaf = split2(s->opt.gamma);
  va.gm1 = s->opt.gamma - 1.0;
  va.gm1f = split2(s->opt.gamma - 1.0);
  va.mode = s->rk2n ? kMode2N : kMode2R;
  va.stage = m;
  va.last = (m == s->stages - 1);
  va.dt = s->dt;
  if (s->rk2n) {
    va.ca = s->rka[m];
    va.cb = s->rkb[m];
  } else {
    va.ca = s->dt * s->rka[m];
    va.cb = s->dt * s->rkb[m];
  }
  va.caf = split2(va.ca);
  va.cbf = split2(va.cb);
  va.dtf = split2(va.dt);
  va.w_in = s->w;
  va.r_in = s->x;
  va.w = s->w;
  va.x = s->x;
  va.fl = s->fl;
  va.tr = s->tr;
  va.write_traces = 1;
  va.scaled = s->rk2n ? 1 : 0;
  va.bulk = (s->ne * s->ND) % 4 == 0 ? 1 : 0;
  return va;
}

// Helpers for adg_rhs_noalloc (noalloc.cu): the same operator tables without a handle,
// and the per-thread error text that adg_last_error(NULL) returns.
void noalloc_build_tables(int N, const double* h, OpTables* T) {
  adg_solver tmp;
  tmp.N = N;
  for (int d = 0; d < 3; ++d) tmp.h[d] = h[d];
  build_tables(&tmp);
  *T = tmp.tab;
}
void noalloc_set_error(const char* msg) { g_err = msg; }
}  // namespace adg

extern "C" {

adg_status adg_default_options(adg_options* opt) {
  if (!opt) return fail(nullptr, ADG_ERR_INVALID, "opt is NULL");
  std::memset(opt, 0, sizeof(*opt));
  opt->rk = ADG_RK_2N_CK45;
  opt->dt = 0.0;
  opt->cfl = 0.1;
  opt->t_end = 0.0;
  opt->gamma = 1.4;
  opt->delay_mode = ADG_DELAY_CAA;
  opt->seed = 0;
  opt->random_delay_max = 0;
  opt->at_np = 0;
  opt->precision = ADG_PREC_FP64;
  opt->cuda_stream = nullptr;
  return ADG_OK;
}

adg_status adg_create(const adg_mesh* mesh, int degree, const int P[3], int max_delay,
                      adg_flux flux, const adg_options* opt, adg_solver** out) {
  if (!out) return fail(nullptr, ADG_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!mesh || !P) return fail(nullptr, ADG_ERR_INVALID, "mesh or P is NULL");
  if (mesh->dim != 2 && mesh->dim != 3) return fail(nullptr, ADG_ERR_INVALID, "dim must be 2 or 3");
  if (degree < 1 || degree > 7) return fail(nullptr, ADG_ERR_INVALID, "degree must be in 1..7");
  if (!valid_degree(mesh->dim, degree))
    return fail(nullptr, ADG_ERR_UNSUPPORTED, "3D is built for degree 1..5");
  if ((int)flux < 0 || (int)flux > 4) return fail(nullptr, ADG_ERR_INVALID, "unknown flux");
  adg_options o;
  if (opt) o = *opt;
  else adg_default_options(&o);
  if ((int)o.rk < 0 || (int)o.rk > 2) return fail(nullptr, ADG_ERR_INVALID, "unknown rk scheme");
  if ((int)o.precision < 0 || (int)o.precision > 2)
    return fail(nullptr, ADG_ERR_INVALID, "unknown precision");
  if ((int)o.kernel_path < 0 || (int)o.kernel_path > 3)
    return fail(nullptr, ADG_ERR_INVALID, "unknown kernel path");
  if (!(o.gamma > 1.0)) return fail(nullptr, ADG_ERR_INVALID, "gamma must exceed 1");
  if (o.dt <= 0 && !(o.cfl > 0)) return fail(nullptr, ADG_ERR_INVALID, "need dt > 0 or cfl > 0");
  if (o.delay_mode != ADG_DELAY_CAA && o.delay_mode != ADG_DELAY_RANDOM)
    return fail(nullptr, ADG_ERR_INVALID, "unknown delay mode");
  if (o.delay_mode == ADG_DELAY_RANDOM && (o.random_delay_max < 0 || o.random_delay_max > 15))
    return fail(nullptr, ADG_ERR_INVALID, "random_delay_max must be in 0..15");
  const int np = o.at_np > 0 ? o.at_np : degree;
  if (np > 7) return fail(nullptr, ADG_ERR_INVALID, "at_np must be <= 7");
  if (flux == ADG_FLUX_LEARNED && np != 2)
    return fail(nullptr, ADG_ERR_INVALID, "the learned flux needs at_np = 2 (three stored levels)");
  if (flux != ADG_FLUX_SYNC && o.delay_mode == ADG_DELAY_CAA) {
    int lmin = (flux == ADG_FLUX_STD_DELAYED) ? 1 : 0;
    if (max_delay < lmin || max_delay > 15)
      return fail(nullptr, ADG_ERR_INVALID, "max_delay out of range (1..15 standard, 0..15 AT)");
  }
  int64_t ne = 1;
  for (int d = 0; d < mesh->dim; ++d) {
    if (mesh->n_elem[d] < 1 || mesh->n_elem[d] > (1 << 20))
      return fail(nullptr, ADG_ERR_INVALID, "n_elem must be in 1..2^20");
    if (P[d] < 1 || mesh->n_elem[d] % P[d] != 0)
      return fail(nullptr, ADG_ERR_INVALID, "P[d] must divide n_elem[d]");
    if (!(mesh->hi[d] > mesh->lo[d])) return fail(nullptr, ADG_ERR_INVALID, "hi must exceed lo");
    ne *= mesh->n_elem[d];
  }
  {
    const int64_t nd = mesh->dim == 3 ? (int64_t)(degree + 1) * (degree + 1) * (degree + 1)
                                      : (int64_t)(degree + 1) * (degree + 1);
    if ((int64_t)(mesh->dim + 2) * ne * nd >= ((int64_t)1 << 31))
      return fail(nullptr, ADG_ERR_UNSUPPORTED, "meshes with 2^31 or more degrees of freedom are not supported");
  }
  if (!kernels_available((int)o.precision, mesh->dim, degree + 1))
    return fail(nullptr, ADG_ERR_UNSUPPORTED, "no kernels built for this precision/degree");

  adg_solver* s = new (std::nothrow) adg_solver();
  if (!s) return fail(nullptr, ADG_ERR_OOM, "host allocation failed");
  s->mesh = *mesh;
  s->dim = mesh->dim;
  s->degree = degree;
  s->N = degree + 1;
  s->NV = s->dim + 2;
  s->ND = s->dim == 3 ? s->N * s->N * s->N : s->N * s->N;
  s->NF = s->ND / s->N;
  s->ne = ne;
  s->ndof = (int64_t)s->NV * ne * s->ND;
  for (int d = 0; d < 3; ++d) s->P[d] = d < s->dim ? P[d] : 1;
  s->max_delay = max_delay;
  s->flux = flux;
  s->opt = o;
  s->np = np;
  s->prec = (int)o.precision;
  s->stages = rk_coeffs(o.rk, s->rka, s->rkb, s->rkc);
  s->rk2n = (o.rk == ADG_RK_2N_CK45);
  s->J = 1.0;
  for (int d = 0; d < 3; ++d) {
    s->h[d] = d < s->dim ? (mesh->hi[d] - mesh->lo[d]) / mesh->n_elem[d] : 1.0;
    if (d < s->dim) s->J *= s->h[d] / 2.0;
  }
  s->margs.n[0] = mesh->n_elem[0];
  s->margs.n[1] = mesh->n_elem[1];
  s->margs.n[2] = s->dim == 3 ? mesh->n_elem[2] : 1;
  s->margs.ne = ne;
  mesh_finish(s->margs);
  build_tables(s);
  // fused per-stage kernel on request (measured on GB300, the split path is faster for
  // every arithmetic: the fused kernel's block-wide phases issue more instructions per node
  // and wait at their barriers); the learned flux keeps the split path (its network runs
  // between the two launches)
  s->fused = flux != ADG_FLUX_LEARNED && fused_tile(s->dim, s->N, s->tile) &&
             o.kernel_path == ADG_PATH_FUSED;
  // element path on request, and by default for the FP32 operator: it evaluates every
  // interior face twice, which the FP32 form (bound by memory and issue) affords and the
  // FP64 and pair forms (bound by the FP64 pipe) do not (measured on GB300: FP32 +2 to
  // +6 %, FP64 -24 %, pairs -21 % in 2D and -46 % in 3D)
  s->faces = flux != ADG_FLUX_LEARNED &&
             (o.kernel_path == ADG_PATH_ELEMENT ||
              (o.kernel_path == ADG_PATH_AUTO && o.precision == ADG_PREC_FP32));
  for (int d = 0; d < 3; ++d) {
    if (d >= s->dim) s->tile[d] = 1;
    s->ntile[d] = (s->margs.n[d] + s->tile[d] - 1) / s->tile[d];
  }

  // subdomain faces: face (d, e) joins e and its +d neighbour; it lies between two
  // subdomains iff P[d] > 1 and e is the last element of its block along d.
  s->n_iface = num_interfaces(s->dim, s->P);
  int32_t* slot_h = nullptr;
  int32_t* iface_h = nullptr;
  std::vector<int32_t> face_d_h, face_e_h;
  if (flux != ADG_FLUX_SYNC) {
    slot_h = new (std::nothrow) int32_t[(size_t)s->dim * ne];
    iface_h = new (std::nothrow) int32_t[(size_t)s->dim * ne + 1];
    if (!slot_h || !iface_h) {
      delete[] slot_h;
      delete[] iface_h;
      delete s;
      return fail(nullptr, ADG_ERR_OOM, "host allocation failed");
    }
    int nsub = s->P[0] * s->P[1] * s->P[2];
    int off = 0;
    for (int d = 0; d < s->dim; ++d) {
      const int bs = s->margs.n[d] / s->P[d];
      for (int64_t e = 0; e < ne; ++e) {
        int c[3] = {(int)(e % s->margs.n[0]), (int)((e / s->margs.n[0]) % s->margs.n[1]),
                    (int)(e / ((int64_t)s->margs.n[0] * s->margs.n[1]))};
        bool pe = s->P[d] > 1 && (c[d] + 1) % bs == 0;
        if (pe) {
          int sub = 0;
          for (int dd = s->dim - 1; dd >= 0; --dd)
            sub = sub * s->P[dd] + c[dd] / (s->margs.n[dd] / s->P[dd]);
          iface_h[s->npe] = off + sub;
          face_d_h.push_back(d);
          face_e_h.push_back((int32_t)e);
          slot_h[(int64_t)d * ne + e] = (int32_t)s->npe++;
        } else {
          slot_h[(int64_t)d * ne + e] = -1;
        }
      }
      if (s->P[d] > 1) off += nsub;
    }
    if (o.delay_mode == ADG_DELAY_RANDOM)
      s->depth = o.random_delay_max + (flux == ADG_FLUX_STD_DELAYED ? 0 : np) + 1;
    else
      s->depth = (flux == ADG_FLUX_STD_DELAYED) ? 1 : np + 1;
  }

  cudaError_t ce = cudaSuccess;
  auto alloc = [&](void** p, size_t bytes) {
    if (ce == cudaSuccess && bytes > 0) ce = cudaMalloc(p, bytes);
  };
  const size_t sb = prec_bytes(s->prec);
  const size_t nst = (size_t)s->ndof;
  const size_t ntr = (size_t)2 * s->dim * s->NV * ne * s->NF;
  const size_t nfl = (size_t)s->dim * s->NV * ne * s->NF;
  s->red_blocks = 152 * 4;
  alloc((void**)&s->w, nst * sizeof(double));
  alloc(&s->x, nst * sb);
  alloc(&s->tr, ntr * sb);
  alloc(&s->fl, nfl * sb);
  alloc((void**)&s->tab_dev, sizeof(OpTables));
  alloc((void**)&s->red_partial, (size_t)s->red_blocks * 5 * sizeof(double));
  alloc((void**)&s->red_out, 8 * sizeof(double));
  alloc((void**)&s->flag, sizeof(int));
  if (s->fused || s->faces) alloc(&s->tr_alt, ntr * sb);
  if (s->fused || s->faces) alloc((void**)&s->kerr, sizeof(int));
  if (flux != ADG_FLUX_SYNC) {
    alloc((void**)&s->pe_slot, (size_t)s->dim * ne * sizeof(int32_t));
    alloc((void**)&s->pe_iface, (size_t)(s->npe + 1) * sizeof(int32_t));
    size_t ringn = (size_t)s->depth * (flux >= ADG_FLUX_AT_TRACE ? 2 : 1) * s->NV * s->npe * s->NF;
    alloc(&s->ring, (ringn + 1) * sb);
    alloc((void**)&s->pe_face_d, (size_t)(s->npe + 1) * sizeof(int32_t));
    if (flux == ADG_FLUX_LEARNED) {
      const size_t nch = (size_t)(s->npe + 1) * s->NF * 2 * s->NV;
      alloc(&s->lw_E, nch * sb);
      alloc((void**)&s->lw_s, nch * sizeof(double));
      alloc((void**)&s->lw_x, nch * 4 * sizeof(float));
      alloc((void**)&s->lw_y, nch * sizeof(float));
    }
    alloc((void**)&s->pe_face_e, (size_t)(s->npe + 1) * sizeof(int32_t));
  }
  // NULL selects the legacy default stream (handle 0), as in the CUDA runtime itself
  s->stream = (cudaStream_t)o.cuda_stream;
  s->own_stream = false;
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(s->tab_dev, &s->tab, sizeof(OpTables), cudaMemcpyHostToDevice, s->stream);
  if (ce == cudaSuccess && flux != ADG_FLUX_SYNC) {
    // levels not yet stored read as zero (and checkpoints copy defined bytes)
    const size_t ringn = (size_t)s->depth * (flux >= ADG_FLUX_AT_TRACE ? 2 : 1) * s->NV * s->npe * s->NF;
    ce = cudaMemsetAsync(s->ring, 0, (ringn + 1) * sb, s->stream);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(s->pe_slot, slot_h, (size_t)s->dim * ne * sizeof(int32_t),
                         cudaMemcpyHostToDevice, s->stream);
    if (ce == cudaSuccess && s->npe > 0)
      ce = cudaMemcpyAsync(s->pe_iface, iface_h, (size_t)s->npe * sizeof(int32_t),
                           cudaMemcpyHostToDevice, s->stream);
    if (ce == cudaSuccess && s->npe > 0)
      ce = cudaMemcpyAsync(s->pe_face_d, face_d_h.data(), (size_t)s->npe * sizeof(int32_t),
                           cudaMemcpyHostToDevice, s->stream);
    if (ce == cudaSuccess && s->npe > 0)
      ce = cudaMemcpyAsync(s->pe_face_e, face_e_h.data(), (size_t)s->npe * sizeof(int32_t),
                           cudaMemcpyHostToDevice, s->stream);
  }
  if (ce == cudaSuccess && s->fused) {
    // defined contents everywhere (checkpoints copy whole trace buffers)
    ce = cudaMemsetAsync(s->tr, 0, ntr * sb, s->stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(s->tr_alt, 0, ntr * sb, s->stream);
    s->tma = encode_state_map(s, &s->tm_w, s->w, 8) && encode_state_map(s, &s->tm_x, s->x, (int)sb);
  }
  if (ce == cudaSuccess && s->kerr) ce = cudaMemsetAsync(s->kerr, 0, sizeof(int), s->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
  delete[] slot_h;
  delete[] iface_h;
  if (ce != cudaSuccess) {
    adg_status st = cuda_fail(nullptr, ce, "adg_create");
    free_all(s);
    delete s;
    return st;
  }
  *out = s;
  return ADG_OK;
}

adg_status adg_set_state(adg_solver* s, const double* u, int64_t count, int on_device) {
  if (!s) return fail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  if (!u) return fail(s, ADG_ERR_INVALID, "u is NULL");
  if (count != s->ndof) return fail(s, ADG_ERR_INVALID, "count does not match n_dof");
  ADG_CUDA(s, cudaMemcpyAsync(s->w, u, count * sizeof(double),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              s->stream));
  return after_state_set(s);
}

adg_status adg_init_vortex(adg_solver* s, double t, double beta, double x0, double y0) {
  if (!s) return fail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  const double Lx = s->mesh.hi[0] - s->mesh.lo[0], Ly = s->mesh.hi[1] - s->mesh.lo[1];
  ADG_CUDA(s, launch_init_vortex(s->dim, s->N, s->margs, s->mesh.lo, s->h, s->tab_dev,
                                 s->opt.gamma, t, beta, x0, y0, Lx, Ly, s->w, s->stream));
  return after_state_set(s);
}

adg_status adg_init_tgv(adg_solver* s, double mach) {
  if (!s) return fail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  if (s->dim != 3) return fail(s, ADG_ERR_INVALID, "the Taylor-Green vortex is 3D");
  if (!(mach > 0)) return fail(s, ADG_ERR_INVALID, "mach must be positive");
  ADG_CUDA(s, launch_init_tgv(s->N, s->margs, s->mesh.lo, s->h, s->tab_dev, s->opt.gamma, mach,
                              s->w, s->stream));
  return after_state_set(s);
}

adg_status adg_step(adg_solver* s, int n_steps) {
  if (!s) return fail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  if (n_steps < 0) return fail(s, ADG_ERR_INVALID, "n_steps must be >= 0");
  if (!s->has_state) return fail(s, ADG_ERR_STATE, "no state: call adg_set_state first");
  if (s->flux == ADG_FLUX_LEARNED && !s->mlp)
    return fail(s, ADG_ERR_STATE, "learned flux without a model: call adg_set_learned_model");
  if (!s->traces_valid) {
    adg_status st = launch_traces_of(s, s->w);
    if (st != ADG_OK) return st;
    s->traces_valid = true;
    s->traces_partial = false;
  }
  const bool pe = s->flux != ADG_FLUX_SYNC && s->npe > 0;
  const bool random = s->opt.delay_mode == ADG_DELAY_RANDOM;
  const bool use_fused = s->fused && !s->log;
  for (int it = 0; it < n_steps; ++it) {
    const int64_t n = s->step;
    int comm = 1, k = 0;
    if (!random) caa_step(s->flux, s->max_delay, s->np, n, &comm, &k);
    const bool store_step = pe && (random || comm);
    if (!use_fused && s->traces_partial) {
      // the split path reads the traces of every face: rebuild them from the solution (the
      // input of stage 0), the same values the fused kernel derives them from
      adg_status st = launch_traces_of(s, s->w);
      if (st != ADG_OK) return st;
      s->traces_partial = false;
    }
    for (int m = 0; m < s->stages; ++m) {
      if (s->log && s->log_count < s->log_cap && s->npe > 0) {
        const int64_t rec = (int64_t)2 * s->NV * s->npe * s->NF;
        ADG_CUDA(s, launch_log_traces(s->prec, s->dim, s->N, s->tr, s->pe_face_d, s->pe_face_e,
                                      s->margs, s->npe, s->log + s->log_count * rec, s->stream));
        s->log_count += 1;
      }
      FluxArgs fa = stage_flux_args(s, m);
      if (pe) {
        if (store_step && m == 0) {
          s->head = (s->head + 1) % s->depth;
          fa.store = 1;
        }
        fa.head = s->head < 0 ? 0 : s->head;
        fa.uniform_delay = random ? 0 : (comm ? 0 : k);
        fa.step = n;
      }
      if (s->faces) {
        // one launch: face fluxes of every element's faces from the traces in tr, volume
        // terms, update, next stage's traces into tr_alt
        FusedArgs ua;
        std::memset(&ua, 0, sizeof(ua));
        ua.v = stage_vol_args(s, m);
        ua.v.tr = s->tr_alt;
        ua.f = fa;
        ua.tr_in = s->tr;
        ua.err = s->kerr;
        ADG_CUDA(s, prof_begin(s, 1));
        ADG_CUDA(s, launch_vol_faces(s->prec, s->dim, s->N, ua, s->stream));
        ADG_CUDA(s, prof_end(s));
        void* t = s->tr;
        s->tr = s->tr_alt;
        s->tr_alt = t;
        continue;
      }
      if (use_fused) {
        FusedArgs ua;
        std::memset(&ua, 0, sizeof(ua));
        ua.v = stage_vol_args(s, m);
        ua.f = fa;
        ua.tr_in = s->tr;
        ua.tr_out = s->tr_alt;
        for (int d = 0; d < 3; ++d) ua.ntile[d] = s->ntile[d];
        ua.tma = s->tma;
        ua.err = s->kerr;
        ADG_CUDA(s, prof_begin(s, 1));
        ADG_CUDA(s, launch_fused(s->prec, s->dim, s->N, ua, s->tm_w, s->tm_x, s->stream));
        ADG_CUDA(s, prof_end(s));
        void* t = s->tr;
        s->tr = s->tr_alt;
        s->tr_alt = t;
        s->traces_partial = true;
        continue;
      }
      ADG_CUDA(s, prof_begin(s, 0));
      ADG_CUDA(s, launch_flux(s->prec, s->dim, s->N, fa, s->stream));
      ADG_CUDA(s, prof_end(s));
      if (s->flux == ADG_FLUX_LEARNED && pe && (random || !comm)) {
        LearnArgs la;
        std::memset(&la, 0, sizeof(la));
        la.m = s->margs;
        la.gamma = s->opt.gamma;
        la.gammaf = split2(s->opt.gamma);
        la.gm1 = fa.gm1;
        la.gm1f = fa.gm1f;
        la.ring = s->ring;
        la.fl = s->fl;
        la.face_d = s->pe_face_d;
        la.face_e = s->pe_face_e;
        la.pe_iface = s->pe_iface;
        la.mlp = s->mlp;
        la.trust = s->trust;
        la.npe = s->npe;
        la.depth = s->depth;
        la.head = fa.head;
        la.random = fa.random;
        la.uniform_delay = fa.uniform_delay;
        la.n_iface = s->n_iface;
        la.dmax = s->opt.random_delay_max;
        la.seed = s->opt.seed;
        la.step = n;
        std::memcpy(la.ctab, fa.ctab, sizeof(la.ctab));
        std::memcpy(la.ctabf, fa.ctabf, sizeof(la.ctabf));
        for (int kt = 0; kt < kMaxCoefDelay; ++kt) la.km[kt] = kt + s->rkc[m];
        la.E = s->lw_E;
        la.s = s->lw_s;
        la.x = s->lw_x;
        la.y = s->lw_y;
        ADG_CUDA(s, launch_learned(s->prec, s->dim, s->N, la, s->stream));
      }
      VolArgs va = stage_vol_args(s, m);
      ADG_CUDA(s, prof_begin(s, 1));
      ADG_CUDA(s, launch_vol(s->prec, s->dim, s->N, va, s->stream));
      ADG_CUDA(s, prof_end(s));
    }
    s->step += 1;
    s->t += s->dt;
  }
  return ADG_OK;
}

adg_status adg_get_state(adg_solver* s, double* u, int64_t count, int on_device) {
  if (!s) return fail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  if (!u) return fail(s, ADG_ERR_INVALID, "u is NULL");
  if (count != s->ndof) return fail(s, ADG_ERR_INVALID, "count does not match n_dof");
  ADG_CUDA(s, cudaMemcpyAsync(u, s->w, count * sizeof(double),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                              s->stream));
  ADG_CUDA(s, cudaStreamSynchronize(s->stream));
  if (s->kerr) {
    int kerr = 0;
    ADG_CUDA(s, cudaMemcpy(&kerr, s->kerr, sizeof(int), cudaMemcpyDeviceToHost));
    if (kerr)
      return fail(s, ADG_ERR_TIMEOUT,
                  "a kernel's wait for its tile copies gave up (fused or element path); the state is not valid");
  }
  return ADG_OK;
}

adg_status adg_checkpoint_bytes(const adg_solver* s, int64_t* bytes) {
  if (!s) return fail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  if (!bytes) return fail(const_cast<adg_solver*>(s), ADG_ERR_INVALID, "bytes is NULL");
  *bytes = ckpt_bytes(s);
  return ADG_OK;
}

adg_status adg_checkpoint_save(adg_solver* s, void* buf, int64_t bytes) {
  if (!s) return fail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  if (!buf) return fail(s, ADG_ERR_INVALID, "buf is NULL");
  if (bytes < ckpt_bytes(s)) return fail(s, ADG_ERR_INVALID, "buffer smaller than adg_checkpoint_bytes");
  if (!s->has_state) return fail(s, ADG_ERR_STATE, "no state to checkpoint");
  if (!s->traces_valid || s->traces_partial) {
    // traces of every face (the fused path keeps only tile-boundary ones), so that any
    // compatible handle can continue from the checkpoint
    adg_status st = launch_traces_of(s, s->w);
    if (st != ADG_OK) return st;
    s->traces_valid = true;
    s->traces_partial = false;
  }
  const CkptHeader h = ckpt_header(s);
  unsigned char* p = static_cast<unsigned char*>(buf);
  std::memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  const size_t sb = prec_bytes(s->prec);
  ADG_CUDA(s, cudaMemcpyAsync(p, s->w, (size_t)h.ndof * 8, cudaMemcpyDeviceToHost, s->stream));
  p += (size_t)h.ndof * 8;
  ADG_CUDA(s, cudaMemcpyAsync(p, s->tr, (size_t)h.n_tr * sb, cudaMemcpyDeviceToHost, s->stream));
  p += (size_t)h.n_tr * sb;
  if (h.n_ring > 0)
    ADG_CUDA(s, cudaMemcpyAsync(p, s->ring, (size_t)h.n_ring * sb, cudaMemcpyDeviceToHost, s->stream));
  ADG_CUDA(s, cudaStreamSynchronize(s->stream));
  return ADG_OK;
}

adg_status adg_checkpoint_restore(adg_solver* s, const void* buf, int64_t bytes) {
  if (!s) return fail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  if (!buf) return fail(s, ADG_ERR_INVALID, "buf is NULL");
  if (bytes < (int64_t)sizeof(CkptHeader)) return fail(s, ADG_ERR_INVALID, "checkpoint truncated");
  CkptHeader h;
  std::memcpy(&h, buf, sizeof(h));
  if (std::memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != 1)
    return fail(s, ADG_ERR_INVALID, "not an ADG checkpoint (version 1)");
  const CkptHeader m = ckpt_header(s);
  struct { const char* name; bool same; } fields[] = {
      {"dim", h.dim == m.dim}, {"degree", h.degree == m.degree}, {"precision", h.prec == m.prec},
      {"flux", h.flux == m.flux}, {"rk", h.rk == m.rk}, {"delay_mode", h.delay_mode == m.delay_mode},
      {"max_delay", h.max_delay == m.max_delay}, {"at_np", h.np == m.np},
      {"random_delay_max", h.rdmax == m.rdmax}, {"seed", h.seed == m.seed},
      {"gamma", h.gamma == m.gamma},
      {"P", h.P[0] == m.P[0] && h.P[1] == m.P[1] && h.P[2] == m.P[2]},
      {"mesh", h.n_elem[0] == m.n_elem[0] && h.n_elem[1] == m.n_elem[1] && h.n_elem[2] == m.n_elem[2] &&
                   h.lo[0] == m.lo[0] && h.lo[1] == m.lo[1] && h.lo[2] == m.lo[2] &&
                   h.hi[0] == m.hi[0] && h.hi[1] == m.hi[1] && h.hi[2] == m.hi[2]},
      {"sizes", h.ndof == m.ndof && h.n_tr == m.n_tr && h.n_ring == m.n_ring && h.depth == m.depth}};
  for (const auto& f : fields)
    if (!f.same) return fail(s, ADG_ERR_INVALID, std::string("checkpoint from an incompatible handle: ") + f.name);
  if (bytes < ckpt_bytes(s)) return fail(s, ADG_ERR_INVALID, "checkpoint truncated");
  if (!(h.dt > 0) || !std::isfinite(h.dt) || h.step < 0 || h.head < -1 || h.head >= (h.depth > 0 ? h.depth : 1))
    return fail(s, ADG_ERR_INVALID, "checkpoint has an invalid step, head or time step");
  const unsigned char* p = static_cast<const unsigned char*>(buf) + sizeof(h);
  const size_t sb = prec_bytes(s->prec);
  ADG_CUDA(s, cudaMemcpyAsync(s->w, p, (size_t)h.ndof * 8, cudaMemcpyHostToDevice, s->stream));
  p += (size_t)h.ndof * 8;
  ADG_CUDA(s, cudaMemcpyAsync(s->tr, p, (size_t)h.n_tr * sb, cudaMemcpyHostToDevice, s->stream));
  p += (size_t)h.n_tr * sb;
  if (h.n_ring > 0)
    ADG_CUDA(s, cudaMemcpyAsync(s->ring, p, (size_t)h.n_ring * sb, cudaMemcpyHostToDevice, s->stream));
  s->dt = h.dt;
  adg_status st = upload_dt_tables(s);
  if (st != ADG_OK) return st;
  ADG_CUDA(s, cudaStreamSynchronize(s->stream));  // the caller's buffer is not kept
  s->has_state = true;
  s->traces_valid = true;
  s->traces_partial = false;
  s->step = h.step;
  s->t = h.t;
  s->head = h.head;
  return ADG_OK;
}

adg_status adg_rhs(adg_solver* s, const double* u, double* k, int64_t count, int on_device) {
  if (!s) return fail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  if (!u || !k) return fail(s, ADG_ERR_INVALID, "u or k is NULL");
  if (count != s->ndof) return fail(s, ADG_ERR_INVALID, "count does not match n_dof");
  const size_t bytes = (size_t)count * sizeof(double);
  if (!on_device) {
    if (!s->tmp_u) ADG_CUDA(s, cudaMalloc((void**)&s->tmp_u, bytes));
    if (!s->tmp_k) ADG_CUDA(s, cudaMalloc((void**)&s->tmp_k, bytes));
    ADG_CUDA(s, cudaMemcpyAsync(s->tmp_u, u, bytes, cudaMemcpyHostToDevice, s->stream));
  }
  const double* ud = on_device ? u : s->tmp_u;
  double* kd = on_device ? k : s->tmp_k;
  adg_status st = launch_traces_of(s, ud);
  if (st != ADG_OK) return st;
  s->traces_valid = false;
  FluxArgs fa = base_flux_args(s);
  fa.pe_mode = 0;
  ADG_CUDA(s, launch_flux(s->prec, s->dim, s->N, fa, s->stream));
  VolArgs va;
  std::memset(&va, 0, sizeof(va));
  va.m = s->margs;
  va.tab = s->tab_dev;
  va.gamma = s->opt.gamma;
  va.gammaf = split2(s->opt.gamma);
  va.gm1 = s->opt.gamma - 1.0;
  va.gm1f = split2(s->opt.gamma - 1.0);
  va.mode = kModeRHS;
  va.w_in = ud;
  va.kout = kd;
  va.fl = s->fl;
  va.tr = s->tr;
  va.write_traces = 0;
  ADG_CUDA(s, launch_vol(s->prec, s->dim, s->N, va, s->stream));
  if (!on_device)
    ADG_CUDA(s, cudaMemcpyAsync(k, s->tmp_k, bytes, cudaMemcpyDeviceToHost, s->stream));
  ADG_CUDA(s, cudaStreamSynchronize(s->stream));
  return ADG_OK;
}

adg_status adg_get_schedule(const adg_solver* s, int64_t n0, int n, int32_t* comm, int32_t* k,
                            int32_t* iface_delay) {
  if (!s) return fail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  if (n < 0 || n0 < 0 || !comm || !k)
    return fail(const_cast<adg_solver*>(s), ADG_ERR_INVALID, "bad schedule arguments");
  return schedule_impl(s->flux, s->opt.delay_mode, s->max_delay, s->np, s->dim, s->P,
                       s->opt.seed, s->opt.random_delay_max, n0, n, comm, k, iface_delay);
}

adg_status adg_info(const adg_solver* s, double* t, int64_t* step, double* dt, int64_t* n_dof) {
  if (!s) return fail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  if (t) *t = s->t;
  if (step) *step = s->step;
  if (dt) *dt = s->dt;
  if (n_dof) *n_dof = s->ndof;
  return ADG_OK;
}

adg_status adg_conservation(adg_solver* s, double* sums) {
  if (!s) return fail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  if (!sums) return fail(s, ADG_ERR_INVALID, "sums is NULL");
  ADG_CUDA(s, launch_conservation(s->dim, s->N, s->margs, s->tab_dev, s->J, s->w, s->red_partial,
                                  s->red_out, s->red_blocks, s->stream));
  ADG_CUDA(s, cudaMemcpyAsync(sums, s->red_out, s->NV * sizeof(double), cudaMemcpyDeviceToHost,
                              s->stream));
  ADG_CUDA(s, cudaStreamSynchronize(s->stream));
  return ADG_OK;
}

adg_status adg_l2_error_vortex(adg_solver* s, double t, double beta, double x0, double y0,
                               double* err3) {
  if (!s) return fail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  if (!err3) return fail(s, ADG_ERR_INVALID, "err3 is NULL");
  const double Lx = s->mesh.hi[0] - s->mesh.lo[0], Ly = s->mesh.hi[1] - s->mesh.lo[1];
  ADG_CUDA(s, launch_l2_vortex(s->dim, s->N, s->margs, s->mesh.lo, s->h, s->tab_dev, s->opt.gamma,
                               t, beta, x0, y0, Lx, Ly, s->w, s->red_partial, s->red_out,
                               s->red_blocks, s->stream));
  double sq[3];
  ADG_CUDA(s, cudaMemcpyAsync(sq, s->red_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  ADG_CUDA(s, cudaStreamSynchronize(s->stream));
  for (int i = 0; i < 3; ++i) err3[i] = std::sqrt(sq[i]);
  return ADG_OK;
}

adg_status adg_check_finite(adg_solver* s) {
  if (!s) return fail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  ADG_CUDA(s, launch_check_finite(s->ndof, s->w, s->flag, s->stream));
  int f = 0;
  ADG_CUDA(s, cudaMemcpyAsync(&f, s->flag, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  ADG_CUDA(s, cudaStreamSynchronize(s->stream));
  if (f) return fail(s, ADG_ERR_NONFINITE, "state holds NaN or Inf");
  return ADG_OK;
}

adg_status adg_set_learned_model(adg_solver* s, const uint16_t* params_bf16, float trust) {
  if (!s) return fail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  if (!params_bf16 || !(trust >= 0.0f)) return fail(s, ADG_ERR_INVALID, "bad model arguments");
  if (!s->mlp) ADG_CUDA(s, cudaMalloc((void**)&s->mlp, kMlpParamCount * sizeof(uint16_t)));
  ADG_CUDA(s, cudaMemcpyAsync(s->mlp, params_bf16, kMlpParamCount * sizeof(uint16_t),
                              cudaMemcpyHostToDevice, s->stream));
  ADG_CUDA(s, cudaStreamSynchronize(s->stream));
  s->trust = trust;
  return ADG_OK;
}

adg_status adg_set_trace_log(adg_solver* s, double* dev_log, int64_t n_records, int64_t* record_len) {
  if (!s) return fail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  if (record_len) *record_len = (int64_t)2 * s->NV * s->npe * s->NF;
  if (n_records < 0) return fail(s, ADG_ERR_INVALID, "n_records must be >= 0");
  s->log = dev_log;
  s->log_cap = dev_log ? n_records : 0;
  s->log_count = 0;
  return ADG_OK;
}

adg_status adg_learned_samples(adg_solver* s, const double* dev_log, int64_t n_records,
                               const int32_t* dev_picks, int64_t n, float* dev_x,
                               float* dev_target, int32_t* dev_ok) {
  if (!s) return fail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  if (!dev_log || !dev_picks || !dev_x || !dev_target || !dev_ok || n < 0 || n >= (1ll << 31))
    return fail(s, ADG_ERR_INVALID, "bad sample arguments");
  (void)n_records;
  // AT weights (N_p = 2) and stage delays for k = 0..15 and every stage
  const int K = kMaxCoefDelay, S = s->stages;
  std::vector<double> ctab((size_t)K * S * 3), km((size_t)K * S);
  for (int k = 0; k < K; ++k)
    for (int m = 0; m < S; ++m) {
      long double c[kMaxN];
      at_weights_ld(2, (long double)k + s->rkc[m], c);
      for (int l = 0; l < 3; ++l) ctab[((size_t)k * S + m) * 3 + l] = (double)c[l];
      km[(size_t)k * S + m] = k + s->rkc[m];
    }
  double* dtab = nullptr;
  ADG_CUDA(s, cudaMalloc((void**)&dtab, (ctab.size() + km.size()) * sizeof(double)));
  cudaError_t e = cudaMemcpy(dtab, ctab.data(), ctab.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(dtab + ctab.size(), km.data(), km.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = launch_samples(dev_log, (int64_t)2 * s->NV * s->npe * s->NF, S, dev_picks, (int)n, dtab,
                       dtab + ctab.size(), K - 1, dev_x, dev_target, dev_ok, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  cudaFree(dtab);
  if (e != cudaSuccess) return cuda_fail(s, e, "adg_learned_samples");
  return ADG_OK;
}

adg_status adg_set_profiling(adg_solver* s, int enable) {
  if (!s) return fail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  s->profiling = enable != 0;
  s->ev_used = 0;
  s->prof_ms[0] = s->prof_ms[1] = 0.0;
  s->prof_n[0] = s->prof_n[1] = 0;
  return ADG_OK;
}

adg_status adg_get_profile(adg_solver* s, double* ms, int64_t* launches) {
  if (!s) return fail(nullptr, ADG_ERR_INVALID, "handle is NULL");
  if (!ms || !launches) return fail(s, ADG_ERR_INVALID, "ms or launches is NULL");
  ADG_CUDA(s, prof_fold(s));
  for (int kind = 0; kind < 2; ++kind) {
    ms[kind] = s->prof_ms[kind];
    launches[kind] = s->prof_n[kind];
    s->prof_ms[kind] = 0.0;
    s->prof_n[kind] = 0;
  }
  return ADG_OK;
}

const char* adg_last_error(const adg_solver* s) { return s ? s->err.c_str() : g_err.c_str(); }

void adg_destroy(adg_solver* s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  free_all(s);
  delete s;
}

adg_status adg_host_gauss(int n, double* x, double* w) {
  if (n < 1 || n > 9 || !x || !w) return fail(nullptr, ADG_ERR_INVALID, "bad arguments");
  gauss_legendre(n, x, w);
  return ADG_OK;
}

adg_status adg_host_at_coeffs(int np, double km, double* c) {
  if (np < 0 || np > 7 || !c) return fail(nullptr, ADG_ERR_INVALID, "bad arguments");
  at_weights(np, km, c);
  return ADG_OK;
}

adg_status adg_host_rk(adg_rk scheme, int* stages, double* a, double* b, double* c) {
  if (!stages || !a || !b || !c) return fail(nullptr, ADG_ERR_INVALID, "bad arguments");
  double ta[8], tb[8], tc[8];
  int s = rk_coeffs(scheme, ta, tb, tc);
  if (!s) return fail(nullptr, ADG_ERR_INVALID, "unknown scheme");
  *stages = s;
  for (int i = 0; i < s; ++i) {
    a[i] = ta[i];
    b[i] = tb[i];
    c[i] = tc[i];
  }
  return ADG_OK;
}

adg_status adg_host_schedule(adg_flux flux, adg_delay_mode mode, int max_delay, int np, int dim,
                             const int P[3], uint64_t seed, int random_delay_max, int64_t n0,
                             int n, int32_t* comm, int32_t* k, int32_t* iface_delay) {
  if (!P || !comm || !k || n < 0 || n0 < 0 || (dim != 2 && dim != 3))
    return fail(nullptr, ADG_ERR_INVALID, "bad arguments");
  if (mode == ADG_DELAY_CAA && flux == ADG_FLUX_STD_DELAYED && max_delay < 1)
    return fail(nullptr, ADG_ERR_INVALID, "max_delay must be >= 1");
  int Pd[3] = {P[0], P[1], dim == 3 ? P[2] : 1};
  return schedule_impl(flux, mode, max_delay, np, dim, Pd, seed, random_delay_max, n0, n, comm, k,
                       iface_delay);
}

int adg_host_num_interfaces(int dim, const int P[3]) {
  if (!P || (dim != 2 && dim != 3)) return -1;
  int Pd[3] = {P[0], P[1], dim == 3 ? P[2] : 1};
  return num_interfaces(dim, Pd);
}

}  // extern "C"
