// Internal declarations shared by the host side and the kernels of the ADG library.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace adg {

constexpr int kMaxN = 8;        // nodes per direction (degree <= 7)
constexpr int kMaxN3D = 6;      // 3D builds degree <= 5
constexpr int kMaxRing = 24;    // ring levels (random_delay_max + np + 1 <= 15 + 7 + 1)
constexpr int kMaxCoefDelay = 16;

// Operator tables in FP64; kernels convert entries to their arithmetic type.
struct OpTables {
  double Q[3][kMaxN * kMaxN];  // (2/h_d) omega_a l_i'(xi_a) / omega_i, entry [i*N + a]
  double Lp[3][kMaxN];         // (1/h_d) l_i(+1) / omega_i: half the lift (the stored
  double Lm[3][kMaxN];         // (1/h_d) l_i(-1) / omega_i   face fluxes are doubled)
  double Tp[kMaxN];            // l_a(+1): trace at the high face
  double Tm[kMaxN];            // l_a(-1): trace at the low face
  double xi[kMaxN];            // Gauss nodes on [-1, 1]
  double wq[kMaxN];            // Gauss weights
  double xe[kMaxN + 1];        // (N+1)-point Gauss nodes for error integrals
  double we[kMaxN + 1];
  double Le[(kMaxN + 1) * kMaxN];  // l_a(xe_p), entry [p*N + a]
  // the same operator tables split into FP32 pairs (hi, lo) for the FP32 and pair kernels
  float2 Qf[3][kMaxN * kMaxN];
  float2 Lpf[3][kMaxN];
  float2 Lmf[3][kMaxN];
  float2 Tpf[kMaxN];
  float2 Tmf[kMaxN];
  // the operator tables times the time step (2N scheme: the volume kernel then produces
  // dt * k directly); filled once dt is known
  double Qs[3][kMaxN * kMaxN];
  double Lps[3][kMaxN];
  double Lms[3][kMaxN];
  float2 Qsf[3][kMaxN * kMaxN];
  float2 Lpsf[3][kMaxN];
  float2 Lmsf[3][kMaxN];
};

struct MeshArgs {
  int n[3];
  int64_t ne;
  int64_t es[3];  // element index stride per direction
  // Division by n[0] and n[1] as a multiply-high (division by invariant integers, Granlund
  // & Montgomery, PLDI 1994): q = floor(e / n) = umulhi64(e, M) with M = ceil(2^64 / n),
  // exact for e < 2^64 / n, hence for every 32-bit e when n < 2^31; n = 1 is special-cased.
  uint64_t divm[2];
};

// Fills es[] and divm[] from n[] (host side).
inline void mesh_finish(MeshArgs& m) {
  m.es[0] = 1;
  m.es[1] = m.n[0];
  m.es[2] = (int64_t)m.n[0] * m.n[1];
  for (int i = 0; i < 2; ++i)
    m.divm[i] = m.n[i] > 1 ? ~0ull / (uint64_t)m.n[i] + 1ull : 0ull;
}

enum UpdateMode { kModeRHS = 0, kMode2R = 1, kMode2N = 2 };

struct __align__(16) VolArgs {
  MeshArgs m;
  const OpTables* tab;
  double gamma;
  float2 gammaf;   // gamma as an FP32 pair
  double gm1;      // gamma - 1 (every node's pressure needs it)
  float2 gm1f;     // gamma - 1 as an FP32 pair
  int mode;        // UpdateMode
  int stage, last; // stage index; last = 1 on the final stage of a step
  double ca, cb;   // 2R: dt*a_m, dt*b_m ; 2N: A_m, B_m
  double dt;
  float2 caf, cbf, dtf;  // the same coefficients as FP32 pairs
  const double* w_in;    // FP64 stage input when it is the solution (2N, and 2R stage 0)
  const void* r_in;      // 2R stages > 0: the stage register r (operator storage type)
  double* w;             // solution (read + write, FP64)
  void* x;               // 2R: r (written); 2N: q (read + written); operator storage type
  double* kout;          // RHS mode: k = M^-1 L(w_in), FP64
  const void* fl;        // face fluxes [d][v][e][j] (storage type of the arithmetic)
  void* tr;              // traces of the next stage input [d][side][v][e][j]
  int write_traces;
  int scaled;            // 1: use the dt-scaled tables (2N), the accumulator is dt * k
  int bulk;              // 1: n_elem * nodes is a multiple of 4, so the element path may
                         // stage whole tiles by TMA bulk copies (16-byte aligned rows)
};

struct __align__(16) FluxArgs {
  MeshArgs m;
  double gamma;
  float2 gammaf;
  double gm1;      // gamma - 1 (every face node's pressures need it)
  float2 gm1f;
  const void* tr;
  void* fl;
  // subdomain-face handling
  int pe_mode;          // 0: all faces fresh; 1: apply ring rules on PE faces
  int flux_kind;        // adg_flux
  const int32_t* pe_slot;   // [d][e] -> PE face slot or -1
  const int32_t* pe_iface;  // [slot] -> interface id
  int64_t npe;              // PE faces
  void* ring;               // [level][v][slot][j] (AT_TRACE: [level][2][v][slot][j])
  int depth, head;          // ring depth, level written last (after this stage's store)
  int store;                // write fresh value to ring[head] (stage 0 of a storing step)
  int random;               // per-interface delays (random mode)
  int uniform_delay;        // CAA: 0 on communication steps, k otherwise
  int nterms;               // 1 (standard) or np+1 (AT)
  uint64_t seed;
  int64_t step;
  int n_iface, dmax, np;
  double ctab[kMaxCoefDelay][kMaxN];  // AT weights per delay for this stage
  float2 ctabf[kMaxCoefDelay][kMaxN]; // the same as FP32 pairs
};

// Arguments of the fused per-stage kernel (fused.cuh): one launch per RK stage does the
// face fluxes and the volume/update work of a tile of elements.
struct __align__(16) FusedArgs {
  VolArgs v;           // RK stage: coefficients, tables, w, x (mode 2R or 2N)
  FluxArgs f;          // face rules: gamma, ring, subdomain slots, AT weights of the stage
  const void* tr_in;   // traces of this stage's input, [d][side][v][e][j] (tile-boundary faces)
  void* tr_out;        // traces of the next stage's input on tile-boundary faces
  int ntile[3];        // tiles per direction
  int tma;             // 1: stage the tile by TMA tensor copies; 0: plain loads
  int* err;            // nonzero after a wait gave up (1: the tile's copies never completed)
};

struct TraceArgs {
  MeshArgs m;
  const OpTables* tab;
  const double* u;
  void* tr;
};

// Learned correction of subdomain traces (learned.cu).
struct LearnArgs {
  MeshArgs m;
  double gamma;
  float2 gammaf;
  double gm1;               // gamma - 1, as in the face-flux arguments
  float2 gm1f;
  const void* ring;         // trace ring [level][2][v][slot][j]
  void* fl;                 // face fluxes to overwrite on subdomain faces
  const int32_t* face_d;    // [slot] direction
  const int32_t* face_e;    // [slot] low-side element
  const int32_t* pe_iface;  // [slot] interface (random mode)
  const uint16_t* mlp;      // BF16 parameters
  float trust;              // largest accepted |correction| in units of the level spread
  int64_t npe;
  int depth, head, random, uniform_delay, n_iface, dmax;
  uint64_t seed;
  int64_t step;
  double ctab[kMaxCoefDelay][kMaxN];
  float2 ctabf[kMaxCoefDelay][kMaxN];
  double km[kMaxCoefDelay];  // stage delay k_m = k + c_m of each delay k
  // per-channel work buffers (channel = ((slot * NF + j) * 2 + side) * (dim+2) + var)
  void* E;                  // AT extrapolation (operator storage type)
  double* s;                // AT error estimate E3 - E2 (0: no correction)
  float* x;                 // network inputs [4]
  float* y;                 // network outputs
};
cudaError_t launch_learned(int prec, int dim, int N, const LearnArgs& a, cudaStream_t s);
cudaError_t launch_samples(const double* log, int64_t rec_len, int stages, const int32_t* picks,
                           int n, const double* ctab, const double* kmtab, int kmax, float* x,
                           float* target, int* ok, cudaStream_t s);
cudaError_t launch_log_traces(int prec, int dim, int N, const void* tr, const int32_t* face_d,
                              const int32_t* face_e, const MeshArgs& m, int64_t npe, double* out,
                              cudaStream_t s);

// Launchers (one per arithmetic), implemented in the kernel translation units.
// prec: 0 = FP64, 1 = FP32, 2 = FP32 pair.
cudaError_t launch_trace(int prec, int dim, int N, const TraceArgs& a, cudaStream_t s);
cudaError_t launch_flux(int prec, int dim, int N, const FluxArgs& a, cudaStream_t s);
cudaError_t launch_vol(int prec, int dim, int N, const VolArgs& a, cudaStream_t s);
// Volume kernel with element-local face fluxes (kv_*.cu): a.v the stage (a.v.tr receives
// the next stage's traces), a.f the face rules, a.tr_in the current traces.
cudaError_t launch_vol_faces(int prec, int dim, int N, const FusedArgs& a, cudaStream_t s);
bool kernels_available(int prec, int dim, int N);
// Fused per-stage kernel (kf_*.cu): tile shape of (dim, N) in elements per direction, and
// the launch with the TMA tensor maps of w and of the RK register.
bool fused_tile(int dim, int N, int* tile);
cudaError_t launch_fused(int prec, int dim, int N, const FusedArgs& a, const CUtensorMap& tw,
                         const CUtensorMap& tx, cudaStream_t s);
size_t storage_bytes(int prec);  // bytes per stored trace/flux value

// Auxiliary kernels (FP64), in aux.cu.
cudaError_t launch_init_vortex(int dim, int N, const MeshArgs& m, const double* lo,
                               const double* h, const OpTables* tab, double gamma, double t,
                               double beta, double x0, double y0, double Lx, double Ly,
                               double* u, cudaStream_t s);
cudaError_t launch_init_tgv(int N, const MeshArgs& m, const double* lo, const double* h,
                            const OpTables* tab, double gamma, double mach, double* u,
                            cudaStream_t s);
cudaError_t launch_conservation(int dim, int N, const MeshArgs& m, const OpTables* tab,
                                double J, const double* u, double* partial, double* out,
                                int nblocks, cudaStream_t s);
cudaError_t launch_max_speed(int dim, int N, const MeshArgs& m, double gamma, const double* u,
                             double* partial, double* out, int nblocks, cudaStream_t s);
cudaError_t launch_l2_vortex(int dim, int N, const MeshArgs& m, const double* lo,
                             const double* h, const OpTables* tab, double gamma, double t,
                             double beta, double x0, double y0, double Lx, double Ly,
                             const double* u, double* partial, double* out, int nblocks,
                             cudaStream_t s);
cudaError_t launch_check_finite(int64_t n, const double* u, int* flag, cudaStream_t s);

}  // namespace adg
