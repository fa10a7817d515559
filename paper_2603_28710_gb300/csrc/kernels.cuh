// Kernel templates of the ADG right-hand side, parameterised by dimension D, nodes per
// direction N = degree + 1 and the arithmetic type R of the operator (double, float or
// the FP32-pair type of df64.cuh).  The solution w is FP64 in every variant; the RK
// register (r or q) is stored in the operator's storage type.
//
// Per Runge-Kutta stage the solver runs two kernels:
//   flux_kernel : one thread per (direction, face, face node): numerical flux of Eq. 8-9
//                 from the two stored traces; on faces between subdomains it applies the
//                 delayed / AT rules of Algorithms 2-3 (Eq. 13-14) against a ring buffer.
//   vol_kernel  : one thread per node, a tile of elements per block: pointwise Euler flux
//                 (Eq. 2), sum-factorised weak derivative along each direction, face lift,
//                 inverse mass (diagonal for collocated Gauss points; folded into the
//                 tables), the low-storage RK update (Eq. 10 or the 2N form), and the
//                 face traces of the next stage input.
// or one kernel:
//   vol_faces_kernel : the volume kernel with each element evaluating the numerical flux
//                 on its own faces from the stored traces (no face-flux array).
// Index arithmetic is 32-bit: the host rejects meshes with 2^31 or more degrees of freedom.
#pragma once
#include <type_traits>
#include <cuda_runtime.h>
#include <stdint.h>

#include "adg_internal.h"
#include "arith.cuh"

namespace adg {

template <int B, int E>
struct IPow { static constexpr int value = B * IPow<B, E - 1>::value; };
template <int B>
struct IPow<B, 0> { static constexpr int value = 1; };

// Element tile of the volume kernel: about TT threads per block, one thread per node.
template <int D, int N, int TT = 128>
struct Tile {
  static constexpr int ND = IPow<N, D>::value;
  static constexpr int NF = ND / N;
  static constexpr int NV = D + 2;
  static constexpr int EPB = (TT / ND) > 0 ? (TT / ND) : 1;
  static constexpr int THREADS = EPB * ND;
};

// Element strides (in values) of the volume kernel's shared-memory tiles.  For 4-byte
// values the stride is padded to be congruent to the node count modulo the 32 banks, so
// that a warp's consecutive nodes fall into consecutive banks across element boundaries
// (unpadded, a 2D p=4 FP32 tile put two elements' nodes into the same banks: 2-way
// conflicts on every store of the pointwise fluxes and the next stage input).
constexpr int bank_pad(int base, int nd, int bytes) {
  return bytes == 4 ? ((nd - base) % 32 + 32) % 32 : 0;
}
template <int D, int N, typename R>
constexpr int sf_stride() {  // pointwise fluxes [el][D][NV][ND]
  return D * (D + 2) * IPow<N, D>::value +
         bank_pad(D * (D + 2) * IPow<N, D>::value, IPow<N, D>::value, (int)sizeof(R));
}
template <int D, int N, typename C>
constexpr int sx_stride() {  // next stage input [el][NV][ND]
  return (D + 2) * IPow<N, D>::value +
         bank_pad((D + 2) * IPow<N, D>::value, IPow<N, D>::value, (int)sizeof(C));
}

// floor(e / m.n[i]) for 0 <= e < 2^31 (multiply-high by the precomputed inverse)
__device__ __forceinline__ int mesh_div(const MeshArgs& m, int i, int e) {
  return m.n[i] == 1 ? e : (int)__umul64hi((unsigned long long)(unsigned)e, m.divm[i]);
}

// Blocks per SM that leave `regs` registers per thread (0: no budget): each of the 4 SM
// sub-partitions holds 16384 registers and a whole number of warps.
constexpr int min_blocks_for(int regs, int threads) {
  if (regs == 0) return 1;
  if (threads <= 64 && regs < 48) regs = 48;
  const int warps = (threads + 31) / 32;
  const int b = (16384 / (regs * 32)) * 4 / warps;
  return b < 1 ? 1 : (b > 32 ? 32 : b);
}

__device__ __forceinline__ void elem_coords(const MeshArgs& m, int e, int* c) {
  const int q = mesh_div(m, 0, e);
  c[0] = e - q * m.n[0];
  c[2] = mesh_div(m, 1, q);
  c[1] = q - c[2] * m.n[1];
}

// index of the neighbour of element e (coordinates c) one step s (+1/-1) along d, periodic
// (selects instead of indexing c by a runtime d keep c in registers)
__device__ __forceinline__ int elem_shift(const MeshArgs& m, int e, const int* c, int d, int s) {
  const int cd = d == 0 ? c[0] : (d == 1 ? c[1] : c[2]);
  int k = cd + s;
  if (k < 0) k += m.n[d];
  if (k >= m.n[d]) k -= m.n[d];
  return e + (k - cd) * (int)m.es[d];
}

// Pointwise Euler flux columns F_d(w), d < D (Eq. 2-3, no source).
template <int D, typename R>
__device__ __forceinline__ void euler_flux_all(const R (&w)[D + 2], R gm1, R (&F)[D][D + 2]) {
  const R irho = r_rcp(w[0]);
  R u[D];
  typename Arith<R>::Acc kacc = acc_zero(typename Arith<R>::Acc());
#pragma unroll
  for (int d = 0; d < D; ++d) {
    u[d] = w[1 + d] * irho;
    kacc = acc_fma(w[1 + d], u[d], kacc);
  }
  const R kin2 = acc_result(kacc);
  const R p = gm1 * sub_half(w[D + 1], kin2);
  const R ep = w[D + 1] + p;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    F[d][0] = w[1 + d];
#pragma unroll
    for (int c = 0; c < D; ++c)  // rho u_c u_d is symmetric: each product once
      F[d][1 + c] = c < d ? F[c][1 + d] : (c == d ? r_fma(w[1 + c], u[d], p) : w[1 + c] * u[d]);
    F[d][D + 1] = ep * u[d];
  }
}

// Flux column along e_d and |u|^2 + c^2 of one trace state (d is a runtime direction;
// selects instead of indexing keep everything in registers).
template <int D, typename R>
__device__ __forceinline__ void side_flux(const R (&w)[D + 2], int d, R gamma, R gm1,
                                          R (&fd)[D + 2], R& s2) {
  const R irho = r_rcp(w[0]);
  R k2 = R(0.0f), ud = R(0.0f), md = w[1];
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const R uc = w[1 + c] * irho;
    k2 = r_fma(w[1 + c], uc, k2);  // rho |u|^2
    if (c == d) {
      ud = uc;
      md = w[1 + c];
    }
  }
  const R p = gm1 * sub_half(w[D + 1], k2);  // (gamma - 1) (E - rho |u|^2 / 2)
  s2 = r_fma(gamma, p, k2) * irho;           // |u|^2 + gamma p / rho
  fd[0] = md;
#pragma unroll
  for (int c = 0; c < D; ++c) fd[1 + c] = c == d ? r_fma(w[1 + c], ud, p) : w[1 + c] * ud;
  fd[D + 1] = (w[D + 1] + p) * ud;
}

// Twice the Rusanov flux along +e_d (Eq. 8) with lambda = 1/2 max(sqrt(|u|^2 + c^2))
// (Eq. 9): f = F(w-) + F(w+) + lambda (w- - w+).  The factor 1/2 is folded into the lift
// coefficients of the volume kernel (one operation less per value; scaling by two is
// exact, so the results equal those of the halved form).  Stored fluxes, the ring of
// subdomain-face levels and their AT combinations all carry the factor two.
template <int D, typename R>
__device__ __forceinline__ void llf_flux(const R (&wm)[D + 2], const R (&wp)[D + 2], int d,
                                         R gamma, R gm1, R (&f)[D + 2]) {
  constexpr int NV = D + 2;
  R fm[NV], fp[NV], sm, sp;
  if constexpr (std::is_same<R, df64>::value) {
    // FP32 pairs: both sides in the two lanes of packed FP32x2 instructions
    df64x2 w2[NV], f2[NV], s2;
#pragma unroll
    for (int v = 0; v < NV; ++v) w2[v] = df64x2_of(wm[v], wp[v]);
    side_flux<D, df64x2>(w2, d, df64x2_of(gamma, gamma), df64x2_of(gm1, gm1), f2, s2);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      fm[v] = df64x2_lane(f2[v], 0);
      fp[v] = df64x2_lane(f2[v], 1);
    }
    sm = df64x2_lane(s2, 0);
    sp = df64x2_lane(s2, 1);
  } else {
    side_flux<D, R>(wm, d, gamma, gm1, fm, sm);
    side_flux<D, R>(wp, d, gamma, gm1, fp, sp);
  }
  const R lam = scale_pow2(r_sqrt(r_max(sm, sp)), 0.5f);
#pragma unroll
  for (int v = 0; v < NV; ++v) f[v] = r_fma(lam, wm[v] - wp[v], fm[v] + fp[v]);
}

// Transverse coordinates of face node j of a face normal to d -> base node index of the
// line of nodes along d through it.
template <int D, int N>
__device__ __forceinline__ int line_base(int d, int j) {
  int base = 0, stride = 1, t = j;
#pragma unroll
  for (int c = 0; c < D; ++c) {
    if (c != d) {
      base += (t % N) * stride;
      t /= N;
    }
    stride *= N;
  }
  return base;
}

// Face node index of volume node (ix) on a face normal to d.
template <int D, int N>
__device__ __forceinline__ int face_index(int d, const int* ix) {
  int j = 0, stride = 1;
#pragma unroll
  for (int c = 0; c < D; ++c) {
    if (c != d) {
      j += ix[c] * stride;
      stride *= N;
    }
  }
  return j;
}

// Asynchronous 4- and 8-byte copies global -> shared memory (cp.async; sm_80 and later).
// The issuing thread waits for its own copies with cp_async_wait<n> (at most n of its
// committed groups still pending); nothing spins.
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int n>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(n) : "memory");
}

// ---- mbarrier and TMA bulk copies (PTX) -----------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for phase `parity` of the barrier for at most `limit` SM clock cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}
// 1D bulk copy global -> shared by the TMA engine (both addresses 16-byte aligned, size a
// multiple of 16 bytes), completion counted on the mbarrier
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// about one second at the GB300 SM clock
constexpr long long kWaitLimitCycles = 2000000000ll;

// Arithmetic of the trace interpolation for an operator arithmetic R: the FP32-pair kernels
// interpolate in native FP64 (their FP64 pipe is otherwise idle and the RK update hands
// over the FP64 stage input), the others in R itself.
template <typename R> struct TraceCompute { using C = R; };
template <> struct TraceCompute<df64> { using C = double; };

__device__ __forceinline__ void store_trace(double* p, double v) { *p = v; }
__device__ __forceinline__ void store_trace(float* p, float v) { *p = v; }
__device__ __forceinline__ void store_trace(float2* p, double v) {
  const df64 q = d2df_int(v);
  *p = make_float2(q.hi, q.lo);
}
__device__ __forceinline__ void store_trace(float2* p, df64 v) { *p = make_float2(v.hi, v.lo); }

// Traces of a tile of elements held in shared memory sX[el][v][node] (compute type C,
// element stride SXS) -> tr.
// FP32 and FP32-pair operators: a thread owns one (direction, side, variable, face node)
// combination, so its line of nodes, stride and interpolation weights are set up once, and
// interpolates it for a run of the tile's elements (the runs split the elements when the
// block has threads to spare); this halves their instruction count in this phase.  The
// FP64 operator is bound by its FP64 pipe, not by issue, and keeps one flat loop over all
// (element, face node) items, which spreads the FP64 work over every thread.
template <int D, int N, typename R, int TT = 128, typename C = R,
          int SXS = (D + 2) * IPow<N, D>::value>
__device__ __forceinline__ void write_traces(const MeshArgs& m, const OpTables* tab, const C* sX,
                                             int e0, typename Arith<R>::S* tr) {
  using T = Tile<D, N, TT>;
  constexpr int ND = T::ND, NF = T::NF, NV = T::NV, EPB = T::EPB;
  const int ne = (int)m.ne;
  if constexpr (std::is_same<R, double>::value) {
    constexpr int TOTAL = EPB * 2 * D * NV * NF;
    for (int g = threadIdx.x; g < TOTAL; g += blockDim.x) {
      const int jj = g % (EPB * NF);
      const int rest = g / (EPB * NF);  // (d*2 + side)*NV + v
      const int el = jj / NF, j = jj - el * NF;
      const int e = e0 + el;
      if (e >= ne) continue;
      const int v = rest % NV, ds = rest / NV;
      const int d = ds >> 1, side = ds & 1;
      const int base = line_base<D, N>(d, j);
      const int stride = d == 0 ? 1 : (d == 1 ? N : N * N);
      const double* tw = side ? tab->Tp : tab->Tm;
      double acc = 0.0;
#pragma unroll
      for (int a = 0; a < N; ++a) acc = fma(tw[a], sX[el * SXS + v * ND + base + a * stride], acc);
      store_trace(tr + ((ds * NV + v) * ne + e) * NF + j, acc);
    }
  } else {
    constexpr int CT = 2 * D * NV * NF;                            // combinations
    constexpr int CH = T::THREADS / CT > 0 ? T::THREADS / CT : 1;  // element runs
    constexpr int RUN = (EPB + CH - 1) / CH;                       // elements per run
    for (int g = threadIdx.x; g < CT * CH; g += blockDim.x) {
      const int c = g % CT, ch = g / CT;
      const int j = c % NF, rest = c / NF;  // rest = (d*2 + side)*NV + v
      const int v = rest % NV, ds = rest / NV;
      const int d = ds >> 1, side = ds & 1;
      const int base = line_base<D, N>(d, j);
      const int stride = d == 0 ? 1 : (d == 1 ? N : N * N);
      const double* tw = side ? tab->Tp : tab->Tm;
      const float2* twf = side ? tab->Tpf : tab->Tmf;
      C t[N];
#pragma unroll
      for (int a = 0; a < N; ++a) t[a] = Arith<C>::tab(tw, twf, a);
      const int el0 = ch * RUN;
      const int el1 = el0 + RUN < EPB ? el0 + RUN : EPB;
      typename Arith<R>::S* dst = tr + ((ds * NV + v) * ne + e0) * NF + j;
      for (int el = el0; el < el1 && e0 + el < ne; ++el) {
        const C* x = sX + el * SXS + v * ND + base;
        typename Arith<C>::Acc acc = acc_zero(typename Arith<C>::Acc());
#pragma unroll
        for (int a = 0; a < N; ++a) acc = acc_fma(t[a], x[a * stride], acc);
        store_trace(dst + el * NF, acc_result(acc));
      }
    }
  }
}

template <int D, int N, typename R>
__global__ void __launch_bounds__(Tile<D, N>::THREADS) trace_kernel(const TraceArgs A) {
  using T = Tile<D, N>;
  using C = typename TraceCompute<R>::C;
  constexpr int ND = T::ND, NV = T::NV, EPB = T::EPB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sX = reinterpret_cast<C*>(smem_raw);
  const int el = threadIdx.x / ND, node = threadIdx.x - el * ND;
  const int e0 = blockIdx.x * EPB;
  const int e = e0 + el;
  const int ne = (int)A.m.ne;
  if (e < ne) {
#pragma unroll
    for (int v = 0; v < NV; ++v)
      sX[(el * NV + v) * ND + node] = Arith<C>::from_double(A.u[(v * ne + e) * ND + node]);
  }
  __syncthreads();
  write_traces<D, N, R, 128, C>(A.m, A.tab, sX, e0, reinterpret_cast<typename Arith<R>::S*>(A.tr));
}

// ---- Runge-Kutta update of one node -------------------------------------------------
// Native FP64: everything in FP64.  FP32 / FP32 pair: the RK register and the stage input
// stay in the operator arithmetic; only the accumulation into w is FP64 (one or two DADD).
__device__ __forceinline__ double add_increment(double w0, double d) { return w0 + d; }
__device__ __forceinline__ double add_increment(double w0, float d) { return w0 + f2d_int(d); }
__device__ __forceinline__ double add_increment(double w0, df64 d) {
  return (w0 + f2d_int(d.hi)) + f2d_int(d.lo);
}

// Value of the next stage input handed to the trace interpolation (compute type C): the
// operator's own value, or the FP64 one for the FP32-pair kernels.
template <typename C, typename R>
__device__ __forceinline__ C trace_value(double, R xr) { return xr; }
template <>
__device__ __forceinline__ double trace_value<double, df64>(double xd, df64) { return xd; }

template <typename R>
struct Update {
  using S = typename Arith<R>::S;
  // returns the next stage input at this node/variable; xd receives it in FP64 where the
  // update has it in FP64 (the FP32-pair traces use it)
  // pre: the solution w0 and the 2N register q at this index were staged in advance (pw0,
  // pq) by the volume kernel
  __device__ static __forceinline__ R apply(const VolArgs& A, int idx, R k, R u_in, double& xd,
                                            bool pre = false, double pw0 = 0.0, R pq = R(0.0f)) {
    if (A.mode == kModeRHS) {
      A.kout[idx] = Arith<R>::to_double(k);
      xd = Arith<R>::to_double(u_in);
      return u_in;
    }
    const double w0 = pre ? pw0 : A.w[idx];
    S* x = reinterpret_cast<S*>(A.x);
    if (A.mode == kMode2R) {
      const R cb = Arith<R>::pair(A.cb, A.cbf), ca = Arith<R>::pair(A.ca, A.caf);
      const double w1 = add_increment(w0, cb * k);
      A.w[idx] = w1;
      if (A.last) {
        xd = w1;
        return Arith<R>::from_double(w1);
      }
      const double r1d = add_increment(w0, ca * k);
      const R r1 = Arith<R>::from_double(r1d);
      Arith<R>::store(x + idx, r1);
      xd = r1d;
      return r1;
    }
    const R cA = Arith<R>::pair(A.ca, A.caf), cB = Arith<R>::pair(A.cb, A.cbf);
    const R dtk = A.scaled ? k : Arith<R>::pair(A.dt, A.dtf) * k;
    const R q1 = (A.stage > 0) ? r_fma(cA, pre ? pq : Arith<R>::load(x + idx), dtk) : dtk;
    const double w1 = add_increment(w0, cB * q1);
    A.w[idx] = w1;
    if (!A.last) Arith<R>::store(x + idx, q1);
    xd = w1;
    if constexpr (std::is_same<R, float>::value) {
      // FP32 operator: the next stage input (stage input u_in = w0 in FP32, plus the
      // increment) within an FP32 ulp of float(w1), without a conversion
      return r_fma(cB, q1, u_in);
    } else {
      return Arith<R>::from_double(w1);
    }
  }
};

template <>
struct Update<double> {
  __device__ static __forceinline__ double apply(const VolArgs& A, int idx, double k, double u_in,
                                                 double& xd, bool = false, double = 0.0,
                                                 double = 0.0) {
    xd = 0.0;
    if (A.mode == kModeRHS) {
      A.kout[idx] = k;
      return u_in;
    }
    const double w0 = A.w[idx];
    double* x = reinterpret_cast<double*>(A.x);
    if (A.mode == kMode2R) {
      const double w1 = fma(A.cb, k, w0);
      A.w[idx] = w1;
      if (A.last) return w1;
      const double r1 = fma(A.ca, k, w0);
      x[idx] = r1;
      return r1;
    }
    const double dtk = A.scaled ? k : A.dt * k;
    const double q1 = A.stage > 0 ? fma(A.ca, x[idx], dtk) : dtk;
    const double w1 = fma(A.cb, q1, w0);
    A.w[idx] = w1;
    if (!A.last) x[idx] = q1;
    return w1;
  }
};

// Pointwise fluxes of a tile in shared memory: [EPB][D][NV][ND] values of R, except for
// the 2D FP32 pairs, which keep pairs of variables together for the packed sweeps:
// [EPB][D][NV/2][ND] of float4 {hi_v, hi_v+1, lo_v, lo_v+1}.  (In 3D the odd variable
// count and the larger tiles cost more registers than the packing saves.)
template <int D, typename R> struct PackedSweeps { static constexpr bool value = false; };
template <> struct PackedSweeps<2, df64> { static constexpr bool value = true; };
template <int D, int N, typename R, int TT>
constexpr size_t vol_flux_bytes() {
  using T = Tile<D, N, TT>;
  using C = typename TraceCompute<R>::C;
  const size_t f = PackedSweeps<D, R>::value ? sizeof(float4) * T::EPB * D * ((T::NV + 1) / 2) * T::ND
                                             : sizeof(R) * T::EPB * sf_stride<D, N, R>();
  const size_t x = sizeof(C) * T::EPB * sx_stride<D, N, C>();  // reused for the next input
  return f > x ? f : x;
}

// Shared memory of the volume kernel: the pointwise fluxes of the tile, then (kStage) the
// per-thread staging slots of the RK operands (FP64 solution; stage register in the
// operator's storage type), then (kFaces) the numerical fluxes on every face of every
// element of the tile, [EPB][D][side][NV][NF] values of R.  The trace epilogue reuses the
// flux area.
template <int D, int N, typename R, int TT, bool kStage, bool kFaces = false>
struct VolSmem {
  using T = Tile<D, N, TT>;
  static constexpr size_t FLUX = vol_flux_bytes<D, N, R, TT>();
  static constexpr size_t W_OFF = (FLUX + 15) / 16 * 16;
  static constexpr size_t Q_OFF = W_OFF + sizeof(double) * T::NV * T::THREADS;
  static constexpr size_t STAGED =
      kStage ? Q_OFF + sizeof(typename Arith<R>::S) * T::NV * T::THREADS : FLUX;
  static constexpr size_t FACE_OFF = (STAGED + 15) / 16 * 16;
  static constexpr size_t BYTES =
      kFaces ? FACE_OFF + sizeof(R) * T::EPB * 2 * D * T::NV * T::NF : STAGED;
};

// Where the volume kernel takes the numerical fluxes of its elements' faces from.
// SplitFaces: the global flux array the face-flux launch wrote (each face once).
// ElementFaces: every element evaluates the numerical flux on each of its own faces from
// the stored traces of the current stage input (each interior face is then evaluated by
// both of its elements, with the same arguments and code, hence the same bits; ring
// stores come from the face's low element only).  The next stage's traces then go to a
// second trace buffer, since neighbouring blocks still read the current ones.
struct SplitFaces {};
struct ElementFaces {
  const FluxArgs& f;  // face rules of the stage (ring, subdomain slots, AT weights)
  const void* tr;     // traces of the current stage input [d][side][v][e][j]
  int* err;           // set to 2 when a wait for the tile's bulk copies gave up
};

// The FP32 and FP32-pair forms wait on memory more than on their pipes: they stage their
// stage input, solution and 2N register through shared memory with asynchronous copies
// issued at the start, so the reads of the RK update are in flight during the volume work
// instead of after it (512^2 p=4: FP32 210 -> 187 us, pairs 8 % faster).  The FP64 form is
// bound by its FP64 pipe and keeps plain loads.
template <typename R> struct VolStages { static constexpr bool value = false; };
template <> struct VolStages<float> { static constexpr bool value = true; };
template <> struct VolStages<df64> { static constexpr bool value = true; };

// asynchronous copy of one stored value (FP32: 4 bytes, FP32 pair: 8 bytes)
__device__ __forceinline__ void cp_async_val(float* smem, const float* gmem) { cp_async4(smem, gmem); }
__device__ __forceinline__ void cp_async_val(float2* smem, const float2* gmem) { cp_async8(smem, gmem); }
__device__ __forceinline__ float from_stored(float v) { return v; }
__device__ __forceinline__ df64 from_stored(float2 v) { return df64(v.x, v.y); }

// One element tile (tile index `tile`) of the volume/update kernel.  A is read through a
// reference so the batched kernels can pass per-instance arguments kept in device memory.
template <int D, int N, typename R, int TT>
__device__ __forceinline__ void element_face_fluxes(const ElementFaces& F, const MeshArgs& m,
                                                    int e, const int* ec, int el, int node,
                                                    bool active, unsigned char* face_smem);

template <int D, int N, typename R, int TT, bool kStage = false, typename Faces = SplitFaces>
__device__ __forceinline__ void vol_body(const VolArgs& A, int tile, unsigned char* smem_raw,
                                         const Faces& faces = Faces()) {
  using T = Tile<D, N, TT>;
  using S = typename Arith<R>::S;
  constexpr bool kFaces = std::is_same<Faces, ElementFaces>::value;
  using SM = VolSmem<D, N, R, TT, kStage, kFaces>;
  // element path with staged operands in 3D: whole tiles are staged by TMA bulk copies (one
  // per variable row, issued by one thread; rows of whole 16-byte units) instead of one
  // asynchronous copy per thread and value (64^3 p=3 FP32: 850 -> 832 us per stage).  In 2D
  // p=4 the rows align only for 16-element tiles, which cost more than the copies save
  // (205 -> 253 us at 512^2).
  constexpr bool kBulk = kFaces && kStage && D == 3 && (Tile<D, N, TT>::THREADS % 4 == 0);
  uint64_t* vbar = nullptr;  // completion barriers of the two copy groups
  if constexpr (kBulk) {
    __shared__ __align__(8) uint64_t bars[2];
    vbar = bars;
  }
  constexpr int ND = T::ND, NF = T::NF, NV = T::NV, EPB = T::EPB;
  using CT = typename TraceCompute<R>::C;
  constexpr int SFS = sf_stride<D, N, R>(), SXS = sx_stride<D, N, CT>();
  static_assert(sizeof(CT) * EPB * SXS <= SM::FLUX, "the next stage input fits the flux area");
  R* sF = reinterpret_cast<R*>(smem_raw);  // [EPB][D][NV][ND], element stride SFS (packed sweeps: sF4 below)
  double* sW = reinterpret_cast<double*>(smem_raw + SM::W_OFF);  // [NV][THREADS] (kStage)
  S* sQ = reinterpret_cast<S*>(smem_raw + SM::Q_OFF);            // [NV][THREADS] (kStage)
  const int el = threadIdx.x / ND, node = threadIdx.x - el * ND;
  const int e0 = tile * EPB;
  const int ne = (int)A.m.ne;
  const int e = e0 + el;
  const bool active = e < ne;

  int ix[3] = {node % N, (node / N) % N, node / (N * N)};
  int ec[3] = {0, 0, 0};
  if (active) elem_coords(A.m, e, ec);

  // 1. stage input at this node and its pointwise fluxes
  R u[NV];
  const bool from_r = (A.mode == kMode2R && A.stage > 0);
  const S* rin = reinterpret_cast<const S*>(A.r_in);
  const int tid = threadIdx.x;
  bool bulk = false, group2 = false;  // block-uniform
  if constexpr (kStage) {
    // group 1: the stage input (FP64 solution, or the 2R register r into the q slots);
    // group 2: the solution when the input was r, and the 2N register q
    const bool upd = active && A.mode != kModeRHS;
    const bool want_q = upd && A.mode == kMode2N && A.stage > 0;
    if constexpr (kBulk) bulk = A.bulk && e0 + EPB <= ne;  // a whole tile, aligned rows
    group2 = upd && (from_r || want_q);
    if (bulk) {
      if (tid == 0) {
        mbar_init(vbar, 1);
        mbar_init(vbar + 1, 1);
      }
      __syncthreads();
      if (tid == 0) {
        constexpr unsigned RW = sizeof(double) * T::THREADS, RS = sizeof(S) * T::THREADS;
        const S* xin = reinterpret_cast<const S*>(A.x);
        mbar_expect_tx(vbar, NV * (from_r ? RS : RW));
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const int row = (v * ne + e0) * ND;
          if (from_r) bulk_load(sQ + v * T::THREADS, rin + row, RS, vbar);
          else bulk_load(sW + v * T::THREADS, A.w_in + row, RW, vbar);
        }
        if (group2) {
          mbar_expect_tx(vbar + 1, NV * ((from_r ? RW : 0u) + (want_q ? RS : 0u)));
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const int row = (v * ne + e0) * ND;
            if (from_r) bulk_load(sW + v * T::THREADS, A.w + row, RW, vbar + 1);
            if (want_q) bulk_load(sQ + v * T::THREADS, xin + row, RS, vbar + 1);
          }
        }
      }
    } else if (active) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const int idx = (v * ne + e) * ND + node;
        if (from_r) cp_async_val(sQ + v * T::THREADS + tid, rin + idx);
        else cp_async8(sW + v * T::THREADS + tid, A.w_in + idx);
      }
    }
    if (!bulk) cp_async_commit();
    if (!bulk && upd && (from_r || want_q)) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const int idx = (v * ne + e) * ND + node;
        if (from_r) cp_async8(sW + v * T::THREADS + tid, A.w + idx);
        if (want_q) cp_async_val(sQ + v * T::THREADS + tid, reinterpret_cast<const S*>(A.x) + idx);
      }
    }
    if (!bulk) cp_async_commit();
    if constexpr (kFaces) element_face_fluxes<D, N, R, TT>(faces, A.m, e, ec, el, node, active, smem_raw + SM::FACE_OFF);
    if (!bulk) {
      cp_async_wait<1>();
    } else if constexpr (kBulk) {
      // a wait that runs out flags the results as invalid and waits once more (bounded)
      // for the copies, so that none is in flight when the block's shared memory is reused
      if (!mbar_wait_bounded(vbar, 0, kWaitLimitCycles)) {
        atomicOr(faces.err, 2);
        mbar_wait_bounded(vbar, 0, kWaitLimitCycles);
      }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v)
      u[v] = !active ? R(1.0f)
                     : (from_r ? from_stored(sQ[v * T::THREADS + tid])
                               : Arith<R>::from_double(sW[v * T::THREADS + tid]));
  } else {
    if constexpr (kFaces) element_face_fluxes<D, N, R, TT>(faces, A.m, e, ec, el, node, active, smem_raw + SM::FACE_OFF);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int idx = (v * ne + e) * ND + node;
      u[v] = !active ? R(1.0f) : (from_r ? Arith<R>::load(rin + idx) : Arith<R>::from_double(A.w_in[idx]));
    }
  }
  constexpr int NP = (NV + 1) / 2;  // variable pairs of the packed sweeps
  float4* sF4 = reinterpret_cast<float4*>(smem_raw);  // [EPB][D][NP][ND] (packed sweeps)
  {
    R F[D][NV];
    euler_flux_all<D, R>(u, Arith<R>::pair(A.gm1, A.gm1f), F);
    if constexpr (PackedSweeps<D, R>::value) {
#pragma unroll
      for (int d = 0; d < D; ++d)
#pragma unroll
        for (int pr = 0; pr < NP; ++pr) {
          const R f0 = F[d][2 * pr];
          const R f1 = 2 * pr + 1 < NV ? F[d][2 * pr + 1] : R(0.0f);
          sF4[((el * D + d) * NP + pr) * ND + node] = make_float4(f0.hi, f1.hi, f0.lo, f1.lo);
        }
    } else {
#pragma unroll
      for (int d = 0; d < D; ++d)
#pragma unroll
        for (int v = 0; v < NV; ++v) sF[el * SFS + (d * NV + v) * ND + node] = F[d][v];
    }
  }
  __syncthreads();

  // 2. weak derivative (sum factorisation: one 1D contraction per direction) + face lift
  using Acc = typename Arith<R>::Acc;
  Acc acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = acc_zero(Acc());
  const S* fl = reinterpret_cast<const S*>(A.fl);
  if (active) {
    df64acc2 acc2[NP];  // packed sweeps: lane k of pair pr accumulates variable 2 pr + k
#pragma unroll
    for (int pr = 0; pr < NP; ++pr) acc2[pr] = acc2_zero();
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int stride = d == 0 ? 1 : (d == 1 ? N : N * N);
      const int base = node - ix[d] * stride;
      const double* Qd = (A.scaled ? A.tab->Qs[d] : A.tab->Q[d]) + ix[d] * N;
      const float2* Qdf = (A.scaled ? A.tab->Qsf[d] : A.tab->Qf[d]) + ix[d] * N;
      if constexpr (PackedSweeps<D, R>::value) {
#pragma unroll
        for (int a = 0; a < N; ++a) {
          const float2 q = Qdf[a];
          const float2 qh = make_float2(q.x, q.x), ql = make_float2(q.y, q.y);
          const float2 nqh = make_float2(-q.x, -q.x);
#pragma unroll
          for (int pr = 0; pr < NP; ++pr) {
            const float4 f = sF4[((el * D + d) * NP + pr) * ND + base + a * stride];
            acc2[pr] = acc2_fma(qh, ql, nqh, make_float2(f.x, f.y), make_float2(f.z, f.w), acc2[pr]);
          }
        }
      } else {
#pragma unroll
        for (int a = 0; a < N; ++a) {
          const R q = Arith<R>::tab(Qd, Qdf, a);
#pragma unroll
          for (int v = 0; v < NV; ++v)
            acc[v] = acc_fma(q, sF[el * SFS + (d * NV + v) * ND + base + a * stride], acc[v]);
        }
      }
    }
    if constexpr (PackedSweeps<D, R>::value) {
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] = acc2_lane(acc2[v / 2], v & 1);
    }
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int j = face_index<D, N>(d, ix);
      const int elo = elem_shift(A.m, e, ec, d, -1);
      const R lp = Arith<R>::tab(A.scaled ? A.tab->Lps[d] : A.tab->Lp[d],
                                 A.scaled ? A.tab->Lpsf[d] : A.tab->Lpf[d], ix[d]);
      const R lm = Arith<R>::tab(A.scaled ? A.tab->Lms[d] : A.tab->Lm[d],
                                 A.scaled ? A.tab->Lmsf[d] : A.tab->Lmf[d], ix[d]);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        R fhi, flo;
        if constexpr (kFaces) {
          const R* sFace = reinterpret_cast<const R*>(smem_raw + SM::FACE_OFF);
          fhi = sFace[(((el * D + d) * 2 + 1) * NV + v) * NF + j];
          flo = sFace[(((el * D + d) * 2 + 0) * NV + v) * NF + j];
        } else {
          fhi = Arith<R>::load(fl + ((d * NV + v) * ne + e) * NF + j);
          flo = Arith<R>::load(fl + ((d * NV + v) * ne + elo) * NF + j);
        }
        acc[v] = acc_fma(lm, flo, acc[v]);
        acc[v] = acc_fma(-lp, fhi, acc[v]);
      }
    }
  }

  // 3. Runge-Kutta update; xnext = input of the next stage
  using C = typename TraceCompute<R>::C;
  C xnext[NV];
  if constexpr (kStage) {
    if (!bulk) {
      cp_async_wait<0>();
    } else if constexpr (kBulk) {
      if (group2 && !mbar_wait_bounded(vbar + 1, 0, kWaitLimitCycles)) {
        atomicOr(faces.err, 2);
        mbar_wait_bounded(vbar + 1, 0, kWaitLimitCycles);
      }
    }
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int idx = (v * ne + e) * ND + node;
    double xd = 0.0;
    R xr = R(0.0f);
    if (active) {
      if constexpr (kStage) {
        // from_r (2R, stage > 0) the q slots hold r, which the 2R update does not read
        xr = Update<R>::apply(A, idx, acc_result(acc[v]), u[v], xd, A.mode != kModeRHS,
                              sW[v * T::THREADS + tid], from_stored(sQ[v * T::THREADS + tid]));
      } else {
        xr = Update<R>::apply(A, idx, acc_result(acc[v]), u[v], xd);
      }
    }
    xnext[v] = trace_value<C, R>(xd, xr);
  }

  // 4. traces of the next stage input
  if (A.write_traces) {
    __syncthreads();
    C* sX = reinterpret_cast<C*>(smem_raw);  // reuse: [EPB][NV][ND], element stride SXS
#pragma unroll
    for (int v = 0; v < NV; ++v) sX[el * SXS + v * ND + node] = xnext[v];
    __syncthreads();
    write_traces<D, N, R, TT, C, SXS>(A.m, A.tab, sX, e0, reinterpret_cast<S*>(A.tr));
  }
}

// Register budget of the single-instance volume kernel (an explicit budget also keeps the
// compiler from trading occupancy for registers).  The FP32 form is latency-bound and
// wants every warp slot.
template <int D, int N, typename R> struct VolKernelRegs {
  static constexpr int value = (D == 2 && (N == 2 || N == 8)) ? 64 : 56;  // no spills (ptxas)
};
template <int D, int N> struct VolKernelRegs<D, N, double> {
  static constexpr int value = D == 2 ? ((N == 3 || N == 8) ? 48 : 40) : 56;  // no spills (ptxas)
};
template <int D, int N> struct VolKernelRegs<D, N, float> {
  static constexpr int value = (D == 2 && N != 3 && N != 4 && N != 6) ? 32 : 40;  // no spills (ptxas, sm_103a)
};

template <int D, int N, typename R, int TT = 128>
__global__ void __launch_bounds__(Tile<D, N, TT>::THREADS,
                                  min_blocks_for(VolKernelRegs<D, N, R>::value,
                                                 Tile<D, N, TT>::THREADS))
vol_kernel(const VolArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  vol_body<D, N, R, TT, VolStages<R>::value>(A, blockIdx.x, smem_raw);
}

// Random-delay draw (same definition as the host schedule).
__device__ __forceinline__ uint64_t splitmix64_dev(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Numerical flux (twice Eq. 8) on face (d, e) -- between element e and its +d neighbour --
// at face node j, from e's trace wm on its +d side and the neighbour's trace wp on its -d
// side.  slot >= 0 marks a face between subdomains (the delayed / AT rules of Algorithms 2-3,
// Eq. 13-14, against the ring of stored levels; stores into the ring at stage 0 of a
// storing step when `owner`).  Shared by the face-flux kernel and the fused kernel, so both
// produce the same bits for the same face.
template <int D, int N, typename R>
__device__ __forceinline__ void face_flux(const FluxArgs& A, int d, int slot, int j,
                                          const R (&wm)[D + 2], const R (&wp)[D + 2], bool owner,
                                          R (&f)[D + 2]) {
  using S = typename Arith<R>::S;
  constexpr int NF = IPow<N, D - 1>::value, NV = D + 2;
  const R gamma = Arith<R>::pair(A.gamma, A.gammaf), gm1 = Arith<R>::pair(A.gm1, A.gm1f);
  if (slot < 0) {
    llf_flux<D, R>(wm, wp, d, gamma, gm1, f);
    return;
  }
  S* ring = reinterpret_cast<S*>(A.ring);
  const bool traces = (A.flux_kind >= 3);  // AT on traces, and the learned mode
  const int npe = (int)A.npe;
  const int lvl_stride = (traces ? 2 : 1) * NV * npe * NF;
  int kt = A.uniform_delay;
  if (A.random) {
    const int iface = A.pe_iface[slot];
    const uint64_t ctr = (uint64_t)A.step * (uint64_t)A.n_iface + (uint64_t)iface;
    kt = (int)(splitmix64_dev(A.seed ^ ctr) % (uint64_t)(A.dmax + 1));
    const int64_t need = (A.nterms == 1) ? kt : kt + A.np;
    if (A.step - need < 0) kt = 0;
  }
  if (A.store && traces && owner) {
    S* dst = ring + A.head * lvl_stride;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      Arith<R>::store(dst + (v * npe + slot) * NF + j, wm[v]);
      Arith<R>::store(dst + ((NV + v) * npe + slot) * NF + j, wp[v]);
    }
  }
  if (kt == 0 || (A.store && !traces)) {
    R fr[NV];
    llf_flux<D, R>(wm, wp, d, gamma, gm1, fr);
    if (A.store && !traces && owner) {
      S* dst = ring + A.head * lvl_stride;
#pragma unroll
      for (int v = 0; v < NV; ++v) Arith<R>::store(dst + (v * npe + slot) * NF + j, fr[v]);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) f[v] = fr[v];
  }
  if (kt != 0) {
    const int off = A.random ? kt : 0;
    using Acc = typename Arith<R>::Acc;
    Acc am[NV], ap[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) { am[v] = acc_zero(Acc()); ap[v] = acc_zero(Acc()); }
    for (int l = 0; l < A.nterms; ++l) {
      int lvl = (A.head - off - l) % A.depth;
      if (lvl < 0) lvl += A.depth;
      const R c = Arith<R>::pair(A.ctab[kt][l], A.ctabf[kt][l]);
      const S* src = ring + lvl * lvl_stride;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        am[v] = acc_fma(c, Arith<R>::load(src + (v * npe + slot) * NF + j), am[v]);
        if (traces) ap[v] = acc_fma(c, Arith<R>::load(src + ((NV + v) * npe + slot) * NF + j), ap[v]);
      }
    }
    if (traces) {
      R em[NV], ep[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) { em[v] = acc_result(am[v]); ep[v] = acc_result(ap[v]); }
      llf_flux<D, R>(em, ep, d, gamma, gm1, f);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) f[v] = acc_result(am[v]);
    }
  }
}

// One block of face-flux threads: block bx over (element, face node) of direction d.
template <int D, int N, typename R>
__device__ __forceinline__ void flux_body(const FluxArgs& A, int bx, int d) {
  using S = typename Arith<R>::S;
  constexpr int NF = IPow<N, D - 1>::value, NV = D + 2;
  const int ne = (int)A.m.ne;
  const int g = bx * blockDim.x + threadIdx.x;
  if (g >= ne * NF) return;
  const int e = g / NF;
  const int j = g - e * NF;
  int ec[3];
  elem_coords(A.m, e, ec);
  const int ehi = elem_shift(A.m, e, ec, d, +1);
  const S* tr = reinterpret_cast<const S*>(A.tr);
  R wm[NV], wp[NV], f[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    wm[v] = Arith<R>::load(tr + (((d * 2 + 1) * NV + v) * ne + e) * NF + j);
    wp[v] = Arith<R>::load(tr + (((d * 2 + 0) * NV + v) * ne + ehi) * NF + j);
  }
  const int slot = A.pe_mode ? A.pe_slot[d * ne + e] : -1;
  face_flux<D, N, R>(A, d, slot, j, wm, wp, true, f);
  S* fl = reinterpret_cast<S*>(A.fl);
#pragma unroll
  for (int v = 0; v < NV; ++v) Arith<R>::store(fl + ((d * NV + v) * ne + e) * NF + j, f[v]);
}

// Numerical fluxes on the 2D faces of element e (tile slot el) into shared memory
// [el][d][side][v][j]: the thread of node `node` takes the face nodes node, node + ND, ...
// Face (d, lo) lies between element lo and its +d neighbour hi; its flux is evaluated from
// lo's +d trace and hi's -d trace exactly as the face-flux launch evaluates it, so both
// elements of the face obtain the same value.
template <int D, int N, typename R, int TT>
__device__ __forceinline__ void element_face_fluxes(const ElementFaces& F, const MeshArgs& m,
                                                    int e, const int* ec, int el, int node,
                                                    bool active, unsigned char* face_smem) {
  using T = Tile<D, N, TT>;
  using S = typename Arith<R>::S;
  constexpr int ND = T::ND, NF = T::NF, NV = T::NV;
  if (!active) return;
  const int ne = (int)m.ne;
  const S* tr = reinterpret_cast<const S*>(F.tr);
  R* sFace = reinterpret_cast<R*>(face_smem) + el * (2 * D * NV * NF);
  for (int q = node; q < 2 * D * NF; q += ND) {
    const int ds = q / NF, j = q - ds * NF;  // ds = 2 d + side (side 1: the +d face)
    const int d = ds >> 1, side = ds & 1;
    const int nb = elem_shift(m, e, ec, d, side ? 1 : -1);
    const int lo = side ? e : nb, hi = side ? nb : e;
    R wm[NV], wp[NV], f[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      wm[v] = Arith<R>::load(tr + (((d * 2 + 1) * NV + v) * ne + lo) * NF + j);
      wp[v] = Arith<R>::load(tr + (((d * 2 + 0) * NV + v) * ne + hi) * NF + j);
    }
    const int slot = F.f.pe_mode ? F.f.pe_slot[d * ne + lo] : -1;
    face_flux<D, N, R>(F.f, d, slot, j, wm, wp, side == 1, f);
#pragma unroll
    for (int v = 0; v < NV; ++v) sFace[(ds * NV + v) * NF + j] = f[v];
  }
}

// One launch per RK stage without the face-flux launch: the volume kernel with every
// element evaluating the numerical fluxes on its own faces (ElementFaces).  Register
// budgets: no spills (ptxas sm_103a); the FP32 form measured best at 48 (40 spilled and
// lost 8 %, 56 gained nothing).
template <int D, int N, typename R> struct VolFacesRegs { static constexpr int value = D == 2 ? 64 : 80; };
template <int D, int N> struct VolFacesRegs<D, N, float> { static constexpr int value = 48; };
template <int D, int N> struct VolFacesRegs<D, N, double> { static constexpr int value = D == 2 ? 72 : 80; };

template <int D, int N, typename R, int TT = 128>
__global__ void __launch_bounds__(Tile<D, N, TT>::THREADS,
                                  min_blocks_for(VolFacesRegs<D, N, R>::value,
                                                 Tile<D, N, TT>::THREADS))
vol_faces_kernel(const FusedArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  vol_body<D, N, R, TT, VolStages<R>::value, ElementFaces>(A.v, blockIdx.x, smem_raw,
                                                           ElementFaces{A.f, A.tr_in, A.err});
}

// Register budget of the face-flux kernel (blocks of 256 threads; no spills, ptxas sm_103a).
template <int D, typename R> struct FluxKernelRegs { static constexpr int value = D == 2 ? 64 : 72; };
template <int D> struct FluxKernelRegs<D, float> { static constexpr int value = 48; };
template <int D> struct FluxKernelRegs<D, df64> { static constexpr int value = 64; };

// grid: x over (element, face node) of one direction, y = direction d
template <int D, int N, typename R>
__global__ void __launch_bounds__(256, min_blocks_for(FluxKernelRegs<D, R>::value, 256))
flux_kernel(const FluxArgs A) {
  flux_body<D, N, R>(A, blockIdx.x, blockIdx.y);
}

// ------------------------------------------------------------------------------------
// Launch helpers instantiated per arithmetic in the kernel translation units.
// ------------------------------------------------------------------------------------
template <int D, int N, typename R>
cudaError_t launch_trace_t(const TraceArgs& a, cudaStream_t s) {
  using T = Tile<D, N>;
  const int64_t blocks = (a.m.ne + T::EPB - 1) / T::EPB;
  const size_t smem = sizeof(R) * T::EPB * T::NV * T::ND;
  trace_kernel<D, N, R><<<(unsigned)blocks, T::THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <int D, int N, typename R>
cudaError_t launch_vol_t(const VolArgs& a, cudaStream_t s) {
  using T = Tile<D, N>;
  const int64_t blocks = (a.m.ne + T::EPB - 1) / T::EPB;
  const size_t smem = VolSmem<D, N, R, 128, VolStages<R>::value>::BYTES;
  if (smem > 48 * 1024) {
    cudaError_t err = cudaFuncSetAttribute(vol_kernel<D, N, R>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
  }
  vol_kernel<D, N, R><<<(unsigned)blocks, T::THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <int D, int N, typename R>
cudaError_t launch_vol_faces_t(const FusedArgs& a, cudaStream_t s) {
  constexpr int TT = 128;  // tiles of about 128 threads, as on the split path
  using T = Tile<D, N, TT>;
  const int64_t blocks = (a.v.m.ne + T::EPB - 1) / T::EPB;
  const size_t smem = VolSmem<D, N, R, TT, VolStages<R>::value, true>::BYTES;
  if (smem > 48 * 1024) {
    cudaError_t err = cudaFuncSetAttribute(vol_faces_kernel<D, N, R, TT>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
  }
  vol_faces_kernel<D, N, R, TT><<<(unsigned)blocks, T::THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <int D, int N, typename R>
cudaError_t launch_flux_t(const FluxArgs& a, cudaStream_t s) {
  constexpr int NF = IPow<N, D - 1>::value;
  const int64_t per_dir = a.m.ne * NF;
  dim3 grid((unsigned)((per_dir + 255) / 256), D);
  flux_kernel<D, N, R><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

// Dispatch over (dim, N) for one arithmetic R.
template <typename R>
struct Dispatch {
  static cudaError_t run_trace(int dim, int N, const TraceArgs& a, cudaStream_t s);
  static cudaError_t run_flux(int dim, int N, const FluxArgs& a, cudaStream_t s);
  static cudaError_t run_vol(int dim, int N, const VolArgs& a, cudaStream_t s);
  static cudaError_t run_vol_faces(int dim, int N, const FusedArgs& a, cudaStream_t s);
};

#define ADG_DISPATCH_BODY(FN, ARGS)                                  \
  if (dim == 2) {                                                    \
    switch (N) {                                                     \
      case 2: return FN<2, 2, R>(ARGS, s);                           \
      case 3: return FN<2, 3, R>(ARGS, s);                           \
      case 4: return FN<2, 4, R>(ARGS, s);                           \
      case 5: return FN<2, 5, R>(ARGS, s);                           \
      case 6: return FN<2, 6, R>(ARGS, s);                           \
      case 7: return FN<2, 7, R>(ARGS, s);                           \
      case 8: return FN<2, 8, R>(ARGS, s);                           \
    }                                                                \
  } else if (dim == 3) {                                             \
    switch (N) {                                                     \
      case 2: return FN<3, 2, R>(ARGS, s);                           \
      case 3: return FN<3, 3, R>(ARGS, s);                           \
      case 4: return FN<3, 4, R>(ARGS, s);                           \
      case 5: return FN<3, 5, R>(ARGS, s);                           \
      case 6: return FN<3, 6, R>(ARGS, s);                           \
    }                                                                \
  }                                                                  \
  return cudaErrorInvalidValue;

template <typename R>
cudaError_t Dispatch<R>::run_trace(int dim, int N, const TraceArgs& a, cudaStream_t s) {
  ADG_DISPATCH_BODY(launch_trace_t, a)
}
template <typename R>
cudaError_t Dispatch<R>::run_flux(int dim, int N, const FluxArgs& a, cudaStream_t s) {
  ADG_DISPATCH_BODY(launch_flux_t, a)
}
template <typename R>
cudaError_t Dispatch<R>::run_vol(int dim, int N, const VolArgs& a, cudaStream_t s) {
  ADG_DISPATCH_BODY(launch_vol_t, a)
}
template <typename R>
cudaError_t Dispatch<R>::run_vol_faces(int dim, int N, const FusedArgs& a, cudaStream_t s) {
  ADG_DISPATCH_BODY(launch_vol_faces_t, a)
}

}  // namespace adg
