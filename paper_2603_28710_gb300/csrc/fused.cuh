// Fused per-stage kernel of the ADG operator: one launch per Runge-Kutta stage does, for
// every tile of TX x TY (x TZ) elements, the face traces, the numerical fluxes on every face
// of the tile (including the delayed / AT rules on faces between subdomains), the pointwise
// Euler fluxes, the sum-factorised weak derivative, face lift, inverse mass and the
// low-storage RK update -- no separate face-flux launch and no global array of face fluxes.
//
// Persistent blocks walk the tiles (tile = block, block + grid, ...) through a two-slot
// pipeline: while a block works on one tile, the TMA engine already copies the next tile's
// solution w (FP64) and RK register (q or r, operator storage type) into the other slot of
// shared memory ([var][z][y][x * nodes] tensor boxes, one copy per array, completion on the
// slot's mbarrier).  Ragged tiles at the mesh edge read zeros beyond it.
//   * traces of the tile's own elements are interpolated from shared memory; only faces on
//     the tile boundary need the neighbour tile's trace, which the previous stage wrote to a
//     global trace buffer (double-buffered across stages: read one, write the other);
//   * at the end of a tile the block writes w and q, and the traces of the next stage input
//     on the tile's boundary faces.
// A face between two tiles is evaluated by both, from the same two traces by the same code
// (face_flux), so both see the same bits and the face terms cancel exactly in the
// conservation sums; its subdomain ring entry is stored by the tile holding the face's low
// element.  The trace of an element's own face is computed from the stage input exactly as
// the previous stage computed it for the neighbour (same values, same interpolation code).
// In the FP32 operator the sweeps and the lift advance two variables per packed FP32x2
// instruction.
//
// Every wait on an mbarrier has a time limit (about one second of SM clock); a block that
// gives up sets an error code in device memory, waits (again bounded) for the copies it
// started, and returns.
#pragma once
#include <cuda.h>

#include <algorithm>

#include "kernels.cuh"

namespace adg {

// Tile shapes (elements per direction) of the fused kernel: whole elements, a few hundred
// threads (one per node), and TX * nodes a multiple of four so that a tile row of FP32
// values is a whole number of 16-byte units (a TMA requirement).
template <int D, int N> struct FusedTile;
template <> struct FusedTile<2, 2> { static constexpr int TX = 8, TY = 8, TZ = 1; };
template <> struct FusedTile<2, 3> { static constexpr int TX = 4, TY = 8, TZ = 1; };
template <> struct FusedTile<2, 4> { static constexpr int TX = 4, TY = 4, TZ = 1; };
template <> struct FusedTile<2, 5> { static constexpr int TX = 4, TY = 2, TZ = 1; };
template <> struct FusedTile<2, 6> { static constexpr int TX = 4, TY = 2, TZ = 1; };
template <> struct FusedTile<2, 7> { static constexpr int TX = 4, TY = 2, TZ = 1; };
template <> struct FusedTile<2, 8> { static constexpr int TX = 2, TY = 2, TZ = 1; };
template <> struct FusedTile<3, 2> { static constexpr int TX = 4, TY = 4, TZ = 2; };
template <> struct FusedTile<3, 3> { static constexpr int TX = 4, TY = 2, TZ = 2; };
template <> struct FusedTile<3, 4> { static constexpr int TX = 2, TY = 2, TZ = 2; };
template <> struct FusedTile<3, 5> { static constexpr int TX = 4, TY = 1, TZ = 1; };
template <> struct FusedTile<3, 6> { static constexpr int TX = 1, TY = 2, TZ = 1; };

template <int D, int N>
struct FT {
  using T = FusedTile<D, N>;
  static constexpr int TX = T::TX, TY = T::TY, TZ = D == 3 ? T::TZ : 1;
  static constexpr int ND = IPow<N, D>::value, NF = ND / N, NV = D + 2;
  static constexpr int EPB = TX * TY * TZ;
  static constexpr int THREADS = EPB * ND;
  // faces of the tile per direction: (T_d + 1) planes times the transverse elements
  static constexpr int F0 = (TX + 1) * TY * TZ;
  static constexpr int F1 = TX * (TY + 1) * TZ;
  static constexpr int F2 = D == 3 ? TX * TY * (TZ + 1) : 0;
  static constexpr int NFACE = F0 + F1 + F2;
  // boundary faces (both sides) per direction
  static constexpr int B0 = 2 * TY * TZ, B1 = 2 * TX * TZ, B2 = D == 3 ? 2 * TX * TY : 0;
  static constexpr int NBND = B0 + B1 + B2;
};

// Compute type of the traces (as in the two-kernel path): FP64 for the FP32-pair operator.
template <typename R>
using TraceC = typename TraceCompute<R>::C;

constexpr size_t align128(size_t b) { return (b + 127) / 128 * 128; }

// Packed FP32x2 sweeps for the FP32 operator: pointwise and face fluxes of variable pairs
// as float2 (the last pair padded in 3D).
template <typename R> struct FusedPacked { static constexpr bool value = false; };
template <> struct FusedPacked<float> { static constexpr bool value = true; };

// Shared memory of the fused kernel (byte offsets, 128-byte aligned regions):
//   two staging slots {W: double [NV][EPB*ND], X: S [NV][EPB*ND]}, filled by TMA;
//   BIG: first U (stage input in the trace compute type, where it is not an alias of a
//        staging array) and T (own traces [EPB][2D][NV][NF]), then the pointwise fluxes
//        ([EPB][D][NV][ND], packed: float2 [EPB][D][NP][ND]), then the next stage input;
//   FF:  face fluxes [NFACE][NV][NF] (packed: float2 [NFACE][NP][NF]);
//   two mbarriers.
template <int D, int N, typename R>
struct FusedSmem {
  using F = FT<D, N>;
  using S = typename Arith<R>::S;
  using C = TraceC<R>;
  static constexpr bool PK = FusedPacked<R>::value;
  static constexpr int NP = (F::NV + 1) / 2;
  static constexpr size_t ROWB = (size_t)F::EPB * F::ND;
  static constexpr size_t WB = align128(sizeof(double) * F::NV * ROWB);
  static constexpr size_t XB = align128(sizeof(S) * F::NV * ROWB);
  static constexpr size_t SLOT = WB + XB;
  static constexpr size_t UB = align128(sizeof(C) * F::NV * ROWB);
  static constexpr size_t TB = align128(sizeof(C) * F::EPB * 2 * D * F::NV * F::NF);
  static constexpr size_t FB = PK ? align128(sizeof(float2) * F::EPB * D * NP * F::ND)
                                  : align128(sizeof(R) * F::EPB * D * F::NV * F::ND);
  static constexpr size_t BIGB = UB + TB > FB ? UB + TB : FB;  // >= UB (next stage input)
  static constexpr size_t FFB = PK ? align128(sizeof(float2) * F::NFACE * NP * F::NF)
                                   : align128(sizeof(R) * F::NFACE * F::NV * F::NF);
  static constexpr size_t BIG = 2 * SLOT;
  static constexpr size_t FF = BIG + BIGB;
  static constexpr size_t BAR = FF + FFB;
  static constexpr size_t BYTES = BAR + 16;
};

// ---- TMA tensor copies (PTX; the mbarrier helpers are in kernels.cuh) -------------
// 3D / 4D tiled tensor copy global -> shared, completion counted on the mbarrier
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            int c3, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

// value of a stored trace / RK register entry in the operator arithmetic
__device__ __forceinline__ double stored_to(double v, double) { return v; }
__device__ __forceinline__ float stored_to(float v, float) { return v; }
__device__ __forceinline__ df64 stored_to(float2 v, df64) { return df64(v.x, v.y); }
// operator value of a trace held in the trace compute type C
__device__ __forceinline__ double trace_to_r(double c, double) { return c; }
__device__ __forceinline__ float trace_to_r(float c, float) { return c; }
__device__ __forceinline__ df64 trace_to_r(double c, df64) { return d2df_int(c); }

// interpolation of a face trace from the values of a line of N nodes (stride in shared
// memory) with weights t[]: the same order of operations as write_traces
template <int N, typename C>
__device__ __forceinline__ C interp_line(const C (&t)[N], const C* x, int stride) {
  typename Arith<C>::Acc acc = acc_zero(typename Arith<C>::Acc());
#pragma unroll
  for (int a = 0; a < N; ++a) acc = acc_fma(t[a], x[a * stride], acc);
  return acc_result(acc);
}

// Register budget of the fused kernel (no spills, ptxas sm_103a).
template <int D, int N, typename R> struct FusedRegs { static constexpr int value = 64; };
template <int D, int N> struct FusedRegs<D, N, float> { static constexpr int value = D == 2 ? 56 : 64; };

template <int D, int N, typename R>
__global__ void __launch_bounds__(FT<D, N>::THREADS,
                                  min_blocks_for(FusedRegs<D, N, R>::value, FT<D, N>::THREADS))
fused_kernel(const __grid_constant__ FusedArgs A, const __grid_constant__ CUtensorMap tm_w,
             const __grid_constant__ CUtensorMap tm_x) {
  using F = FT<D, N>;
  using S = typename Arith<R>::S;
  using C = TraceC<R>;
  using SM = FusedSmem<D, N, R>;
  constexpr bool PK = SM::PK;
  constexpr int NP = SM::NP;
  constexpr int ND = F::ND, NF = F::NF, NV = F::NV, EPB = F::EPB, THREADS = F::THREADS;
  constexpr int TX = F::TX, TY = F::TY, TZ = F::TZ;
  constexpr int ROW = EPB * ND;  // values of one variable in the tile
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* big = smem + SM::BIG;
  C* sUm = reinterpret_cast<C*>(big);                 // materialised stage input (B0-B1)
  C* sT = reinterpret_cast<C*>(big + SM::UB);         // own traces (B1-C)
  R* sF = reinterpret_cast<R*>(big);                  // pointwise fluxes (B2-D1)
  float2* sF2 = reinterpret_cast<float2*>(big);       // packed pointwise fluxes
  C* sN = reinterpret_cast<C*>(big);                  // next stage input (D2-E)
  R* sFF = reinterpret_cast<R*>(smem + SM::FF);
  float2* sFF2 = reinterpret_cast<float2*>(smem + SM::FF);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SM::BAR);

  const VolArgs& V = A.v;
  const MeshArgs& m = V.m;
  const int ne = (int)m.ne;
  const int tid = threadIdx.x;
  const int ntiles = A.ntile[0] * A.ntile[1] * A.ntile[2];
  const bool two_n = V.mode == kMode2N;
  const bool from_x = !two_n && V.stage > 0;   // 2R stage > 0: the stage input is r
  const bool load_x = V.stage > 0;             // q (2N) or r (2R) is needed
  const unsigned tx_bytes =
      (unsigned)(sizeof(double) * NV * ROW + (load_x ? sizeof(S) * NV * ROW : 0));
  const int n01 = m.n[0] * m.n[1];

  const int nt0 = A.ntile[0], nt01 = A.ntile[0] * A.ntile[1];
  const int mn0 = m.n[0], mn1 = m.n[1], mn2 = m.n[2];
  // thread 0: copies of `tile` into slot b (TMA) -- the slot's previous contents were
  // last read before the barrier that precedes this call
  auto issue = [&](int tile, int b) {
    const int c0 = (tile % nt0) * TX * ND, c1 = ((tile / nt0) % A.ntile[1]) * TY;
    const int c2 = (tile / nt01) * TZ;
    double* dw = reinterpret_cast<double*>(smem + b * SM::SLOT);
    S* dx = reinterpret_cast<S*>(smem + b * SM::SLOT + SM::WB);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar + b, tx_bytes);
    if constexpr (D == 2) {
      tma_load_3d(dw, &tm_w, c0, c1, 0, bar + b);
      if (load_x) tma_load_3d(dx, &tm_x, c0, c1, 0, bar + b);
    } else {
      tma_load_4d(dw, &tm_w, c0, c1, c2, 0, bar + b);
      if (load_x) tma_load_4d(dx, &tm_x, c0, c1, c2, 0, bar + b);
    }
  };

  if (A.tma) {
    if (tid == 0) {
      mbar_init(bar, 1);
      mbar_init(bar + 1, 1);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0 && (int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
  }

  // this thread's node within a tile
  const int el = tid / ND, node = tid - el * ND;
  const int ex = el % TX, ey = (el / TX) % TY, ez = el / (TX * TY);
  const int ix[3] = {node % N, (node / N) % N, node / (N * N)};

  int it = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int b = it & 1;
    double* sW = reinterpret_cast<double*>(smem + b * SM::SLOT);
    S* sX = reinterpret_cast<S*>(smem + b * SM::SLOT + SM::WB);
    const int o0 = (tile % nt0) * TX, o1 = ((tile / nt0) % A.ntile[1]) * TY, o2 = (tile / nt01) * TZ;
    const int E0 = min(TX, mn0 - o0), E1 = min(TY, mn1 - o1), E2 = min(TZ, mn2 - o2);
    auto gel = [=](int x, int y, int z) { return (o0 + x) + mn0 * (o1 + y) + n01 * (o2 + z); };

    // ---- A. the tile's data: wait for its copies and start those of the next tile -------
    if (A.tma) {
      if (tid == 0 && tile + (int)gridDim.x < ntiles) issue(tile + gridDim.x, b ^ 1);
      if (!mbar_wait_bounded(bar + b, (it >> 1) & 1, kWaitLimitCycles)) {
        atomicOr(A.err, 1);
        mbar_wait_bounded(bar + b, (it >> 1) & 1, kWaitLimitCycles);
        mbar_wait_bounded(bar + (b ^ 1), ((it + 1) >> 1) & 1, kWaitLimitCycles);
        return;
      }
    } else {
      const S* xg = reinterpret_cast<const S*>(V.x);
      for (int i = tid; i < NV * ROW; i += THREADS) {
        const int v = i / ROW, r = i - v * ROW;
        const int te = r / ND, nd = r - te * ND;
        const int x = te % TX, y = (te / TX) % TY, z = te / (TX * TY);
        const bool in = x < E0 && y < E1 && z < E2;
        const int idx = in ? (v * ne + gel(x, y, z)) * ND + nd : 0;
        sW[i] = in ? V.w[idx] : 0.0;
        if (load_x) sX[i] = in ? xg[idx] : S();
      }
      __syncthreads();
    }

    const bool active = ex < E0 && ey < E1 && ez < E2;
    const int e = active ? gel(ex, ey, ez) : 0;

    // ---- B0. stage input: operator value u (registers), trace-compute copy U ---------------
    const C* sUin;
    if constexpr (std::is_same<C, double>::value) {
      sUin = from_x ? reinterpret_cast<const C*>(std::is_same<S, double>::value ? (const void*)sX
                                                                                  : (const void*)sUm)
                    : reinterpret_cast<const C*>(sW);
    } else {
      sUin = from_x ? reinterpret_cast<const C*>(sX) : sUm;
    }
    R u[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int i = v * ROW + tid;
      if (!active) {
        u[v] = (v == 0 || v == NV - 1) ? R(1.0f) : R(0.0f);
      } else if (from_x) {
        u[v] = stored_to(sX[i], R());
      } else {
        u[v] = Arith<R>::from_double(sW[i]);
      }
      if constexpr (std::is_same<C, float>::value) {
        if (!from_x) sUm[i] = active ? Arith<float>::from_double(sW[i]) : 0.0f;
      } else if constexpr (!std::is_same<S, double>::value) {
        if (from_x) sUm[i] = active ? Arith<R>::to_double(u[v]) : 0.0;
      }
    }
    __syncthreads();

    // ---- B1. traces of the tile's elements on all their faces (from U) -------------------
    {
      constexpr int CT = 2 * D * NV * NF;  // (direction, side, variable, face node) combinations
      for (int g = tid; g < CT * EPB; g += THREADS) {
        const int c = g % CT, te = g / CT;
        const int j = c % NF, rest = c / NF;  // rest = (d*2 + side)*NV + v
        const int v = rest % NV, ds = rest / NV;
        const int d = ds >> 1, side = ds & 1;
        const int base = line_base<D, N>(d, j);
        const int stride = d == 0 ? 1 : (d == 1 ? N : N * N);
        const double* tw = side ? V.tab->Tp : V.tab->Tm;
        const float2* twf = side ? V.tab->Tpf : V.tab->Tmf;
        C t[N];
#pragma unroll
        for (int a = 0; a < N; ++a) t[a] = Arith<C>::tab(tw, twf, a);
        sT[((te * 2 * D + ds) * NV + v) * NF + j] = interp_line<N, C>(t, sUin + v * ROW + te * ND + base, stride);
      }
    }
    __syncthreads();

    // ---- C. numerical fluxes on every face of the tile ------------------------------------
    {
      const S* trg = reinterpret_cast<const S*>(A.tr_in);
      for (int g = tid; g < F::NFACE * NF; g += THREADS) {
        const int fid = g / NF, j = g - fid * NF;
        int d, c, a0, a1;  // direction, plane, transverse tile coordinates
        int f = fid;
        if (f < F::F0) {
          d = 0; c = f % (TX + 1); a0 = (f / (TX + 1)) % TY; a1 = f / ((TX + 1) * TY);
        } else if (f - F::F0 < F::F1) {
          f -= F::F0; d = 1; a0 = f % TX; c = (f / TX) % (TY + 1); a1 = f / (TX * (TY + 1));
        } else {
          f -= F::F0 + F::F1; d = 2; a0 = f % TX; a1 = (f / TX) % TY; c = f / (TX * TY);
        }
        int xl, yl, zl, xh, yh, zh, Ed;
        if (d == 0) { xl = c - 1; yl = a0; zl = a1; xh = c; yh = a0; zh = a1; Ed = E0; }
        else if (d == 1) { xl = a0; yl = c - 1; zl = a1; xh = a0; yh = c; zh = a1; Ed = E1; }
        else { xl = a0; yl = a1; zl = c - 1; xh = a0; yh = a1; zh = c; Ed = E2; }
        const bool trans_ok = (d == 0) ? (a0 < E1 && a1 < E2)
                                       : (d == 1 ? (a0 < E0 && a1 < E2) : (a0 < E0 && a1 < E1));
        if (!trans_ok || c > Ed) continue;
        R wm[NV], wp[NV], fl[NV];
        int elow;
        if (c >= 1) {
          const int te = (zl * TY + yl) * TX + xl;
          elow = gel(xl, yl, zl);
#pragma unroll
          for (int v = 0; v < NV; ++v) wm[v] = trace_to_r(sT[((te * 2 * D + 2 * d + 1) * NV + v) * NF + j], R());
        } else {
          // low element in the neighbouring tile (periodic): its +d trace from the buffer
          const int eh = gel(xh, yh, zh);
          int ec[3];
          elem_coords(m, eh, ec);
          elow = elem_shift(m, eh, ec, d, -1);
#pragma unroll
          for (int v = 0; v < NV; ++v)
            wm[v] = Arith<R>::load(trg + (((d * 2 + 1) * NV + v) * ne + elow) * NF + j);
        }
        if (c < Ed) {
          const int te = (zh * TY + yh) * TX + xh;
#pragma unroll
          for (int v = 0; v < NV; ++v) wp[v] = trace_to_r(sT[((te * 2 * D + 2 * d) * NV + v) * NF + j], R());
        } else {
          const int el_ = gel(xl, yl, zl);
          int ec[3];
          elem_coords(m, el_, ec);
          const int ehi = elem_shift(m, el_, ec, d, +1);
#pragma unroll
          for (int v = 0; v < NV; ++v)
            wp[v] = Arith<R>::load(trg + (((d * 2 + 0) * NV + v) * ne + ehi) * NF + j);
        }
        const int slot = A.f.pe_mode ? A.f.pe_slot[d * ne + elow] : -1;
        face_flux<D, N, R>(A.f, d, slot, j, wm, wp, c >= 1, fl);
        if constexpr (PK) {
#pragma unroll
          for (int pr = 0; pr < NP; ++pr)
            sFF2[(fid * NP + pr) * NF + j] =
                make_float2(fl[2 * pr], 2 * pr + 1 < NV ? fl[2 * pr + 1] : 0.0f);
        } else {
#pragma unroll
          for (int v = 0; v < NV; ++v) sFF[(fid * NV + v) * NF + j] = fl[v];
        }
      }
    }
    __syncthreads();

    // ---- B2. pointwise Euler fluxes (over U and T, both no longer needed) -----------------
    {
      R Fp[D][NV];
      euler_flux_all<D, R>(u, Arith<R>::pair(V.gm1, V.gm1f), Fp);
      if constexpr (PK) {
#pragma unroll
        for (int d = 0; d < D; ++d)
#pragma unroll
          for (int pr = 0; pr < NP; ++pr)
            sF2[((el * D + d) * NP + pr) * ND + node] =
                make_float2(Fp[d][2 * pr], 2 * pr + 1 < NV ? Fp[d][2 * pr + 1] : 0.0f);
      } else {
#pragma unroll
        for (int d = 0; d < D; ++d)
#pragma unroll
          for (int v = 0; v < NV; ++v) sF[((el * D + d) * NV + v) * ND + node] = Fp[d][v];
      }
    }
    __syncthreads();

    // ---- D1. weak derivative + face lift ----------------------------------------------------
    using Acc = typename Arith<R>::Acc;
    Acc acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = acc_zero(Acc());
    if (active) {
      // faces of this element along d: low plane = its own tile coordinate, high = +1
      int flo[3], fhi[3];
      flo[0] = (ez * TY + ey) * (TX + 1) + ex;
      fhi[0] = flo[0] + 1;
      flo[1] = F::F0 + (ez * (TY + 1) + ey) * TX + ex;
      fhi[1] = flo[1] + TX;
      flo[2] = F::F0 + F::F1 + (ez * TY + ey) * TX + ex;
      fhi[2] = flo[2] + TX * TY;
      if constexpr (PK) {
        float2 a2[NP];
#pragma unroll
        for (int pr = 0; pr < NP; ++pr) a2[pr] = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const int stride = d == 0 ? 1 : (d == 1 ? N : N * N);
          const int base = node - ix[d] * stride;
          const float2* Qdf = (V.scaled ? V.tab->Qsf[d] : V.tab->Qf[d]) + ix[d] * N;
#pragma unroll
          for (int a = 0; a < N; ++a) {
            const float q = Qdf[a].x;
            const float2 q2 = make_float2(q, q);
#pragma unroll
            for (int pr = 0; pr < NP; ++pr)
              a2[pr] = __ffma2_rn(q2, sF2[((el * D + d) * NP + pr) * ND + base + a * stride], a2[pr]);
          }
        }
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const int j = face_index<D, N>(d, ix);
          const float lp = (V.scaled ? V.tab->Lpsf[d] : V.tab->Lpf[d])[ix[d]].x;
          const float lm = (V.scaled ? V.tab->Lmsf[d] : V.tab->Lmf[d])[ix[d]].x;
          const float2 lm2 = make_float2(lm, lm), nlp2 = make_float2(-lp, -lp);
#pragma unroll
          for (int pr = 0; pr < NP; ++pr) {
            a2[pr] = __ffma2_rn(lm2, sFF2[(flo[d] * NP + pr) * NF + j], a2[pr]);
            a2[pr] = __ffma2_rn(nlp2, sFF2[(fhi[d] * NP + pr) * NF + j], a2[pr]);
          }
        }
        if constexpr (std::is_same<Acc, float>::value) {
#pragma unroll
          for (int v = 0; v < NV; ++v) acc[v] = (v & 1) ? a2[v / 2].y : a2[v / 2].x;
        }
      } else {
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const int stride = d == 0 ? 1 : (d == 1 ? N : N * N);
          const int base = node - ix[d] * stride;
          const double* Qd = (V.scaled ? V.tab->Qs[d] : V.tab->Q[d]) + ix[d] * N;
          const float2* Qdf = (V.scaled ? V.tab->Qsf[d] : V.tab->Qf[d]) + ix[d] * N;
#pragma unroll
          for (int a = 0; a < N; ++a) {
            const R q = Arith<R>::tab(Qd, Qdf, a);
#pragma unroll
            for (int v = 0; v < NV; ++v)
              acc[v] = acc_fma(q, sF[((el * D + d) * NV + v) * ND + base + a * stride], acc[v]);
          }
        }
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const int j = face_index<D, N>(d, ix);
          const R lp = Arith<R>::tab(V.scaled ? V.tab->Lps[d] : V.tab->Lp[d],
                                     V.scaled ? V.tab->Lpsf[d] : V.tab->Lpf[d], ix[d]);
          const R lm = Arith<R>::tab(V.scaled ? V.tab->Lms[d] : V.tab->Lm[d],
                                     V.scaled ? V.tab->Lmsf[d] : V.tab->Lmf[d], ix[d]);
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            acc[v] = acc_fma(lm, sFF[(flo[d] * NV + v) * NF + j], acc[v]);
            acc[v] = acc_fma(-lp, sFF[(fhi[d] * NV + v) * NF + j], acc[v]);
          }
        }
      }
    }
    __syncthreads();  // the pointwise fluxes are read; BIG takes the next stage input

    // ---- D2. RK update: w0 and the register from the staging slot, next input into BIG ----
    {
      S* xg = reinterpret_cast<S*>(V.x);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const int i = v * ROW + tid;
        C next = C(0.0f);
        if (active) {
          const int idx = (v * ne + e) * ND + node;
          const R k = acc_result(acc[v]);
          const double w0 = sW[i];
          if (two_n) {
            const R cA = Arith<R>::pair(V.ca, V.caf), cB = Arith<R>::pair(V.cb, V.cbf);
            const R dtk = V.scaled ? k : Arith<R>::pair(V.dt, V.dtf) * k;
            const R q1 = V.stage > 0 ? r_fma(cA, stored_to(sX[i], R()), dtk) : dtk;
            double w1;
            if constexpr (std::is_same<R, double>::value) w1 = fma(V.cb, q1, w0);
            else w1 = add_increment(w0, cB * q1);
            V.w[idx] = w1;
            if (!V.last) Arith<R>::store(xg + idx, q1);
            next = std::is_same<C, float>::value ? C(Arith<float>::from_double(w1)) : C(w1);
          } else {
            double w1;
            if constexpr (std::is_same<R, double>::value) w1 = fma(V.cb, k, w0);
            else w1 = add_increment(w0, Arith<R>::pair(V.cb, V.cbf) * k);
            V.w[idx] = w1;
            if (V.last) {
              next = std::is_same<C, float>::value ? C(Arith<float>::from_double(w1)) : C(w1);
            } else {
              double r1d;
              if constexpr (std::is_same<R, double>::value) r1d = fma(V.ca, k, w0);
              else r1d = add_increment(w0, Arith<R>::pair(V.ca, V.caf) * k);
              const R r1 = Arith<R>::from_double(r1d);
              Arith<R>::store(xg + idx, r1);
              if constexpr (std::is_same<C, double>::value) next = Arith<R>::to_double(r1);
              else next = r1;
            }
          }
        }
        sN[i] = next;
      }
    }
    __syncthreads();

    // ---- E. traces of the next stage input on the tile-boundary faces ---------------------
    {
      S* tro = reinterpret_cast<S*>(A.tr_out);
      constexpr int PER = NV * NF;
      for (int g = tid; g < F::NBND * PER; g += THREADS) {
        int bb = g / PER;
        const int r = g - bb * PER;
        const int v = r / NF, j = r - v * NF;
        int d, side, a0, a1;
        if (bb < F::B0) {
          d = 0; side = bb & 1; bb >>= 1; a0 = bb % TY; a1 = bb / TY;
        } else if (bb - F::B0 < F::B1) {
          bb -= F::B0; d = 1; side = bb & 1; bb >>= 1; a0 = bb % TX; a1 = bb / TX;
        } else {
          bb -= F::B0 + F::B1; d = 2; side = bb & 1; bb >>= 1; a0 = bb % TX; a1 = bb / TX;
        }
        int x, y, z;
        if (d == 0) {
          if (a0 >= E1 || a1 >= E2) continue;
          x = side ? E0 - 1 : 0; y = a0; z = a1;
        } else if (d == 1) {
          if (a0 >= E0 || a1 >= E2) continue;
          x = a0; y = side ? E1 - 1 : 0; z = a1;
        } else {
          if (a0 >= E0 || a1 >= E1) continue;
          x = a0; y = a1; z = side ? E2 - 1 : 0;
        }
        const int te = (z * TY + y) * TX + x;
        const int base = line_base<D, N>(d, j);
        const int stride = d == 0 ? 1 : (d == 1 ? N : N * N);
        const double* tw = side ? V.tab->Tp : V.tab->Tm;
        const float2* twf = side ? V.tab->Tpf : V.tab->Tmf;
        C t[N];
#pragma unroll
        for (int a = 0; a < N; ++a) t[a] = Arith<C>::tab(tw, twf, a);
        const C val = interp_line<N, C>(t, sN + v * ROW + te * ND + base, stride);
        store_trace(tro + (((d * 2 + side) * NV + v) * ne + gel(x, y, z)) * NF + j, val);
      }
    }
    __syncthreads();  // the slot and BIG are free for the next tile
  }
}

// Host-side launch of the fused kernel for one arithmetic.
template <int D, int N, typename R>
cudaError_t launch_fused_t(const FusedArgs& a, const CUtensorMap& tw, const CUtensorMap& tx,
                           cudaStream_t s) {
  using F = FT<D, N>;
  const size_t smem = FusedSmem<D, N, R>::BYTES;
  cudaError_t err = cudaFuncSetAttribute(fused_kernel<D, N, R>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  // persistent grid: every resident block slot of the device, at most one block per tile
  int dev = 0, sms = 0, per_sm = 0;
  err = cudaGetDevice(&dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (err == cudaSuccess)
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_kernel<D, N, R>, F::THREADS, smem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const long long tiles = (long long)a.ntile[0] * a.ntile[1] * a.ntile[2];
  const long long blocks = std::min<long long>(tiles, (long long)sms * per_sm);
  fused_kernel<D, N, R><<<(unsigned)blocks, F::THREADS, smem, s>>>(a, tw, tx);
  return cudaGetLastError();
}

template <typename R>
struct FusedDispatch {
  static cudaError_t run(int dim, int N, const FusedArgs& a, const CUtensorMap& tw,
                         const CUtensorMap& tx, cudaStream_t s) {
    if (dim == 2) {
      switch (N) {
        case 2: return launch_fused_t<2, 2, R>(a, tw, tx, s);
        case 3: return launch_fused_t<2, 3, R>(a, tw, tx, s);
        case 4: return launch_fused_t<2, 4, R>(a, tw, tx, s);
        case 5: return launch_fused_t<2, 5, R>(a, tw, tx, s);
        case 6: return launch_fused_t<2, 6, R>(a, tw, tx, s);
        case 7: return launch_fused_t<2, 7, R>(a, tw, tx, s);
        case 8: return launch_fused_t<2, 8, R>(a, tw, tx, s);
      }
    } else if (dim == 3) {
      switch (N) {
        case 2: return launch_fused_t<3, 2, R>(a, tw, tx, s);
        case 3: return launch_fused_t<3, 3, R>(a, tw, tx, s);
        case 4: return launch_fused_t<3, 4, R>(a, tw, tx, s);
        case 5: return launch_fused_t<3, 5, R>(a, tw, tx, s);
        case 6: return launch_fused_t<3, 6, R>(a, tw, tx, s);
      }
    }
    return cudaErrorInvalidValue;
  }
};

}  // namespace adg
