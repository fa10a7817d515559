// Batched kernels: many independent solver instances of the same dimension and degree in
// one launch.  Each launch is persistent (a grid-stride loop over "virtual blocks"); the
// virtual blocks of all instances are numbered consecutively and a block finds its
// instance by binary search over the per-instance offsets.  The element work itself is the
// single-instance code (vol_body / flux_body), reading per-instance, per-stage arguments
// from device memory, so a batched step gives bit-identical results to separate solvers.
#pragma once
#include "kernels.cuh"

namespace adg {

// Per-instance schedule state advanced on the device at the start of every step.
struct BatchSched {
  int random;        // per-interface random delays
  int pe;            // instance has subdomain faces and a delayed flux mode
  int flux_kind;     // adg_flux
  int L, np, depth;  // schedule parameters
  int head;          // ring level written last (-1: none yet)
  int pad;
  long long step;    // index of the step about to run
};

struct BatchGroupArgs {
  const int* inst;   // instance ids of the group
  const int* off;    // [n+1] first virtual block of each instance
  int n;             // instances in the group
  int total;         // virtual blocks in total
};

// Instances whose block offsets a persistent block keeps in shared memory; larger groups
// search the offsets in global memory.
constexpr int kMaxSharedOffsets = 512;

// Copy of the group's block offsets into shared memory (when they fit), once per block.
__device__ __forceinline__ const int* stage_offsets(const BatchGroupArgs& g, int* soff) {
  if (g.n >= kMaxSharedOffsets) return g.off;
  for (int i = threadIdx.x; i <= g.n; i += blockDim.x) soff[i] = g.off[i];
  __syncthreads();
  return soff;
}

// instance k of virtual block vb: off[k] <= vb < off[k+1] (binary search)
__device__ __forceinline__ int find_instance(const int* off, int n, int vb) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= vb) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Copy of one argument struct into shared memory by the whole block (16-byte words), so the
// element code reads it from shared memory instead of re-reading global memory after every
// global store it cannot prove to be unrelated.
template <typename T>
__device__ __forceinline__ void stage_args(T* dst, const T* src) {
  static_assert(sizeof(T) % 16 == 0, "argument structs are padded to 16 bytes");
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(T) / 16); i += blockDim.x) d[i] = s[i];
}

// Register budget of the batched volume kernels.  The persistent loop and the arguments
// read from shared memory raise their register use over the single-instance kernels (FP32:
// 48 against 32 at 128 threads, over 90 for tiles of 64 threads when left to the
// compiler), which cuts the occupancy the latency-bound FP32 form needs.  Budgets without
// spills (ptxas, sm_103a): FP32 40 registers in 2D (48 at N = 4 and 8 and for tiles of at
// most 64 threads), 56 in 3D; FP64 and FP32 pairs 16 above the single-instance budget
// (24 at N = 8).
template <int D, int N, typename R> struct VolRegs {
  static constexpr int value = VolKernelRegs<D, N, R>::value + (N == 8 ? 24 : 16);
};
template <int D, int N> struct VolRegs<D, N, float> {
  static constexpr int value = D != 2 ? 56 : ((N == 4 || N == 8) ? 48 : 40);
};

template <int D, int N, typename R, int TT>
__global__ void __launch_bounds__(Tile<D, N, TT>::THREADS,
                                  min_blocks_for(VolRegs<D, N, R>::value, Tile<D, N, TT>::THREADS))
batch_vol_kernel(const VolArgs* va, int nstages, int stage, BatchGroupArgs g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) VolArgs sa;
  __shared__ int soff[kMaxSharedOffsets];
  const int* off = stage_offsets(g, soff);
  int cur = -1;  // instance whose arguments sa holds (uniform over the block)
  for (int vb = blockIdx.x; vb < g.total; vb += gridDim.x) {
    const int k = find_instance(off, g.n, vb);
    if (k != cur) {
      stage_args(&sa, &va[g.inst[k] * nstages + stage]);
      __syncthreads();
      cur = k;
    }
    vol_body<D, N, R, TT>(sa, vb - off[k], smem_raw);
    __syncthreads();  // shared memory (and sa) are reused by the next virtual block
  }
}

// Element path of the batch (FP32 operator): the volume kernel with every element
// evaluating the numerical fluxes on its own faces, reading each instance's stage and face
// arguments (the face arguments carry the schedule the device advances) from shared
// memory.  No face-flux launch.
template <int D, int N, typename R> struct VolFacesBatchRegs { static constexpr int value = D == 2 ? 72 : 80; };

template <int D, int N, typename R, int TT>
__global__ void __launch_bounds__(Tile<D, N, TT>::THREADS,
                                  min_blocks_for(VolFacesBatchRegs<D, N, R>::value,
                                                 Tile<D, N, TT>::THREADS))
batch_vol_faces_kernel(const VolArgs* va, const FluxArgs* fa, int nstages, int stage,
                       BatchGroupArgs g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) VolArgs sa;
  __shared__ __align__(16) FluxArgs sf;
  __shared__ int soff[kMaxSharedOffsets];
  const int* off = stage_offsets(g, soff);
  int cur = -1;  // instance whose arguments sa and sf hold (uniform over the block)
  for (int vb = blockIdx.x; vb < g.total; vb += gridDim.x) {
    const int k = find_instance(off, g.n, vb);
    if (k != cur) {
      stage_args(&sa, &va[g.inst[k] * nstages + stage]);
      stage_args(&sf, &fa[g.inst[k] * nstages + stage]);
      __syncthreads();
      cur = k;
    }
    vol_body<D, N, R, TT, false, ElementFaces>(sa, vb - off[k], smem_raw, ElementFaces{sf, sf.tr});
    __syncthreads();  // shared memory (and the arguments) are reused by the next virtual block
  }
}

// virtual block of instance k: D * blocks_x of it, ordered (d, bx)
template <int D, int N, typename R>
__global__ void __launch_bounds__(256)
batch_flux_kernel(const FluxArgs* fa, int nstages, int stage, BatchGroupArgs g) {
  constexpr int NF = IPow<N, D - 1>::value;
  __shared__ __align__(16) FluxArgs sa;
  __shared__ int soff[kMaxSharedOffsets];
  const int* off = stage_offsets(g, soff);
  int cur = -1;  // instance whose arguments sa holds (uniform over the block)
  for (int vb = blockIdx.x; vb < g.total; vb += gridDim.x) {
    const int k = find_instance(off, g.n, vb);
    if (k != cur) {
      __syncthreads();  // every thread is done with the previous instance's arguments
      stage_args(&sa, &fa[g.inst[k] * nstages + stage]);
      __syncthreads();
      cur = k;
    }
    const int bpd = ((int)sa.m.ne * NF + 255) / 256;
    const int local = vb - off[k];
    const int d = local / bpd;
    flux_body<D, N, R>(sa, local - d * bpd, d);
  }
}

// Launchers over (dim, N, TT) for one arithmetic (2D and 3D, TT in {64, 128, 256}).
template <typename R>
struct BatchDispatch {
  // occ != nullptr: no launch; *occ = resident blocks per SM of the kernel
  template <int D, int N, int TT>
  static cudaError_t vol_t(const VolArgs* va, int ns, int st, const BatchGroupArgs& g, int grid,
                           cudaStream_t s, int* occ) {
    using T = Tile<D, N, TT>;
    const size_t smem = vol_flux_bytes<D, N, R, TT>();
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(batch_vol_kernel<D, N, R, TT>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    if (occ)
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, batch_vol_kernel<D, N, R, TT>,
                                                           T::THREADS, smem);
    batch_vol_kernel<D, N, R, TT><<<grid, T::THREADS, smem, s>>>(va, ns, st, g);
    return cudaGetLastError();
  }
  template <int D, int N, int TT>
  static cudaError_t vol_faces_t(const VolArgs* va, const FluxArgs* fa, int ns, int st,
                                 const BatchGroupArgs& g, int grid, cudaStream_t s, int* occ) {
    using T = Tile<D, N, TT>;
    const size_t smem = VolSmem<D, N, R, TT, false, true>::BYTES;
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(batch_vol_faces_kernel<D, N, R, TT>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    if (occ)
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, batch_vol_faces_kernel<D, N, R, TT>,
                                                           T::THREADS, smem);
    batch_vol_faces_kernel<D, N, R, TT><<<grid, T::THREADS, smem, s>>>(va, fa, ns, st, g);
    return cudaGetLastError();
  }
  template <int D, int N>
  static cudaError_t flux_t(const FluxArgs* fa, int ns, int st, const BatchGroupArgs& g, int grid,
                            cudaStream_t s, int* occ) {
    if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, batch_flux_kernel<D, N, R>, 256, 0);
    batch_flux_kernel<D, N, R><<<grid, 256, 0, s>>>(fa, ns, st, g);
    return cudaGetLastError();
  }
  // fa != nullptr: the element-path kernel (face fluxes from fa's traces; built for the
  // FP32 operator, the arithmetic whose batches take the element path)
  template <int D, int N>
  static cudaError_t vol_tt(int tt, const VolArgs* va, const FluxArgs* fa, int ns, int st,
                            const BatchGroupArgs& g, int grid, cudaStream_t s, int* occ) {
    if (fa) {
      if constexpr (std::is_same<R, float>::value) {
        switch (tt) {
          case 64: return vol_faces_t<D, N, 64>(va, fa, ns, st, g, grid, s, occ);
          case 128: return vol_faces_t<D, N, 128>(va, fa, ns, st, g, grid, s, occ);
          case 256: return vol_faces_t<D, N, 256>(va, fa, ns, st, g, grid, s, occ);
        }
      }
      return cudaErrorInvalidValue;
    }
    switch (tt) {
      case 64: return vol_t<D, N, 64>(va, ns, st, g, grid, s, occ);
      case 128: return vol_t<D, N, 128>(va, ns, st, g, grid, s, occ);
      case 256: return vol_t<D, N, 256>(va, ns, st, g, grid, s, occ);
    }
    return cudaErrorInvalidValue;
  }
  static cudaError_t vol(int dim, int N, int tt, const VolArgs* va, const FluxArgs* fa, int ns,
                         int st, const BatchGroupArgs& g, int grid, cudaStream_t s, int* occ) {
    if (dim == 2) {
      switch (N) {
        case 2: return vol_tt<2, 2>(tt, va, fa, ns, st, g, grid, s, occ);
        case 3: return vol_tt<2, 3>(tt, va, fa, ns, st, g, grid, s, occ);
        case 4: return vol_tt<2, 4>(tt, va, fa, ns, st, g, grid, s, occ);
        case 5: return vol_tt<2, 5>(tt, va, fa, ns, st, g, grid, s, occ);
        case 6: return vol_tt<2, 6>(tt, va, fa, ns, st, g, grid, s, occ);
        case 7: return vol_tt<2, 7>(tt, va, fa, ns, st, g, grid, s, occ);
        case 8: return vol_tt<2, 8>(tt, va, fa, ns, st, g, grid, s, occ);
      }
    } else if (dim == 3) {
      switch (N) {
        case 2: return vol_tt<3, 2>(tt, va, fa, ns, st, g, grid, s, occ);
        case 3: return vol_tt<3, 3>(tt, va, fa, ns, st, g, grid, s, occ);
        case 4: return vol_tt<3, 4>(tt, va, fa, ns, st, g, grid, s, occ);
        case 5: return vol_tt<3, 5>(tt, va, fa, ns, st, g, grid, s, occ);
        case 6: return vol_tt<3, 6>(tt, va, fa, ns, st, g, grid, s, occ);
      }
    }
    return cudaErrorInvalidValue;
  }
  static cudaError_t flux(int dim, int N, const FluxArgs* fa, int ns, int st,
                          const BatchGroupArgs& g, int grid, cudaStream_t s, int* occ) {
    if (dim == 2) {
      switch (N) {
        case 2: return flux_t<2, 2>(fa, ns, st, g, grid, s, occ);
        case 3: return flux_t<2, 3>(fa, ns, st, g, grid, s, occ);
        case 4: return flux_t<2, 4>(fa, ns, st, g, grid, s, occ);
        case 5: return flux_t<2, 5>(fa, ns, st, g, grid, s, occ);
        case 6: return flux_t<2, 6>(fa, ns, st, g, grid, s, occ);
        case 7: return flux_t<2, 7>(fa, ns, st, g, grid, s, occ);
        case 8: return flux_t<2, 8>(fa, ns, st, g, grid, s, occ);
      }
    } else if (dim == 3) {
      switch (N) {
        case 2: return flux_t<3, 2>(fa, ns, st, g, grid, s, occ);
        case 3: return flux_t<3, 3>(fa, ns, st, g, grid, s, occ);
        case 4: return flux_t<3, 4>(fa, ns, st, g, grid, s, occ);
        case 5: return flux_t<3, 5>(fa, ns, st, g, grid, s, occ);
        case 6: return flux_t<3, 6>(fa, ns, st, g, grid, s, occ);
      }
    }
    return cudaErrorInvalidValue;
  }
};

}  // namespace adg
