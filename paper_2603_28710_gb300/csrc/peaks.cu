// Arithmetic peak probes (adg_measure_peak in include/adg.h): the rates that bound the
// operator kernels, measured on the GPU the library runs on instead of taken from a data
// sheet.  Each probe keeps every warp slot busy with independent dependency chains of one
// instruction kind and times launches of about 50 ms with CUDA events (best of three, after
// a warm-up launch).
//
//   kind 0  FP64 FMA (DFMA):               12 independent chains per thread
//   kind 1  FP32 FMA (FFMA):               12 independent chains per thread
//   kind 2  FP64 tensor MMA (DMMA):        mma.sync m8n8k4 f64, 4 independent accumulators per warp
//   kind 3  DFMA and DMMA together:        even warps run kind 0, odd warps kind 2
//   kind 4  packed FP32x2 FMA (FFMA2):     12 independent chains of float2 per thread
//   kind 5  FP64 add (DADD):               12 independent chains per thread (1 flop each)
//   kind 6  FP64 multiply (DMUL):          12 independent chains per thread (1 flop each)
//
// Kind 3 tells whether the FP64 tensor path adds throughput to the FP64 FMA pipe (its rate
// is then close to the sum of kinds 0 and 2) or shares it (close to either alone).
// The SM clock during the launch is measured too (clock64 cycles of one thread against the
// global nanosecond timer), so a rate can be stated per SM and clock cycle.
#include <cuda_runtime.h>

#include <string>

#include "../../include/adg.h"

namespace adg {
void noalloc_set_error(const char* msg);  // per-thread error text (host.cu)
}

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 12;

// Every chain has its own multiplier and addend, held in registers: they depend on the
// thread, so the compiler cannot make them constant-bank operands (FP64 FMAs with
// constant-bank operands measured 16 % slower on GB300: 1.006 against 1.193 TFLOP/s).
__device__ __forceinline__ void dfma_chains(double (&a)[kChains], const double (&b)[kChains],
                                            const double (&c)[kChains], int iters) {
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b[j], c[j]);
  }
}

__device__ __forceinline__ void dmma_chains(double (&acc)[4][2], double a, double b, int iters) {
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      asm volatile(
          "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
          : "+d"(acc[j][0]), "+d"(acc[j][1])
          : "d"(a), "d"(b));
  }
}

// The results feed a store that never happens for these inputs (|a| stays below 2), so
// the compiler keeps every operation.
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void __launch_bounds__(kThreads) probe_kernel(int kind, int iters, double seed,
                                                         double* sink, long long* clk) {
  const int warp = threadIdx.x >> 5;
  long long c0 = 0;
  unsigned long long t0 = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c0 = clock64();
    t0 = global_ns();
  }
  const bool use_mma = kind == 2 || (kind == 3 && (warp & 1));
  if (kind == 1) {
    float a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = (float)seed * (j + 1) + threadIdx.x * 1e-7f;
    const float b = 0.999999f * (1.0f + threadIdx.x * 1e-9f), c = 1e-7f * (1.0f + blockIdx.x * 1e-9f);
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s > 1e30f) sink[blockIdx.x] = s;
  } else if (kind == 4) {
    float2 a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j)
      a[j] = make_float2((float)seed * (j + 1), (float)seed * (j + 2) + threadIdx.x * 1e-7f);
    const float tv = 1.0f + threadIdx.x * 1e-9f;  // registers, not constant-bank operands
    const float2 b = make_float2(0.999999f * tv, 0.999998f * tv), c = make_float2(1e-7f * tv, 2e-7f * tv);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = __ffma2_rn(a[j], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j].x + a[j].y;
    if (s > 1e30f) sink[blockIdx.x] = s;
  } else if (kind == 5 || kind == 6) {
    double a[kChains], b[kChains];
    const double tv = 1.0 + threadIdx.x * 1e-12;  // per-chain operands in registers
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
      a[j] = seed * (j + 1) + threadIdx.x * 1e-9;
      b[j] = (kind == 5 ? 1e-12 * (j + 1) : 0.9999999 - 1e-9 * j) * tv;
    }
    // one loop per kind: a select inside the loop would execute both operations
    if (kind == 5) {
#pragma unroll 4
      for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = a[j] + b[j];
      }
    } else {
#pragma unroll 4
      for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = a[j] * b[j];
      }
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s > 1e300) sink[blockIdx.x] = s;
  } else if (use_mma) {
    double acc[4][2];
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j][0] = acc[j][1] = seed * (j + 1);
    dmma_chains(acc, 1e-3, 0.999, iters / 4);  // 4 MMAs per iteration, each 512 flops per warp
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) s += acc[j][0] + acc[j][1];
    if (s > 1e300) sink[blockIdx.x] = s;
  } else {
    double a[kChains], b[kChains], c[kChains];
    const double tv = 1.0 + threadIdx.x * 1e-12, bv = 1.0 + blockIdx.x * 1e-12;
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
      a[j] = seed * (j + 1) + threadIdx.x * 1e-9;
      b[j] = (0.999999 - 1e-7 * j) * tv;
      c[j] = 1e-9 * (j + 1) * bv;
    }
    dfma_chains(a, b, c, iters);
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s > 1e300) sink[blockIdx.x] = s;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    clk[0] = clock64() - c0;
    clk[1] = (long long)(global_ns() - t0);
  }
}

// flops of one launch: per FMA thread 2 * kChains * iters (FP32x2: twice that); per MMA
// warp (iters / 4) * 4 * 512
double launch_flops(int kind, int blocks, int iters) {
  const double warps = (double)blocks * (kThreads / 32);
  const double fma_warp = 32.0 * 2.0 * kChains * iters;
  const double mma_warp = (double)(iters / 4) * 4 * 512.0;
  switch (kind) {
    case 0: case 1: return warps * fma_warp;
    case 5: case 6: return warps * fma_warp / 2.0;
    case 4: return warps * fma_warp * 2.0;
    case 2: return warps * mma_warp;
    case 3: return warps / 2 * (fma_warp + mma_warp);
  }
  return 0.0;
}

adg_status probe_fail(adg_status st, const std::string& m) {
  adg::noalloc_set_error(m.c_str());
  return st;
}

}  // namespace

extern "C" adg_status adg_measure_peak(int kind, double* tflops, double* ms, double* sm_mhz) {
  if (kind < 0 || kind > 6 || !tflops) return probe_fail(ADG_ERR_INVALID, "bad peak-probe arguments");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return probe_fail(ADG_ERR_CUDA, std::string("device query: ") + cudaGetErrorString(e));
  // eight blocks of 256 threads per SM: 64 warps per SM, sixteen per sub-partition
  const int blocks = sms * 8;
  // about 50 ms per launch at the nominal rates (FP64 1.25, FP32 75 TFLOP/s)
  const int iters = (kind == 1) ? 500000 : (kind == 4 ? 250000 : 8000);
  double* sink = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaMalloc((void**)&sink, (size_t)blocks * sizeof(double) + 16);
  long long* clk = reinterpret_cast<long long*>(sink + blocks);
  float best = 0.f;
  double mhz = 0.0;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // first launch is a warm-up
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) probe_kernel<<<blocks, kThreads, 0, s>>>(kind, iters, 0.5, sink, clk);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    long long c[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(c, clk, sizeof(c), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && rep > 0 && (best == 0.f || t < best)) {
      best = t;
      mhz = c[1] > 0 ? 1e3 * (double)c[0] / (double)c[1] : 0.0;
    }
  }
  if (sink) cudaFree(sink);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (e != cudaSuccess) return probe_fail(ADG_ERR_CUDA, std::string("peak probe: ") + cudaGetErrorString(e));
  *tflops = launch_flops(kind, blocks, iters) / (best * 1e-3) / 1e12;
  if (ms) *ms = best;
  if (sm_mhz) *sm_mhz = mhz;
  return ADG_OK;
}
