// Arithmetic layer of the operator kernels: storage type, loads/stores and the few math
// functions the Euler flux needs, for each arithmetic type R.
#pragma once
#include <cuda_runtime.h>

namespace adg {

template <typename R>
struct Arith;

template <>
struct Arith<double> {
  using S = double;
  __device__ static __forceinline__ double load(const double* p) { return __ldg(p); }
  __device__ static __forceinline__ void store(double* p, double v) { *p = v; }
  __device__ static __forceinline__ double to_double(double v) { return v; }
};

template <>
struct Arith<float> {
  using S = float;
  __device__ static __forceinline__ float load(const float* p) { return __ldg(p); }
  __device__ static __forceinline__ void store(float* p, float v) { *p = v; }
  __device__ static __forceinline__ double to_double(float v) { return (double)v; }
};

__device__ __forceinline__ double r_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float r_rcp(float x) { return 1.0f / x; }
__device__ __forceinline__ double r_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float r_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double r_max(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float r_max(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double r_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float r_fma(float a, float b, float c) { return fmaf(a, b, c); }

}  // namespace adg
