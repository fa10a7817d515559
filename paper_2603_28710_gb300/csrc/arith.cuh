// Arithmetic layer of the operator kernels: storage type, conversions, table access,
// dot-product accumulators and the few math functions the Euler flux needs, for each
// operator arithmetic R (double, float, df64).
#pragma once
#include <cuda_runtime.h>

#include "df64.cuh"

namespace adg {

// ---- conversions without F2F --------------------------------------------------------
// On GB300 the F2F conversions between FP64 and FP32 issue at the FP64 rate (about 2 per
// clock per SM, like DADD), 60x slower than FP32 arithmetic, so the reduced-precision
// kernels convert with integer operations instead.  Valid for normal values with
// |x| < 3.4e38; magnitudes below 2^-126 become signed zero.

// double -> float, rounded to nearest (ties away from zero)
__device__ __forceinline__ float d2f_int(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
  const unsigned long long r = (b & 0x7FFFFFFFFFFFFFFFull) + (1ull << 28);  // + half FP32 ulp
  const int er = (int)(r >> 52);
  const unsigned fb = sgn | ((unsigned)(er - 896) << 23) | ((unsigned)(r >> 29) & 0x7FFFFFu);
  return __uint_as_float(er > 896 ? fb : sgn);
}

// float -> double, exact (subnormal floats give signed zero)
__device__ __forceinline__ double f2d_int(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long b =
      sgn | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)(e ? b : sgn));
}

template <typename R>
struct Arith;

template <>
struct Arith<double> {
  using S = double;   // storage of traces / fluxes / ring entries
  using Acc = double; // dot-product accumulator
  __device__ static __forceinline__ double load(const double* p) { return __ldg(p); }
  __device__ static __forceinline__ void store(double* p, double v) { *p = v; }
  __device__ static __forceinline__ double to_double(double v) { return v; }
  __device__ static __forceinline__ double from_double(double v) { return v; }
  __device__ static __forceinline__ double tab(const double* d, const float2*, int i) { return d[i]; }
  __device__ static __forceinline__ double pair(double d, float2) { return d; }
};

template <>
struct Arith<float> {
  using S = float;
  using Acc = float;
  __device__ static __forceinline__ float load(const float* p) { return __ldg(p); }
  __device__ static __forceinline__ void store(float* p, float v) { *p = v; }
  __device__ static __forceinline__ double to_double(float v) { return f2d_int(v); }
  __device__ static __forceinline__ float from_double(double v) { return d2f_int(v); }
  __device__ static __forceinline__ float tab(const double*, const float2* f, int i) { return f[i].x; }
  __device__ static __forceinline__ float pair(double, float2 f) { return f.x; }
};

template <>
struct Arith<df64> {
  using S = float2;
  using Acc = df64acc;
  __device__ static __forceinline__ df64 load(const float2* p) {
    float2 v = __ldg(p);
    return df64(v.x, v.y);
  }
  __device__ static __forceinline__ void store(float2* p, df64 v) { *p = make_float2(v.hi, v.lo); }
  __device__ static __forceinline__ double to_double(df64 v) { return f2d_int(v.hi) + f2d_int(v.lo); }
  __device__ static __forceinline__ df64 from_double(double v) { return d2df_int(v); }
  __device__ static __forceinline__ df64 tab(const double*, const float2* f, int i) {
    return df64(f[i].x, f[i].y);
  }
  __device__ static __forceinline__ df64 pair(double, float2 f) { return df64(f.x, f.y); }
};

// FP64 reciprocal: an FP32 seed r0 (integer conversions, MUFU approximation, relative
// error |e| about 2^-22 with e = 1 - x r0) refined by the geometric series
// 1/x = r0 / (1 - e) = r0 (1 + e + e^2 + ...), kept to second order: the truncation leaves
// e^3 (about 2^-66), below FP64 rounding.  3 DFMA instead of the IEEE division sequence;
// not correctly rounded (within an ulp).  For 1e-37 < |x| < 1e37.
__device__ __forceinline__ double r_rcp(double x) {
  float xf = d2f_int(x), rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(xf));
  const double r0 = f2d_int(rf);
  const double e = fma(-x, r0, 1.0);
  const double p = fma(e, e, e);  // e + e^2
  return fma(r0, p, r0);
}
// FP32 operator: the hardware approximations (PTX rcp.approx / sqrt.approx, at most one
// ulp and 2^-23 relative error), one instruction each instead of the IEEE sequences.
__device__ __forceinline__ float r_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double r_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float r_sqrt(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double r_max(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float r_max(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double r_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float r_fma(float a, float b, float c) { return fmaf(a, b, c); }

// w - k / 2 (one fused operation where the arithmetic has one)
__device__ __forceinline__ double sub_half(double w, double k) { return fma(-0.5, k, w); }
__device__ __forceinline__ float sub_half(float w, float k) { return fmaf(-0.5f, k, w); }
__device__ __forceinline__ df64 sub_half(df64 w, df64 k) { return w - df64(0.5f * k.hi, 0.5f * k.lo); }

// multiplication by a power of two (exact)
__device__ __forceinline__ double scale_pow2(double x, float p2) { return x * (double)p2; }
__device__ __forceinline__ float scale_pow2(float x, float p2) { return x * p2; }


// accumulators: plain FMA chains for the native types
__device__ __forceinline__ double acc_zero(double) { return 0.0; }
__device__ __forceinline__ float acc_zero(float) { return 0.0f; }
__device__ __forceinline__ double acc_fma(double a, double b, double t) { return fma(a, b, t); }
__device__ __forceinline__ float acc_fma(float a, float b, float t) { return fmaf(a, b, t); }
__device__ __forceinline__ double acc_result(double t) { return t; }
__device__ __forceinline__ float acc_result(float t) { return t; }

}  // namespace adg
