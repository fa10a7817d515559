// FP32-pair ("double-word") arithmetic for the operator kernels.
//
// A value is hi + lo with |lo| <= ulp(hi)/2, about 48 significant bits.  GB300 issues
// FP32 FMAs at about 62x the FP64 rate, so an operator written in this arithmetic runs
// faster than native FP64 while staying within a few units of 2^-48 of it.  Building
// blocks, all from the published error-free transformations:
//   TwoSum (Knuth, TAOCP vol. 2): s + e == a + b exactly, 6 flops, no ordering assumption;
//   FastTwoSum (Dekker 1971): same when |a| >= |b|, 3 flops;
//   TwoProd with FMA: p + e == a * b exactly, 2 flops;
//   double-word add / multiply: the accurate algorithms of Joldes, Muller & Popescu,
//     "Tight and rigorous error bounds for basic building blocks of double-word
//     arithmetic", ACM TOMS 44(2), 2017 (relative error <= 3u^2 and 4u^2, u = 2^-24);
//   reciprocal and square root: an FP32 seed refined by one Newton step carried out in
//     double-word arithmetic (error of order u^2);
//   dot products: a compensated accumulator in the style of Dot2 (Ogita, Rump & Oishi,
//     SIAM J. Sci. Comput. 26(6), 2005): the exact FP32 product and sum errors are
//     gathered in a second FP32 word, so a sum of n products carries an error of about
//     n u^2 sum |a_i b_i| instead of n u sum |a_i b_i|.
// The compiler must not reassociate FP32 operations here (no fast-math flags).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace adg {

struct df64 {
  float hi, lo;
  __device__ __forceinline__ df64() {}
  __device__ __forceinline__ df64(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ explicit df64(float h) : hi(h), lo(0.0f) {}
};

// Split of an FP64 value into an FP32 pair with integer operations only (see arith.cuh on
// the cost of F2F): hi = x rounded to 24 significant bits, lo = x - hi (|lo| <= ulp(hi)/2,
// the residual's integer mantissa is rounded to 24 bits, total error <= 2^-49 |x|).
// lo needs |x| >= 2^-74 (else it is dropped: FP32 accuracy for tiny values); |x| < 2^-126
// gives (0, 0).
__device__ __forceinline__ df64 d2df_int(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
  const unsigned long long a = b & 0x7FFFFFFFFFFFFFFFull;
  const unsigned long long hb = (a + (1ull << 28)) & ~((1ull << 29) - 1ull);
  const int e = (int)(a >> 52);
  const int eh = (int)(hb >> 52);
  const float hi = __uint_as_float(sgn | ((unsigned)(eh - 896) << 23) | ((unsigned)(hb >> 29) & 0x7FFFFFu));
  const long long dres = (long long)(a - hb);  // (|x| - |hi|) in units of 2^(e-1075), |dres| <= 2^28
  const float scale = __uint_as_float((unsigned)(e - 948) << 23);  // 2^(e-1075)
  float lo = (e >= 949) ? __int2float_rn((int)dres) * scale : 0.0f;
  lo = __uint_as_float(__float_as_uint(lo) ^ sgn);
  return (eh > 896) ? df64(hi, lo) : df64(__uint_as_float(sgn), 0.0f);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// accurate double-word + double-word
__device__ __forceinline__ df64 operator+(df64 x, df64 y) {
  float sh, sl, th, tl, vh, vl, zh, zl;
  two_sum(x.hi, y.hi, sh, sl);
  two_sum(x.lo, y.lo, th, tl);
  float c = __fadd_rn(sl, th);
  fast_two_sum(sh, c, vh, vl);
  float w = __fadd_rn(tl, vl);
  fast_two_sum(vh, w, zh, zl);
  return df64(zh, zl);
}

__device__ __forceinline__ df64 operator-(df64 x) { return df64(-x.hi, -x.lo); }
__device__ __forceinline__ df64 operator-(df64 x, df64 y) { return x + (-y); }

// double-word * double-word with FMA
__device__ __forceinline__ df64 operator*(df64 x, df64 y) {
  float ch, cl1;
  two_prod(x.hi, y.hi, ch, cl1);
  float tl0 = __fmul_rn(x.lo, y.lo);
  float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
  float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
  float cl3 = __fadd_rn(cl1, cl2);
  float zh, zl;
  fast_two_sum(ch, cl3, zh, zl);
  return df64(zh, zl);
}

// multiplication by a power of two is exact
__device__ __forceinline__ df64 scale_pow2(df64 x, float p2) { return df64(x.hi * p2, x.lo * p2); }

__device__ __forceinline__ df64 r_rcp(df64 y) {
  // r0 ~ 1/y.hi; e = 1 - y r0 (fma keeps it exact up to the lo term); r = r0 + r0 e
  float r0 = __frcp_rn(y.hi);
  float e = __fmaf_rn(-y.hi, r0, 1.0f);
  e = __fmaf_rn(-y.lo, r0, e);
  float zh, zl;
  fast_two_sum(r0, __fmul_rn(r0, e), zh, zl);
  return df64(zh, zl);
}

__device__ __forceinline__ df64 r_sqrt(df64 x) {
  if (x.hi <= 0.0f) return df64(0.0f, 0.0f);
  // s0 = sqrt(x.hi) rounded; residual x - s0^2 exactly enough; s = s0 + res / (2 s0)
  float s0 = __fsqrt_rn(x.hi);
  float ph, pl;
  two_prod(s0, s0, ph, pl);
  float res = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, ph), pl), x.lo);
  float corr = __fdividef(res, 2.0f * s0);
  float zh, zl;
  fast_two_sum(s0, corr, zh, zl);
  return df64(zh, zl);
}

__device__ __forceinline__ bool operator>(df64 a, df64 b) {
  return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo);
}
__device__ __forceinline__ df64 r_max(df64 a, df64 b) { return (b > a) ? b : a; }
__device__ __forceinline__ df64 r_fma(df64 a, df64 b, df64 c) { return a * b + c; }

// Compensated sum of products: value = s + c (unnormalised).
struct df64acc {
  float s, c;
};
__device__ __forceinline__ df64acc acc_zero(df64acc) { return df64acc{0.0f, 0.0f}; }
__device__ __forceinline__ df64acc acc_fma(df64 a, df64 b, df64acc t) {
  float p, pe, s, se;
  two_prod(a.hi, b.hi, p, pe);
  two_sum(t.s, p, s, se);
  float c = __fadd_rn(t.c, __fadd_rn(se, pe));
  c = __fmaf_rn(a.hi, b.lo, c);
  c = __fmaf_rn(a.lo, b.hi, c);
  return df64acc{s, c};
}
__device__ __forceinline__ df64 acc_result(df64acc t) {
  float zh, zl;
  two_sum(t.s, t.c, zh, zl);
  return df64(zh, zl);
}

// Two compensated dot products advanced together with the packed FP32x2 instructions of
// sm_100 and later (FFMA2 / FADD2 / FMUL2: two independent, correctly rounded FP32
// operations per instruction): lane k of every float2 belongs to the k-th dot product.
// Lane by lane the operation sequence of acc_fma (its subtractions written as fused
// multiply-adds by -1 and as negated sums, which round the same way), with half the
// instructions.
struct df64acc2 {
  float2 s, c;
};
__device__ __forceinline__ df64acc2 acc2_zero() {
  return df64acc2{make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
}
// t + a * (fh + fl) lane-wise, a = (ah, al) one pair shared by both lanes, nah = -ah
__device__ __forceinline__ df64acc2 acc2_fma(float2 ah, float2 al, float2 nah, float2 fh,
                                             float2 fl, df64acc2 t) {
  const float2 m1 = make_float2(-1.0f, -1.0f);
  const float2 pn = __fmul2_rn(nah, fh);      // -p, p = ah fh rounded
  const float2 pe = __ffma2_rn(ah, fh, pn);   // ah fh - p, exact
  const float2 s = __ffma2_rn(pn, m1, t.s);   // t.s + p
  const float2 bp = __ffma2_rn(t.s, m1, s);   // s - t.s
  const float2 ap = __ffma2_rn(bp, m1, s);    // s - bp
  const float2 e1 = __ffma2_rn(ap, m1, t.s);  // t.s - ap
  const float2 e2n = __fadd2_rn(pn, bp);      // -(p - bp)
  const float2 se = __ffma2_rn(e2n, m1, e1);  // (t.s - ap) + (p - bp): the TwoSum error
  float2 c = __fadd2_rn(t.c, __fadd2_rn(se, pe));
  c = __ffma2_rn(ah, fl, c);
  c = __ffma2_rn(al, fh, c);
  return df64acc2{s, c};
}
// lane k as a scalar accumulator
__device__ __forceinline__ df64acc acc2_lane(const df64acc2& t, int k) {
  return k == 0 ? df64acc{t.s.x, t.c.x} : df64acc{t.s.y, t.c.y};
}

// Two independent double-word values in the lanes of float2 words (lane k: hi.k + lo.k),
// with the scalar algorithms above executed lane-wise by the packed FP32x2 instructions:
// the two sides of a face run their pointwise flux in one instruction stream.
struct df64x2 {
  float2 hi, lo;
  __device__ __forceinline__ df64x2() {}
  __device__ __forceinline__ df64x2(float2 h, float2 l) : hi(h), lo(l) {}
  __device__ __forceinline__ explicit df64x2(float h)
      : hi(make_float2(h, h)), lo(make_float2(0.0f, 0.0f)) {}
};
__device__ __forceinline__ df64x2 df64x2_of(df64 a, df64 b) {
  return df64x2(make_float2(a.hi, b.hi), make_float2(a.lo, b.lo));
}
__device__ __forceinline__ df64 df64x2_lane(const df64x2& x, int k) {
  return k == 0 ? df64(x.hi.x, x.lo.x) : df64(x.hi.y, x.lo.y);
}

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
  const float2 m1 = make_float2(-1.0f, -1.0f);
  s = __fadd2_rn(a, b);
  const float2 bp = __ffma2_rn(a, m1, s);   // s - a
  const float2 ap = __ffma2_rn(bp, m1, s);  // s - bp
  e = __fadd2_rn(__ffma2_rn(ap, m1, a), __ffma2_rn(bp, m1, b));  // (a - ap) + (b - bp)
}
__device__ __forceinline__ void fast_two_sum2(float2 a, float2 b, float2& s, float2& e) {
  const float2 m1 = make_float2(-1.0f, -1.0f);
  s = __fadd2_rn(a, b);
  e = __ffma2_rn(__ffma2_rn(a, m1, s), m1, b);  // b - (s - a)
}
__device__ __forceinline__ df64x2 operator+(df64x2 x, df64x2 y) {
  float2 sh, sl, th, tl, vh, vl, zh, zl;
  two_sum2(x.hi, y.hi, sh, sl);
  two_sum2(x.lo, y.lo, th, tl);
  const float2 c = __fadd2_rn(sl, th);
  fast_two_sum2(sh, c, vh, vl);
  const float2 w = __fadd2_rn(tl, vl);
  fast_two_sum2(vh, w, zh, zl);
  return df64x2(zh, zl);
}
__device__ __forceinline__ df64x2 operator-(df64x2 x) { return df64x2(neg2(x.hi), neg2(x.lo)); }
__device__ __forceinline__ df64x2 operator-(df64x2 x, df64x2 y) { return x + (-y); }
__device__ __forceinline__ df64x2 operator*(df64x2 x, df64x2 y) {
  const float2 ch = __fmul2_rn(x.hi, y.hi);
  const float2 cl1 = __ffma2_rn(x.hi, y.hi, neg2(ch));  // exact product error
  const float2 tl0 = __fmul2_rn(x.lo, y.lo);
  const float2 tl1 = __ffma2_rn(x.hi, y.lo, tl0);
  const float2 cl2 = __ffma2_rn(x.lo, y.hi, tl1);
  const float2 cl3 = __fadd2_rn(cl1, cl2);
  float2 zh, zl;
  fast_two_sum2(ch, cl3, zh, zl);
  return df64x2(zh, zl);
}
__device__ __forceinline__ df64x2 r_fma(df64x2 a, df64x2 b, df64x2 c) { return a * b + c; }
__device__ __forceinline__ df64x2 r_rcp(df64x2 y) {
  // per lane: FP32 seed, then the pair Newton step of r_rcp(df64)
  const float2 r0 = make_float2(__frcp_rn(y.hi.x), __frcp_rn(y.hi.y));
  float2 e = __ffma2_rn(neg2(y.hi), r0, make_float2(1.0f, 1.0f));
  e = __ffma2_rn(neg2(y.lo), r0, e);
  float2 zh, zl;
  fast_two_sum2(r0, __fmul2_rn(r0, e), zh, zl);
  return df64x2(zh, zl);
}
__device__ __forceinline__ df64x2 sub_half(df64x2 w, df64x2 k) {
  const float2 h = make_float2(0.5f, 0.5f);
  return w - df64x2(__fmul2_rn(h, k.hi), __fmul2_rn(h, k.lo));
}

}  // namespace adg
