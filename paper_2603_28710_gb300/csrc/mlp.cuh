// Shared pieces of the learned ghost-trace predictor (mlp.cu and the solver's learned
// flux correction): parameter layout, BF16 conversions and single-sample inference.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace adg {

constexpr int kMlpParams = 4545;
constexpr int kW1 = 0, kB1 = 256, kW2 = 320, kB2 = 4416, kW3 = 4480, kB3 = 4544;

// BF16 <-> FP32: BF16 is the upper half of an FP32; rounding to nearest even.
__host__ __device__ __forceinline__ float bf16_to_float(uint16_t b) {
  union { unsigned u; float f; } c;
  c.u = (unsigned)b << 16;
  return c.f;
}
__host__ __device__ __forceinline__ uint16_t float_to_bf16(float f) {
  union { unsigned u; float f; } c;
  c.f = f;
  unsigned u = c.u;
  if ((u & 0x7F800000u) == 0x7F800000u) return (uint16_t)((u >> 16) | ((u & 0xFFFFu) ? 0x40u : 0u));
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

// y = w3 . tanh(W2 tanh(W1 x + b1) + b2) + b3 with W (FP32 copy of the BF16 weights) in
// shared memory; FP32 accumulation.
__device__ __forceinline__ float mlp_eval(const float* W, const float* x) {
  float h1[64];
#pragma unroll
  for (int j = 0; j < 64; ++j) {
    float z = W[kB1 + j];
#pragma unroll
    for (int i = 0; i < 4; ++i) z = fmaf(W[kW1 + j * 4 + i], x[i], z);
    h1[j] = tanhf(z);
  }
  float y = W[kB3];
  for (int j = 0; j < 64; ++j) {
    float z = W[kB2 + j];
#pragma unroll
    for (int i = 0; i < 64; ++i) z = fmaf(W[kW2 + j * 64 + i], h1[i], z);
    y = fmaf(W[kW3 + j], tanhf(z), y);
  }
  return y;
}

}  // namespace adg
