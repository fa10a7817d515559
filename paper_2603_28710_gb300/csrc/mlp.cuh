// Shared pieces of the learned ghost-trace predictor (mlp.cu and the solver's learned
// flux correction): parameter layout and BF16 conversions.
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


}  // namespace adg
