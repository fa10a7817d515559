// Learned ghost-trace predictor: a small MLP, 4 inputs -> 64 -> 64 -> 1, tanh hidden
// activations, BF16 weights read into FP32 and FP32 accumulation everywhere.  Kernels for
// the mean-squared-error gradient of a sample set (forward + backward, FP32 pipe), an Adam
// step on FP32 master weights that refreshes their BF16 copy, and inference (the hidden
// layer on the tensor cores).
//
// Parameter layout (kMlpParams = 4545 values):
//   W1[64][4] | b1[64] | W2[64][64] | b2[64] | w3[64] | b3
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/adg.h"
#include "mlp.cuh"

namespace adg {
void noalloc_set_error(const char* msg);

namespace {

constexpr int kSamples = 128;   // samples per chunk (one per thread)
constexpr int kPad = kSamples + 1;  // row stride of the per-sample tables (no bank conflicts)

// shared memory: weights | X[4][kPad] | H1[64][kPad] | H2[64][kPad] | DZ2[64][kPad] | DZ1[64][kPad] | DY[kPad]
constexpr int kSmemFloats = 4548 + 4 * kPad + 4 * 64 * kPad + kPad;

__global__ void __launch_bounds__(kSamples)
mlp_grad_kernel(const uint16_t* __restrict__ pbf, const float* __restrict__ x,
                const float* __restrict__ t, int n, float inv_n, float* __restrict__ grad,
                float* __restrict__ loss) {
  extern __shared__ float sm[];
  float* W = sm;
  float* X = W + 4548;
  float* H1 = X + 4 * kPad;
  float* H2 = H1 + 64 * kPad;
  float* DZ2 = H2 + 64 * kPad;
  float* DZ1 = DZ2 + 64 * kPad;
  float* DY = DZ1 + 64 * kPad;
  const int tid = threadIdx.x;
  for (int i = tid; i < kMlpParams; i += blockDim.x) W[i] = bf16_to_float(pbf[i]);
  // each thread owns gradient entries tid, tid + 128, ... (36 of them at most)
  constexpr int kOwn = (kMlpParams + kSamples - 1) / kSamples;
  float gacc[kOwn];
#pragma unroll
  for (int k = 0; k < kOwn; ++k) gacc[k] = 0.0f;
  float lacc = 0.0f;
  __syncthreads();
  const int chunks = (n + kSamples - 1) / kSamples;
  for (int c = blockIdx.x; c < chunks; c += gridDim.x) {
    const int s = c * kSamples + tid;
    const bool valid = s < n;
    float xi[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      xi[i] = valid ? x[(size_t)s * 4 + i] : 0.0f;
      X[i * kPad + tid] = xi[i];
    }
    // forward
    for (int j = 0; j < 64; ++j) {
      float z = W[kB1 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i) z = fmaf(W[kW1 + j * 4 + i], xi[i], z);
      H1[j * kPad + tid] = tanhf(z);
    }
    float y = W[kB3];
    for (int j = 0; j < 64; ++j) {
      float z = W[kB2 + j];
      for (int i = 0; i < 64; ++i) z = fmaf(W[kW2 + j * 64 + i], H1[i * kPad + tid], z);
      const float h = tanhf(z);
      H2[j * kPad + tid] = h;
      y = fmaf(W[kW3 + j], h, y);
    }
    const float r = valid ? (y - t[s]) : 0.0f;
    lacc = fmaf(r * r, inv_n, lacc);
    const float dy = 2.0f * r * inv_n;
    DY[tid] = dy;
    // backward
    for (int j = 0; j < 64; ++j) {
      const float h = H2[j * kPad + tid];
      DZ2[j * kPad + tid] = dy * W[kW3 + j] * (1.0f - h * h);
    }
    for (int i = 0; i < 64; ++i) {
      float dh = 0.0f;
      for (int j = 0; j < 64; ++j) dh = fmaf(W[kW2 + j * 64 + i], DZ2[j * kPad + tid], dh);
      const float h = H1[i * kPad + tid];
      DZ1[i * kPad + tid] = dh * (1.0f - h * h);
    }
    __syncthreads();
    // gradient contributions of this chunk, summed over its samples
#pragma unroll
    for (int k = 0; k < kOwn; ++k) {
      const int e = tid + k * kSamples;
      if (e >= kMlpParams) break;
      float acc = 0.0f;
      if (e < kB1) {                       // W1[j][i]
        const int j = e >> 2, i = e & 3;
        for (int q = 0; q < kSamples; ++q) acc = fmaf(DZ1[j * kPad + q], X[i * kPad + q], acc);
      } else if (e < kW2) {                // b1[j]
        const int j = e - kB1;
        for (int q = 0; q < kSamples; ++q) acc += DZ1[j * kPad + q];
      } else if (e < kB2) {                // W2[j][i]
        const int j = (e - kW2) >> 6, i = (e - kW2) & 63;
        for (int q = 0; q < kSamples; ++q) acc = fmaf(DZ2[j * kPad + q], H1[i * kPad + q], acc);
      } else if (e < kW3) {                // b2[j]
        const int j = e - kB2;
        for (int q = 0; q < kSamples; ++q) acc += DZ2[j * kPad + q];
      } else if (e < kB3) {                // w3[j]
        const int j = e - kW3;
        for (int q = 0; q < kSamples; ++q) acc = fmaf(DY[q], H2[j * kPad + q], acc);
      } else {                             // b3
        for (int q = 0; q < kSamples; ++q) acc += DY[q];
      }
      gacc[k] += acc;
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < kOwn; ++k) {
    const int e = tid + k * kSamples;
    if (e < kMlpParams) atomicAdd(&grad[e], gacc[k]);
  }
  // block-reduce the loss
  __shared__ float red[kSamples];
  red[tid] = lacc;
  __syncthreads();
  for (int st = kSamples / 2; st > 0; st >>= 1) {
    if (tid < st) red[tid] += red[tid + st];
    __syncthreads();
  }
  if (tid == 0) atomicAdd(loss, red[0]);
}

// ---- inference on the tensor cores --------------------------------------------------
// The 64 x 64 hidden layer of a tile of 16 samples is a [16 x 64] x [64 x 64] product: warp-
// level BF16 MMAs (mma.sync m16n8k16, FP32 accumulation).  The BF16 weights enter exactly;
// the FP32 activations of the first layer are split into three BF16 terms
// h = h0 + h1 + h2 (each the BF16 rounding of what the previous terms leave; residual below
// 2^-24 |h|), so the product keeps FP32 accuracy at three MMAs per k-step.  The 4 -> 64
// input layer, the tanh activations and the 64 -> 1 output layer stay on the FP32 pipe.
//
// Fragment layouts of mma.m16n8k16 (PTX ISA; g = lane / 4, t = lane % 4):
//   A (16 x 16, row-major, 4 x b32 = 8 bf16): reg 0 = rows g, cols 2t, 2t+1; reg 1 = row g+8;
//     reg 2 = row g, cols 2t+8, 2t+9; reg 3 = row g+8, cols 2t+8, 2t+9 (lower half first)
//   B (16 x 8, column-major, 2 x b32): reg 0 = rows (k) 2t, 2t+1 of column (n) g; reg 1 =
//     rows 2t+8, 2t+9
//   C/D (16 x 8, f32): c0, c1 = row g, cols 2t, 2t+1; c2, c3 = row g+8

__device__ __forceinline__ unsigned short bf16_bits_rn(float f) { return float_to_bf16(f); }

__device__ __forceinline__ unsigned pack_bf16(float lo_col, float hi_col) {
  return (unsigned)bf16_bits_rn(lo_col) | ((unsigned)bf16_bits_rn(hi_col) << 16);
}

// three-term BF16 split of two adjacent activations into three packed registers
__device__ __forceinline__ void split3(float a, float b, unsigned& r0, unsigned& r1, unsigned& r2) {
  const float a0 = bf16_to_float(bf16_bits_rn(a)), b0 = bf16_to_float(bf16_bits_rn(b));
  const float a1r = a - a0, b1r = b - b0;  // exact (Sterbenz)
  const float a1 = bf16_to_float(bf16_bits_rn(a1r)), b1 = bf16_to_float(bf16_bits_rn(b1r));
  r0 = pack_bf16(a0, b0);
  r1 = pack_bf16(a1, b1);
  r2 = pack_bf16(a1r - a1, b1r - b1);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], unsigned b0,
                                         unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int kInferWarps = 4;

__global__ void __launch_bounds__(32 * kInferWarps)
mlp_forward_mma_kernel(const uint16_t* __restrict__ pbf, const float* __restrict__ x, int n,
                       float* __restrict__ y) {
  __shared__ float Wf[kW2];                  // W1 | b1 (FP32)
  __shared__ float Wo[kMlpParams - kB2];     // b2 | w3 | b3 (FP32)
  __shared__ __align__(16) uint16_t W2[64 * 64];  // [n = out][k = in], BF16
  for (int i = threadIdx.x; i < kW2; i += blockDim.x) Wf[i] = bf16_to_float(pbf[i]);
  for (int i = threadIdx.x; i < kMlpParams - kB2; i += blockDim.x) Wo[i] = bf16_to_float(pbf[kB2 + i]);
  for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) W2[i] = pbf[kW2 + i];
  __syncthreads();
  const unsigned* W2w = reinterpret_cast<const unsigned*>(W2);  // pairs along k
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int tiles = (n + 15) / 16;
  for (int tile = blockIdx.x * kInferWarps + (threadIdx.x >> 5); tile < tiles;
       tile += gridDim.x * kInferWarps) {
    const int r0 = tile * 16 + g, r1 = r0 + 8;
    float x0[4], x1[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      x0[i] = r0 < n ? x[(size_t)r0 * 4 + i] : 0.0f;
      x1[i] = r1 < n ? x[(size_t)r1 * 4 + i] : 0.0f;
    }
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[j][q] = 0.0f;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      // first-layer activations of this k-block: columns c0, c0+1 and c0+8, c0+9 of rows r0, r1
      const int c0 = kk * 16 + 2 * t;
      float h[2][4];  // [row][col c0, c0+1, c0+8, c0+9]
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = c0 + (q & 1) + (q >> 1) * 8;
        float z0 = Wf[kB1 + c], z1 = Wf[kB1 + c];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          z0 = fmaf(Wf[kW1 + c * 4 + i], x0[i], z0);
          z1 = fmaf(Wf[kW1 + c * 4 + i], x1[i], z1);
        }
        h[0][q] = tanhf(z0);
        h[1][q] = tanhf(z1);
      }
      unsigned a[3][4];
      split3(h[0][0], h[0][1], a[0][0], a[1][0], a[2][0]);
      split3(h[1][0], h[1][1], a[0][1], a[1][1], a[2][1]);
      split3(h[0][2], h[0][3], a[0][2], a[1][2], a[2][2]);
      split3(h[1][2], h[1][3], a[0][3], a[1][3], a[2][3]);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int nrow = j * 8 + g;  // output unit of this lane's B column
        const unsigned b0 = W2w[(nrow * 64 + kk * 16 + 2 * t) >> 1];
        const unsigned b1 = W2w[(nrow * 64 + kk * 16 + 2 * t + 8) >> 1];
        mma_bf16(acc[j], a[0], b0, b1);
        mma_bf16(acc[j], a[1], b0, b1);
        mma_bf16(acc[j], a[2], b0, b1);
      }
    }
    // second activation and the output layer: this lane holds columns 2t, 2t+1 of each
    // 8-column block for rows r0 (acc[j][0..1]) and r1 (acc[j][2..3])
    float y0 = 0.0f, y1 = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int c = j * 8 + 2 * t + q;
        const float w3 = Wo[kW3 - kB2 + c], b2 = Wo[c];
        y0 = fmaf(w3, tanhf(acc[j][q] + b2), y0);
        y1 = fmaf(w3, tanhf(acc[j][2 + q] + b2), y1);
      }
    y0 += __shfl_xor_sync(0xffffffffu, y0, 1);
    y0 += __shfl_xor_sync(0xffffffffu, y0, 2);
    y1 += __shfl_xor_sync(0xffffffffu, y1, 1);
    y1 += __shfl_xor_sync(0xffffffffu, y1, 2);
    if (t == 0) {
      const float b3 = Wo[kB3 - kB2];
      if (r0 < n) y[r0] = y0 + b3;
      if (r1 < n) y[r1] = y1 + b3;
    }
  }
}

// Adam (Kingma & Ba 2015) on the FP32 master weights; refreshes the BF16 copy and clears
// the gradient for the next accumulation.
__global__ void mlp_adam_kernel(float* __restrict__ p, uint16_t* __restrict__ pbf,
                                float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, float lr, float b1, float b2, float eps,
                                float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpParams) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  pbf[i] = float_to_bf16(pi);
  g[i] = 0.0f;
}

__global__ void to_bf16_kernel(const float* __restrict__ p, uint16_t* __restrict__ pbf, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) pbf[i] = float_to_bf16(p[i]);
}

}  // namespace

cudaError_t mlp_infer(const uint16_t* params, const float* x, int64_t n, float* y, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t tiles = (n + 15) / 16;
  const int64_t want = (tiles + kInferWarps - 1) / kInferWarps;
  const int blocks = (int)(want < 152 * 16 ? want : 152 * 16);
  mlp_forward_mma_kernel<<<blocks, 32 * kInferWarps, 0, s>>>(params, x, (int)n, y);
  return cudaGetLastError();
}

namespace {

adg_status mfail(adg_status st, const std::string& m) {
  noalloc_set_error(m.c_str());
  return st;
}

}  // namespace
}  // namespace adg

using namespace adg;

extern "C" {

adg_status adg_mlp_grad(const uint16_t* params_bf16, const float* x, const float* target,
                        int64_t n, float* grad, float* loss, void* cuda_stream) {
  if (!params_bf16 || !x || !target || !grad || !loss || n < 0)
    return mfail(ADG_ERR_INVALID, "bad arguments");
  if (n == 0) return ADG_OK;
  if (n >= ((int64_t)1 << 31)) return mfail(ADG_ERR_INVALID, "too many samples");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const size_t smem = sizeof(float) * kSmemFloats;
  cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return mfail(ADG_ERR_CUDA, cudaGetErrorString(e));
  const int chunks = (int)((n + kSamples - 1) / kSamples);
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = chunks < sms ? chunks : sms;
  mlp_grad_kernel<<<grid, kSamples, smem, s>>>(params_bf16, x, target, (int)n, 1.0f / (float)n, grad, loss);
  e = cudaGetLastError();
  return e == cudaSuccess ? ADG_OK : mfail(ADG_ERR_CUDA, cudaGetErrorString(e));
}

adg_status adg_mlp_forward(const uint16_t* params_bf16, const float* x, int64_t n, float* y,
                           void* cuda_stream) {
  if (!params_bf16 || !x || !y || n < 0) return mfail(ADG_ERR_INVALID, "bad arguments");
  if (n == 0) return ADG_OK;
  if (n >= ((int64_t)1 << 31)) return mfail(ADG_ERR_INVALID, "too many samples");
  cudaError_t e = mlp_infer(params_bf16, x, n, y, (cudaStream_t)cuda_stream);
  return e == cudaSuccess ? ADG_OK : mfail(ADG_ERR_CUDA, cudaGetErrorString(e));
}

adg_status adg_mlp_adam(float* params, uint16_t* params_bf16, float* grad, float* m, float* v,
                        float lr, float beta1, float beta2, float eps, int t, void* cuda_stream) {
  if (!params || !params_bf16 || !grad || !m || !v || t < 1) return mfail(ADG_ERR_INVALID, "bad arguments");
  const float c1 = 1.0f - powf(beta1, (float)t), c2 = 1.0f - powf(beta2, (float)t);
  mlp_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, (cudaStream_t)cuda_stream>>>(
      params, params_bf16, grad, m, v, lr, beta1, beta2, eps, c1, c2);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ADG_OK : mfail(ADG_ERR_CUDA, cudaGetErrorString(e));
}

adg_status adg_mlp_to_bf16(const float* params, uint16_t* params_bf16, void* cuda_stream) {
  if (!params || !params_bf16) return mfail(ADG_ERR_INVALID, "bad arguments");
  to_bf16_kernel<<<(kMlpParams + 255) / 256, 256, 0, (cudaStream_t)cuda_stream>>>(params, params_bf16, kMlpParams);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ADG_OK : mfail(ADG_ERR_CUDA, cudaGetErrorString(e));
}

int adg_mlp_num_params(void) { return kMlpParams; }

}  // extern "C"
