// Learned ghost-trace predictor: a small MLP, 4 inputs -> 64 -> 64 -> 1, tanh hidden
// activations, BF16 weights read into FP32 and FP32 accumulation everywhere.  Kernels for
// the mean-squared-error gradient of a sample set (forward + backward), an Adam step on
// FP32 master weights that refreshes their BF16 copy, and inference.
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

__global__ void mlp_forward_kernel(const uint16_t* __restrict__ pbf, const float* __restrict__ x,
                                   int n, float* __restrict__ y) {
  __shared__ float W[4548];
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) W[i] = bf16_to_float(pbf[i]);
  __syncthreads();
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    float xi[4] = {x[(size_t)s * 4], x[(size_t)s * 4 + 1], x[(size_t)s * 4 + 2], x[(size_t)s * 4 + 3]};
    y[s] = mlp_eval(W, xi);
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
  const int blocks = (int)((n + 255) / 256) < 152 * 8 ? (int)((n + 255) / 256) : 152 * 8;
  mlp_forward_kernel<<<blocks, 256, 0, s>>>(params, x, (int)n, y);
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
  const int blocks = (int)((n + 255) / 256) < 152 * 8 ? (int)((n + 255) / 256) : 152 * 8;
  mlp_forward_kernel<<<blocks, 256, 0, (cudaStream_t)cuda_stream>>>(params_bf16, x, (int)n, y);
  cudaError_t e = cudaGetLastError();
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
