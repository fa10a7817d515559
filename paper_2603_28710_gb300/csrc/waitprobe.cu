// Check of the bounded device-side wait (adg_probe_wait in include/adg.h): the fused and
// element-path kernels wait for their tiles' TMA copies on an mbarrier with a time limit
// (mbar_wait_bounded) and report a wait that gave up through an error flag instead of
// hanging.  This probe runs that same wait on a barrier nothing ever arrives at, so that the
// give-up path can be exercised without a fault: every thread must give up after the limit.
#include <string>

#include "../../include/adg.h"
#include "kernels.cuh"

namespace adg {
void noalloc_set_error(const char* msg);

namespace {

__global__ void wait_probe_kernel(long long limit, int* gave_up, long long* cycles) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);  // expects one arrival that never comes
  __syncthreads();
  const long long t0 = clock64();
  const bool done = mbar_wait_bounded(&bar, 0, limit);
  const long long t1 = clock64();
  if (!done) atomicAdd(gave_up, 1);
  if (threadIdx.x == 0) *cycles = t1 - t0;
}

}  // namespace
}  // namespace adg

extern "C" adg_status adg_probe_wait(int64_t limit_cycles, int* threads_gave_up, int64_t* cycles) {
  if (limit_cycles <= 0 || limit_cycles > 4000000000ll || !threads_gave_up) {
    adg::noalloc_set_error("adg_probe_wait: need 0 < limit_cycles <= 4e9 and threads_gave_up");
    return ADG_ERR_INVALID;
  }
  int* buf = nullptr;
  cudaStream_t s = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc((void**)&buf, 16);
  if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, 16, s);
  long long* clk = reinterpret_cast<long long*>(buf + 2);
  if (e == cudaSuccess) {
    adg::wait_probe_kernel<<<1, 128, 0, s>>>((long long)limit_cycles, buf, clk);
    e = cudaGetLastError();
  }
  int n = 0;
  long long c = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&n, buf, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&c, clk, sizeof(long long), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (buf) cudaFree(buf);
  if (s) cudaStreamDestroy(s);
  if (e != cudaSuccess) {
    adg::noalloc_set_error((std::string("adg_probe_wait: ") + cudaGetErrorString(e)).c_str());
    return ADG_ERR_CUDA;
  }
  *threads_gave_up = n;
  if (cycles) *cycles = c;
  return ADG_OK;
}
