// Operator kernels instantiated for the float arithmetic.
#include "kernels.cuh"

namespace adg {

cudaError_t launch_trace_fp32(int dim, int N, const TraceArgs& a, cudaStream_t s) {
  return Dispatch<float>::run_trace(dim, N, a, s);
}
cudaError_t launch_flux_fp32(int dim, int N, const FluxArgs& a, cudaStream_t s) {
  return Dispatch<float>::run_flux(dim, N, a, s);
}
cudaError_t launch_vol_fp32(int dim, int N, const VolArgs& a, cudaStream_t s) {
  return Dispatch<float>::run_vol(dim, N, a, s);
}

}  // namespace adg
