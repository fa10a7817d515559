// Operator kernels instantiated for the FP32-pair arithmetic (df64.cuh).
#include "kernels.cuh"

namespace adg {

cudaError_t launch_trace_df64(int dim, int N, const TraceArgs& a, cudaStream_t s) {
  return Dispatch<df64>::run_trace(dim, N, a, s);
}
cudaError_t launch_flux_df64(int dim, int N, const FluxArgs& a, cudaStream_t s) {
  return Dispatch<df64>::run_flux(dim, N, a, s);
}
cudaError_t launch_vol_df64(int dim, int N, const VolArgs& a, cudaStream_t s) {
  return Dispatch<df64>::run_vol(dim, N, a, s);
}

}  // namespace adg
