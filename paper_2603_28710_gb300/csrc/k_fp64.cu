// Operator kernels instantiated for the double arithmetic.
#include "kernels.cuh"

namespace adg {

cudaError_t launch_trace_fp64(int dim, int N, const TraceArgs& a, cudaStream_t s) {
  return Dispatch<double>::run_trace(dim, N, a, s);
}
cudaError_t launch_flux_fp64(int dim, int N, const FluxArgs& a, cudaStream_t s) {
  return Dispatch<double>::run_flux(dim, N, a, s);
}
cudaError_t launch_vol_fp64(int dim, int N, const VolArgs& a, cudaStream_t s) {
  return Dispatch<double>::run_vol(dim, N, a, s);
}

}  // namespace adg
