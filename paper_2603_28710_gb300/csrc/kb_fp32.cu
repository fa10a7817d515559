// Batched kernels instantiated for the float arithmetic.
#include "batch.cuh"

namespace adg {

cudaError_t batch_vol_fp32(int dim, int N, int tt, const VolArgs* va, const FluxArgs* fa, int ns,
                              int st, const BatchGroupArgs& g, int grid, cudaStream_t s, int* occ) {
  return BatchDispatch<float>::vol(dim, N, tt, va, fa, ns, st, g, grid, s, occ);
}
cudaError_t batch_flux_fp32(int dim, int N, const FluxArgs* fa, int ns, int st,
                               const BatchGroupArgs& g, int grid, cudaStream_t s, int* occ) {
  return BatchDispatch<float>::flux(dim, N, fa, ns, st, g, grid, s, occ);
}

}  // namespace adg
