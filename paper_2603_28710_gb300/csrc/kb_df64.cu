// Batched kernels instantiated for the df64 arithmetic.
#include "batch.cuh"

namespace adg {

cudaError_t batch_vol_df64(int dim, int N, int tt, const VolArgs* va, const FluxArgs* fa, int ns,
                              int st, const BatchGroupArgs& g, int grid, cudaStream_t s, int* occ) {
  return BatchDispatch<df64>::vol(dim, N, tt, va, fa, ns, st, g, grid, s, occ);
}
cudaError_t batch_flux_df64(int dim, int N, const FluxArgs* fa, int ns, int st,
                               const BatchGroupArgs& g, int grid, cudaStream_t s, int* occ) {
  return BatchDispatch<df64>::flux(dim, N, fa, ns, st, g, grid, s, occ);
}

}  // namespace adg
