// Fused per-stage kernels instantiated for the df64 arithmetic.
#include "fused.cuh"

namespace adg {

cudaError_t launch_fused_df64(int dim, int N, const FusedArgs& a, const CUtensorMap& tw,
                            const CUtensorMap& tx, cudaStream_t s) {
  return FusedDispatch<df64>::run(dim, N, a, tw, tx, s);
}

}  // namespace adg
