// Fused per-stage kernels instantiated for the float arithmetic.
#include "fused.cuh"

namespace adg {

cudaError_t launch_fused_fp32(int dim, int N, const FusedArgs& a, const CUtensorMap& tw,
                            const CUtensorMap& tx, cudaStream_t s) {
  return FusedDispatch<float>::run(dim, N, a, tw, tx, s);
}

}  // namespace adg
