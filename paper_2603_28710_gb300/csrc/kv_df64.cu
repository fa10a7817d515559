// Volume kernels with element-local face fluxes, instantiated for the df64 arithmetic.
#include "kernels.cuh"

namespace adg {

cudaError_t launch_vol_faces_df64(int dim, int N, const FusedArgs& a, cudaStream_t s) {
  return Dispatch<df64>::run_vol_faces(dim, N, a, s);
}

}  // namespace adg
