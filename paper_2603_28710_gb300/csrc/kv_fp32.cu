// Volume kernels with element-local face fluxes, instantiated for the float arithmetic.
#include "kernels.cuh"

namespace adg {

cudaError_t launch_vol_faces_fp32(int dim, int N, const FusedArgs& a, cudaStream_t s) {
  return Dispatch<float>::run_vol_faces(dim, N, a, s);
}

}  // namespace adg
