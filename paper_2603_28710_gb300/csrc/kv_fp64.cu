// Volume kernels with element-local face fluxes, instantiated for the double arithmetic.
#include "kernels.cuh"

namespace adg {

cudaError_t launch_vol_faces_fp64(int dim, int N, const FusedArgs& a, cudaStream_t s) {
  return Dispatch<double>::run_vol_faces(dim, N, a, s);
}

}  // namespace adg
