// Fused per-stage kernels instantiated for the double arithmetic.
#include "fused.cuh"

namespace adg {

cudaError_t launch_fused_fp64(int dim, int N, const FusedArgs& a, const CUtensorMap& tw,
                            const CUtensorMap& tx, cudaStream_t s) {
  return FusedDispatch<double>::run(dim, N, a, tw, tx, s);
}

bool fused_tile(int dim, int N, int* t) {
#define ADG_TILE(DD, NN)          \
  if (dim == DD && N == NN) {     \
    t[0] = FT<DD, NN>::TX;        \
    t[1] = FT<DD, NN>::TY;        \
    t[2] = FT<DD, NN>::TZ;        \
    return true;                  \
  }
  ADG_TILE(2, 2) ADG_TILE(2, 3) ADG_TILE(2, 4) ADG_TILE(2, 5) ADG_TILE(2, 6) ADG_TILE(2, 7)
  ADG_TILE(2, 8) ADG_TILE(3, 2) ADG_TILE(3, 3) ADG_TILE(3, 4) ADG_TILE(3, 5) ADG_TILE(3, 6)
#undef ADG_TILE
  return false;
}

}  // namespace adg
