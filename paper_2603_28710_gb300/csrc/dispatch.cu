// Selects the kernel set of an operator arithmetic (0 = FP64, 1 = FP32, 2 = FP32 pair).
#include "adg_internal.h"

namespace adg {

cudaError_t launch_trace_fp64(int, int, const TraceArgs&, cudaStream_t);
cudaError_t launch_flux_fp64(int, int, const FluxArgs&, cudaStream_t);
cudaError_t launch_vol_fp64(int, int, const VolArgs&, cudaStream_t);
cudaError_t launch_trace_fp32(int, int, const TraceArgs&, cudaStream_t);
cudaError_t launch_flux_fp32(int, int, const FluxArgs&, cudaStream_t);
cudaError_t launch_vol_fp32(int, int, const VolArgs&, cudaStream_t);
cudaError_t launch_trace_df64(int, int, const TraceArgs&, cudaStream_t);
cudaError_t launch_flux_df64(int, int, const FluxArgs&, cudaStream_t);
cudaError_t launch_vol_df64(int, int, const VolArgs&, cudaStream_t);

cudaError_t launch_fused_fp64(int, int, const FusedArgs&, const CUtensorMap&, const CUtensorMap&,
                              cudaStream_t);
cudaError_t launch_fused_fp32(int, int, const FusedArgs&, const CUtensorMap&, const CUtensorMap&,
                              cudaStream_t);
cudaError_t launch_fused_df64(int, int, const FusedArgs&, const CUtensorMap&, const CUtensorMap&,
                              cudaStream_t);

cudaError_t launch_vol_faces_fp64(int, int, const FusedArgs&, cudaStream_t);
cudaError_t launch_vol_faces_fp32(int, int, const FusedArgs&, cudaStream_t);
cudaError_t launch_vol_faces_df64(int, int, const FusedArgs&, cudaStream_t);

cudaError_t launch_vol_faces(int prec, int dim, int N, const FusedArgs& a, cudaStream_t s) {
  switch (prec) {
    case 0: return launch_vol_faces_fp64(dim, N, a, s);
    case 1: return launch_vol_faces_fp32(dim, N, a, s);
    case 2: return launch_vol_faces_df64(dim, N, a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_fused(int prec, int dim, int N, const FusedArgs& a, const CUtensorMap& tw,
                         const CUtensorMap& tx, cudaStream_t s) {
  switch (prec) {
    case 0: return launch_fused_fp64(dim, N, a, tw, tx, s);
    case 1: return launch_fused_fp32(dim, N, a, tw, tx, s);
    case 2: return launch_fused_df64(dim, N, a, tw, tx, s);
  }
  return cudaErrorInvalidValue;
}

bool kernels_available(int prec, int dim, int N) {
  if (prec < 0 || prec > 2) return false;
  if (dim == 2) return N >= 2 && N <= 8;
  if (dim == 3) return N >= 2 && N <= 6;
  return false;
}

size_t storage_bytes(int prec) { return prec == 1 ? sizeof(float) : (prec == 2 ? sizeof(float2) : sizeof(double)); }

cudaError_t launch_trace(int prec, int dim, int N, const TraceArgs& a, cudaStream_t s) {
  switch (prec) {
    case 0: return launch_trace_fp64(dim, N, a, s);
    case 1: return launch_trace_fp32(dim, N, a, s);
    case 2: return launch_trace_df64(dim, N, a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_flux(int prec, int dim, int N, const FluxArgs& a, cudaStream_t s) {
  switch (prec) {
    case 0: return launch_flux_fp64(dim, N, a, s);
    case 1: return launch_flux_fp32(dim, N, a, s);
    case 2: return launch_flux_df64(dim, N, a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_vol(int prec, int dim, int N, const VolArgs& a, cudaStream_t s) {
  switch (prec) {
    case 0: return launch_vol_fp64(dim, N, a, s);
    case 1: return launch_vol_fp32(dim, N, a, s);
    case 2: return launch_vol_df64(dim, N, a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace adg
