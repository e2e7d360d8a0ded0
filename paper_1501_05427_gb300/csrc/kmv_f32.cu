// FP32 tile-generating K V (SIMT, ex2 on the MUFU pipe): dispatch on the padded dimension.
#include "ulisse_internal.cuh"

namespace ulisse {

cudaError_t launch_kmv_f32(KmvLaunch& L, cudaStream_t s) {
  if (L.R < 1 || L.R > kMaxRChunk) return cudaErrorInvalidValue;
  switch (L.DP) {
    case 2: return launch_kmv_f32_dp2(L, s);
    case 4: return launch_kmv_f32_dp4(L, s);
    case 8: return launch_kmv_f32_dp8(L, s);
    case 16: return launch_kmv_f32_dp16(L, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ulisse
