// FP32 instantiations of the tile-generating K V kernel (SIMT, ex2 on the MUFU pipe).
#include "kmv_launch.cuh"

namespace ulisse {

using RF32 = RList<1, 2, 3, 4, 5, 6, 8, 9, 12, 16, 17, 20, 24, 32>;

cudaError_t launch_kmv_f32(KmvLaunch& L, cudaStream_t s) {
  if (L.R < 1 || L.R > kMaxRChunk) return cudaErrorInvalidValue;
  switch (L.DP) {
    case 2: return dispatch_r<float, 2, 2>(L, s, RF32{});
    case 4: return dispatch_r<float, 4, 2>(L, s, RF32{});
    case 8: return dispatch_r<float, 8, 2>(L, s, RF32{});
    case 16: return dispatch_r<float, 16, 2>(L, s, RF32{});
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ulisse
