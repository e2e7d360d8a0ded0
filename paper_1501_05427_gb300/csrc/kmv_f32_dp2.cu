// FP32 instantiations of the tile-generating K V kernel for inputs padded to 2 dimensions.
#include "kmv_launch.cuh"

namespace ulisse {

cudaError_t launch_kmv_f32_dp2(KmvLaunch& L, cudaStream_t s) {
  using RK = RList<1, 2, 3, 4, 5, 6, 8, 9, 12, 16, 17, 20, 24, 32>;
  using RD = RList<1, 2, 4, 8, 16, 32>;
  return dispatch_mode<float, 2, 2, 4, RK, RD>(L, s);
}

}  // namespace ulisse
