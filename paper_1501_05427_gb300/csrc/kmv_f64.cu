// FP64 instantiations of the tile-generating K V kernel (the paper's double-precision CMVPs).
#include "kmv_launch.cuh"

namespace ulisse {

using RF64 = RList<1, 2, 4, 5, 8, 16, 32>;
using RF64D = RList<1, 4, 8, 32>;

cudaError_t launch_kmv_f64(KmvLaunch& L, cudaStream_t s) {
  if (L.R < 1 || L.R > kMaxRChunk) return cudaErrorInvalidValue;
  switch (L.DP) {
    case 2: return dispatch_mode<double, 2, 1, 1, RF64, RF64D>(L, s);
    case 4: return dispatch_mode<double, 4, 1, 1, RF64, RF64D>(L, s);
    case 8: return dispatch_mode<double, 8, 1, 1, RF64, RF64D>(L, s);
    case 16: return dispatch_mode<double, 16, 1, 1, RF64, RF64D>(L, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ulisse
