// Device calibration for roofline reports: the throughput of the exponential unit.
//
// Every generated covariance entry exp(-1/2 sum_d (x_id - x_jd)^2 / l_d^2) needs one
// base-2 exponential (ex2.approx.ftz.f32); on the tensor-core path that is what remains on
// the CUDA cores, so its rate is the ceiling the tile-generating products are reported
// against.  This measures it on the device at hand instead of deriving it from unit counts.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/ulisse.h"

namespace {

constexpr int kChains = 16;     // independent exponentials in flight per thread
constexpr int kThreads = 256;

__device__ float g_ex2_sink;

// Each thread iterates x <- 2^(-x) on kChains independent values (bounded: the map has a
// fixed point near 0.64), so the loop issues kChains exponentials per iteration with no
// dependence between them; the sum is kept live through a store that never happens.
__global__ void __launch_bounds__(kThreads) ex2_rate_kernel(int iters) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1e-3f * (float)(threadIdx.x & 31) + 0.01f * (float)k;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      const float a = -x[k];
      asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(x[k]) : "f"(a));
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == -1.0f) g_ex2_sink = s;   // never true (every x is positive)
}

}  // namespace

extern "C" ulisse_status ulisse_measure_ex2_rate(void* stream, int reps, double* ex2_per_s,
                                                 double* best_ms) {
  if (!ex2_per_s || reps < 1 || reps > 1000) return ULISSE_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ULISSE_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return ULISSE_ERR_CUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ex2_rate_kernel, kThreads, 0) !=
      cudaSuccess)
    return ULISSE_ERR_CUDA;
  const int blocks = sms * std::max(per_sm, 1);
  const int iters = 4096;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return ULISSE_ERR_CUDA;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return ULISSE_ERR_CUDA;
  }
  ex2_rate_kernel<<<blocks, kThreads, 0, s>>>(iters / 8);   // warm-up
  float best = 0.f;
  cudaError_t e = cudaGetLastError();
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    cudaEventRecord(a, s);
    ex2_rate_kernel<<<blocks, kThreads, 0, s>>>(iters);
    cudaEventRecord(b, s);
    e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaGetLastError();
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess && (best == 0.f || ms < best)) best = ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess || best <= 0.f) return ULISSE_ERR_CUDA;
  const double count = (double)blocks * kThreads * (double)iters * kChains;
  *ex2_per_s = count / (best * 1e-3);
  if (best_ms) *best_ms = best;
  return ULISSE_OK;
}
