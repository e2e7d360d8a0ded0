// Persistent fused gradient pass over the row blocks of many problems (see batch.cuh).  Per
// item the sweep is that of the single-problem pass (grad.cu): the rank-M form
// W_ab = sum_m a_m[a] b_m[b] for four j's from vectorised shared loads, the kernel value and
// the squared prescaled differences, FP32 sums over a j-tile folded into FP64 across tiles.
// The item's FP64 sums go to its own slot; a second launch sums each problem's slots in
// row-block order (deterministic) and applies lambda to the diagonal component.
#include <algorithm>
#include <mutex>

#include "batch.cuh"
#include "kmv_kernel.cuh"

namespace ulisse {

constexpr int kGBatchXStage = kBN * kBatchMaxDP;

template <int DP, int M>
__device__ __forceinline__ bool grad_batch_item(const BatchGradDesc& P, int rb, int slot,
                                                float* sX, float* sB, uint64_t* bar,
                                                const int* s_bcol, uint32_t& g,
                                                double (*s_red)[kMaxD + 2], double* partials) {
  constexpr int NT = kBatchNT, TM = kBatchTM, BM = kBatchBM, NW = NT / 32;
  constexpr int NACC = DP + 2;
  const int tid = threadIdx.x;
  const long long n = P.n;
  const long long row0 = (long long)rb * BM;
  const int nt = (int)((n + kBN - 1) / kBN);
  const int Ma = P.M;
  const uint32_t g0 = g;
  const uint32_t tile_bytes = (uint32_t)(kBN * DP * sizeof(float) + Ma * kBN * sizeof(float));
  auto issue = [&](int lt) {
    const int s = (int)((g0 + (uint32_t)lt) % kStages);
    const long long j0 = (long long)lt * kBN;
    mbar_arrive_expect_tx(&bar[s], tile_bytes);
    bulk_g2s(sX + s * kGBatchXStage, P.xhat + j0 * DP, kBN * DP * sizeof(float), &bar[s]);
    for (int m = 0; m < Ma; ++m)
      bulk_g2s(sB + (s * M + m) * kBN, P.B + (long long)s_bcol[m] * P.ld + j0,
               kBN * sizeof(float), &bar[s]);
  };
  int issued = 0;
  if (tid == 0)
    for (; issued < min(kStages, nt); ++issued) issue(issued);

  const float c0 = P.params->c0f, c1 = P.params->c1f;
  float xi[TM][DP];
  float av[TM][M];
#pragma unroll
  for (int t = 0; t < TM; ++t) {
    const long long i = row0 + t * NT + tid;
    if (i < n) {
      load_row<float, DP>(P.xhat + i * DP, xi[t]);
    } else {
#pragma unroll
      for (int k = 0; k < DP; ++k) xi[t][k] = 0.f;
    }
#pragma unroll
    for (int m = 0; m < M; ++m)
      av[t][m] = (m < Ma && i < n) ? P.sa[m] * P.A[(long long)P.amap[m] * P.ld + i] : 0.f;
  }
  double acc[NACC];
#pragma unroll
  for (int k = 0; k < NACC; ++k) acc[k] = 0.0;

  for (int lt = 0; lt < nt; ++lt) {
    const uint32_t gg = g0 + (uint32_t)lt;
    const int s = (int)(gg % kStages);
    const bool ok = mbar_wait_bounded(&bar[s], (gg / kStages) & 1u);
    if (ok) {
      const float* tX = sX + s * kGBatchXStage;
      const float* tB = sB + s * M * kBN;
      float gl[DP];
      float gs = 0.f;
#pragma unroll
      for (int k = 0; k < DP; ++k) gl[k] = 0.f;
#pragma unroll 1
      for (int jq = 0; jq < kBN; jq += 4) {
        float W[TM][4];
#pragma unroll
        for (int t = 0; t < TM; ++t)
#pragma unroll
          for (int q = 0; q < 4; ++q) W[t][q] = 0.f;
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const float4 b4 = *reinterpret_cast<const float4*>(tB + m * kBN + jq);
#pragma unroll
          for (int t = 0; t < TM; ++t) {
            W[t][0] = fmaf(av[t][m], b4.x, W[t][0]);
            W[t][1] = fmaf(av[t][m], b4.y, W[t][1]);
            W[t][2] = fmaf(av[t][m], b4.z, W[t][2]);
            W[t][3] = fmaf(av[t][m], b4.w, W[t][3]);
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float xj[DP];
          load_row<float, DP>(tX + (jq + q) * DP, xj);
#pragma unroll
          for (int t = 0; t < TM; ++t) {
            float sq[DP];
            float dist = 0.f;
#pragma unroll
            for (int k = 0; k < DP; ++k) {
              const float df = xi[t][k] - xj[k];
              sq[k] = df * df;
              dist += sq[k];
            }
            const float Pv = ex2_approx(fmaf(-c1, dist, c0)) * W[t][q];
            gs += Pv;
#pragma unroll
            for (int k = 0; k < DP; ++k) gl[k] = fmaf(Pv, sq[k], gl[k]);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < DP; ++k) acc[k] += (double)gl[k];
      acc[DP] += (double)gs;
    }
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        for (int lt2 = max(0, issued - kStages); lt2 < issued; ++lt2) {
          const uint32_t g2 = g0 + (uint32_t)lt2;
          (void)mbar_wait_bounded(&bar[g2 % kStages], (g2 / kStages) & 1u);
        }
      }
      return false;
    }
    if (tid == 0 && issued < nt) issue(issued++);
  }
  g = g0 + (uint32_t)nt;

  // Diagonal W_aa for the lambda component.
#pragma unroll
  for (int t = 0; t < TM; ++t) {
    const long long i = row0 + t * NT + tid;
    if (i >= n) continue;
    float w = 0.f;
#pragma unroll
    for (int m = 0; m < M; ++m)
      if (m < Ma) w = fmaf(av[t][m], P.B[(long long)s_bcol[m] * P.ld + i], w);
    acc[DP + 1] += (double)w;
  }
  const int w = tid >> 5, lane = tid & 31;
#pragma unroll
  for (int k = 0; k < NACC; ++k) {
    const double v = warp_sum(acc[k]);
    if (lane == 0) s_red[w][k] = v;
  }
  __syncthreads();
  double* part = partials + (long long)slot * kMaxP;
  if (tid < NACC) {
    double v = 0.0;
    for (int ww = 0; ww < NW; ++ww) v += s_red[ww][tid];
    // slots: lengthscales 0..d-1, then sigma^2 at d, lambda at d+1
    if (tid < P.d) part[tid] = v;
    else if (tid == DP) part[P.d] = v;
    else if (tid == DP + 1) part[P.d + 1] = v;
  }
  return true;
}

template <int M>
__global__ void __launch_bounds__(kBatchNT) grad_batch_kernel(const BatchGradDesc* __restrict__ descs,
                                                              const BatchItem* __restrict__ items,
                                                              int n_items, int* queue,
                                                              double* __restrict__ partials,
                                                              int* status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* sX = reinterpret_cast<float*>(smem_raw);
  float* sB = sX + kStages * kGBatchXStage;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sB + kStages * M * kBN);
  __shared__ int s_bcol[M];
  __shared__ int s_item;
  __shared__ double s_red[kBatchNT / 32][kMaxD + 2];
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
    fence_barrier_init();
  }
  __syncthreads();
  uint32_t g = 0;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(queue, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const BatchItem item = items[it];
    const BatchGradDesc P = descs[item.prob];
    const int Ma = min(P.M, M);
    if (tid < M) s_bcol[tid] = (tid < Ma) ? P.bmap[tid] : 0;
    for (int idx = tid; idx < kStages * (M - Ma) * kBN; idx += kBatchNT) {
      const int st = idx / ((M - Ma) * kBN);
      const int rem = idx - st * (M - Ma) * kBN;
      sB[(st * M + Ma) * kBN + rem] = 0.f;
    }
    __syncthreads();
    bool ok = true;
    switch (P.DP) {
      case 2: ok = grad_batch_item<2, M>(P, item.rb, item.slot, sX, sB, bar, s_bcol, g, s_red, partials); break;
      case 4: ok = grad_batch_item<4, M>(P, item.rb, item.slot, sX, sB, bar, s_bcol, g, s_red, partials); break;
      default: ok = grad_batch_item<8, M>(P, item.rb, item.slot, sX, sB, bar, s_bcol, g, s_red, partials); break;
    }
    if (!ok) {
      if (tid == 0) atomicOr(status, kStatusTimeout);
      return;
    }
    __syncthreads();   // s_item, s_bcol and s_red are rewritten by the next item
  }
}

// One CTA per problem: g[k] = sum over its slots in order (times lambda for the last one).
__global__ void grad_batch_reduce_kernel(const BatchGradDesc* __restrict__ descs,
                                         const double* __restrict__ partials) {
  const BatchGradDesc P = descs[blockIdx.x];
  const int p = P.d + 2;
  const int k = threadIdx.x;
  if (k >= p) return;
  double v = 0.0;
  for (int r = 0; r < P.n_slots; ++r) v += partials[(long long)(P.slot0 + r) * kMaxP + k];
  if (k == p - 1) v *= P.params->lambda;
  P.g_out[k] = v;
}

template <int M>
static size_t grad_batch_smem() {
  return (size_t)kStages * (kGBatchXStage + M * kBN) * sizeof(float) + kStages * sizeof(uint64_t);
}

template <int M>
static int grad_batch_occupancy() {
  static int occ = 1;
  static std::once_flag once;
  std::call_once(once, [] {
    auto fn = grad_batch_kernel<M>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_batch_smem<M>());
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, kBatchNT, grad_batch_smem<M>()) !=
        cudaSuccess)
      o = 1;
    occ = std::max(o, 1);
  });
  return occ;
}

template <int M>
static cudaError_t grad_batch_launch(const BatchGradDesc* descs, const BatchItem* items,
                                     int n_items, int* queue, double* partials, int num_sms,
                                     int* status, cudaStream_t s) {
  const int grid = std::max(1, std::min(n_items, num_sms * grad_batch_occupancy<M>()));
  grad_batch_kernel<M><<<grid, kBatchNT, grad_batch_smem<M>(), s>>>(descs, items, n_items, queue,
                                                                   partials, status);
  return cudaGetLastError();
}

void prime_grad_batch() {
  (void)grad_batch_occupancy<5>();
  (void)grad_batch_occupancy<9>();
  (void)grad_batch_occupancy<17>();
}

cudaError_t launch_grad_batch(const BatchGradDesc* descs, int n_probs, const BatchItem* items,
                              int n_items, int* queue, double* partials, int M, int num_sms,
                              int* status, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (M <= 5) e = grad_batch_launch<5>(descs, items, n_items, queue, partials, num_sms, status, s);
  else if (M <= 9) e = grad_batch_launch<9>(descs, items, n_items, queue, partials, num_sms, status, s);
  else if (M <= 17) e = grad_batch_launch<17>(descs, items, n_items, queue, partials, num_sms, status, s);
  else return cudaErrorInvalidValue;
  if (e != cudaSuccess) return e;
  grad_batch_reduce_kernel<<<n_probs, 32, 0, s>>>(descs, partials);
  return cudaGetLastError();
}

}  // namespace ulisse
