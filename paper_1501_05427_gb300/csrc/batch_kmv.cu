// Persistent K V over the row blocks of many problems (see batch.cuh).  Per item the tile
// loop is that of the single-problem kernel (kmv_kernel.cuh, mode K): bulk copies of x^_J and
// of the live columns' V_J into a kStages-deep mbarrier ring, kernel values for two rows and
// four j's at a time, contraction from registers (per-tile sums folded into running totals).  The ring carries on across items: a CTA
// counts every tile it consumes, and that count gives the stage and the parity of the next
// wait, so the barriers are initialised once per CTA.  The input width DP (2, 4 or 8) is
// chosen per item.
#include <algorithm>
#include <mutex>

#include "batch.cuh"
#include "kmv_kernel.cuh"

namespace ulisse {

constexpr int kBatchXStage = kBN * kBatchMaxDP;   // floats of x^ per stage

template <int DP, int R>
__device__ __forceinline__ bool kmv_batch_item(const BatchKmvDesc& P, int rb, int Ra,
                                               float* sX, float* sV, uint64_t* bar,
                                               const int* s_vcol, uint32_t& g) {
  constexpr int NT = kBatchNT, TM = kBatchTM, BM = kBatchBM;
  const int tid = threadIdx.x;
  const long long n = P.n;
  const long long row0 = (long long)rb * BM;
  const int nt = (int)((n + kBN - 1) / kBN);
  const uint32_t g0 = g;
  const uint32_t tile_bytes = (uint32_t)(kBN * DP * sizeof(float) + Ra * kBN * sizeof(float));
  auto issue = [&](int lt) {
    const int s = (int)((g0 + (uint32_t)lt) % kStages);
    const long long j0 = (long long)lt * kBN;
    mbar_arrive_expect_tx(&bar[s], tile_bytes);
    bulk_g2s(sX + s * kBatchXStage, P.xhat + j0 * DP, kBN * DP * sizeof(float), &bar[s]);
    for (int r = 0; r < Ra; ++r)
      bulk_g2s(sV + (s * R + r) * kBN, P.V + (long long)s_vcol[r] * P.ldv + j0,
               kBN * sizeof(float), &bar[s]);
  };
  int issued = 0;  // thread 0 only
  if (tid == 0)
    for (; issued < min(kStages, nt); ++issued) issue(issued);

  const float c0 = P.params->c0f, c1 = P.params->c1f;
  const float lam = P.params->lambdaf;
  float xi[TM][DP];
#pragma unroll
  for (int t = 0; t < TM; ++t) {
    const long long i = row0 + t * NT + tid;
    if (i < n) {
      load_row<float, DP>(P.xhat + i * DP, xi[t]);
    } else {
#pragma unroll
      for (int k = 0; k < DP; ++k) xi[t][k] = 0.f;
    }
  }
  float acc[TM][R];
#pragma unroll
  for (int t = 0; t < TM; ++t)
#pragma unroll
    for (int r = 0; r < R; ++r) acc[t][r] = 0.f;

  for (int lt = 0; lt < nt; ++lt) {
    const uint32_t gg = g0 + (uint32_t)lt;
    const int s = (int)(gg % kStages);
    const bool ok = mbar_wait_bounded(&bar[s], (gg / kStages) & 1u);
    if (ok) {
      const float* tX = sX + s * kBatchXStage;
      const float* tV = sV + s * R * kBN;
      // one tile's sums apart, then folded into the running totals: the rounding of a
      // row's sum grows with the number of tiles (n / 64), not with n
      float tacc[TM][R];
#pragma unroll
      for (int t = 0; t < TM; ++t)
#pragma unroll
        for (int r = 0; r < R; ++r) tacc[t][r] = 0.f;
#pragma unroll 1
      for (int jq = 0; jq < kBN; jq += 4) {
        float kq[TM][4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float xj[DP];
          load_row<float, DP>(tX + (jq + q) * DP, xj);
#pragma unroll
          for (int t = 0; t < TM; ++t) {
            float dist = 0.f;
#pragma unroll
            for (int k = 0; k < DP; ++k) {
              const float df = xi[t][k] - xj[k];
              dist = fmaf(df, df, dist);
            }
            kq[t][q] = ex2_approx(fmaf(-c1, dist, c0));
          }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const float4 w = *reinterpret_cast<const float4*>(tV + r * kBN + jq);
#pragma unroll
          for (int t = 0; t < TM; ++t) {
            float u = tacc[t][r];
            u = fmaf(kq[t][0], w.x, u);
            u = fmaf(kq[t][1], w.y, u);
            u = fmaf(kq[t][2], w.z, u);
            u = fmaf(kq[t][3], w.w, u);
            tacc[t][r] = u;
          }
        }
      }
#pragma unroll
      for (int t = 0; t < TM; ++t)
#pragma unroll
        for (int r = 0; r < R; ++r) acc[t][r] += tacc[t][r];
    }
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        // Let copies still in flight land before the CTA's shared memory is released.
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
#pragma unroll
  for (int t = 0; t < TM; ++t) {
    const long long i = row0 + t * NT + tid;
    if (i >= n) continue;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r >= Ra) break;
      const float u = fmaf(lam, P.V[(long long)s_vcol[r] * P.ldv + i], acc[t][r]);
      P.U[(long long)P.umap[r] * P.ldu + i] = u;
    }
  }
  return true;
}

template <int R>
__global__ void __launch_bounds__(kBatchNT) kmv_batch_kernel(const BatchKmvDesc* __restrict__ descs,
                                                             const BatchItem* __restrict__ items,
                                                             int n_items, int* queue, int* status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* sX = reinterpret_cast<float*>(smem_raw);
  float* sV = sX + kStages * kBatchXStage;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sV + kStages * R * kBN);
  __shared__ int s_vcol[R];
  __shared__ int s_item;
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
    const BatchKmvDesc P = descs[item.prob];
    const int Ra = min(*P.nlive, R);
    if (Ra > 0) {
      if (tid < R) s_vcol[tid] = (tid < Ra) ? P.vmap[tid] : 0;
      // Column slots beyond the live count read as zero in every stage.
      for (int idx = tid; idx < kStages * (R - Ra) * kBN; idx += kBatchNT) {
        const int st = idx / ((R - Ra) * kBN);
        const int rem = idx - st * (R - Ra) * kBN;
        sV[(st * R + Ra) * kBN + rem] = 0.f;
      }
      __syncthreads();
      bool ok = true;
      switch (P.DP) {
        case 2: ok = kmv_batch_item<2, R>(P, item.rb, Ra, sX, sV, bar, s_vcol, g); break;
        case 4: ok = kmv_batch_item<4, R>(P, item.rb, Ra, sX, sV, bar, s_vcol, g); break;
        default: ok = kmv_batch_item<8, R>(P, item.rb, Ra, sX, sV, bar, s_vcol, g); break;
      }
      if (!ok) {
        if (tid == 0) atomicOr(status, kStatusTimeout);
        return;
      }
    }
    __syncthreads();   // s_item and s_vcol are rewritten by the next item
  }
}

template <int R>
static size_t kmv_batch_smem() {
  return (size_t)kStages * (kBatchXStage + R * kBN) * sizeof(float) + kStages * sizeof(uint64_t);
}

template <int R>
static int kmv_batch_occupancy() {
  static int occ = 1;
  static std::once_flag once;
  std::call_once(once, [] {
    auto fn = kmv_batch_kernel<R>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kmv_batch_smem<R>());
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, kBatchNT, kmv_batch_smem<R>()) !=
        cudaSuccess)
      o = 1;
    occ = std::max(o, 1);
  });
  return occ;
}

template <int R>
static cudaError_t kmv_batch_launch(const BatchKmvDesc* descs, const BatchItem* items,
                                    int n_items, int* queue, int num_sms, int* status,
                                    cudaStream_t s) {
  const int grid = std::max(1, std::min(n_items, num_sms * kmv_batch_occupancy<R>()));
  kmv_batch_kernel<R><<<grid, kBatchNT, kmv_batch_smem<R>(), s>>>(descs, items, n_items, queue,
                                                                 status);
  return cudaGetLastError();
}

void prime_kmv_batch() {
  (void)kmv_batch_occupancy<2>();
  (void)kmv_batch_occupancy<4>();
  (void)kmv_batch_occupancy<9>();
  (void)kmv_batch_occupancy<17>();
  (void)kmv_batch_occupancy<32>();
}

cudaError_t launch_kmv_batch(const BatchKmvDesc* descs, const BatchItem* items, int n_items,
                             int* queue, int R_max, int num_sms, int* status, cudaStream_t s) {
  if (n_items <= 0 || R_max <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (R_max <= 2) return kmv_batch_launch<2>(descs, items, n_items, queue, num_sms, status, s);
  if (R_max <= 4) return kmv_batch_launch<4>(descs, items, n_items, queue, num_sms, status, s);
  if (R_max <= 9) return kmv_batch_launch<9>(descs, items, n_items, queue, num_sms, status, s);
  if (R_max <= 17) return kmv_batch_launch<17>(descs, items, n_items, queue, num_sms, status, s);
  if (R_max <= 32) return kmv_batch_launch<32>(descs, items, n_items, queue, num_sms, status, s);
  return cudaErrorInvalidValue;
}

}  // namespace ulisse
