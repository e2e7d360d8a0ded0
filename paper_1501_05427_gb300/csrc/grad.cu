// Fused gradient pass (Eq. gradient:unbiased, Sec. 4.1): one sweep over generated tiles of
// the covariance gives every component of
//     g~_i = sum_m a_m^T dK_i b_m,   a_0 = 1/2 a1, b_0 = a2,  a_j = -1/(2 N_r) z_j, b_j = r_j,
// through the rank-M form W_ab = sum_m a_m[a] b_m[b]:
//     g~_{log l_k}      = sum_ab k_s(a,b) W_ab (x^_ak - x^_bk)^2      (x^ = x / l)
//     g~_{log sigma^2}  = sum_ab k_s(a,b) W_ab
//     g~_{log lambda}   = lambda sum_a W_aa
// Tiles are staged like the K V kernel (bulk copies + mbarrier ring).  Each thread keeps
// its rows' a-values in registers, forms W for four j's from vectorised shared loads of b,
// and accumulates the p-1 tile sums in FP32 over one j-tile, then in FP64 across tiles.
// The CTAs' FP64 partials are summed in a fixed order by the last CTA to arrive.
#include "kmv_kernel.cuh"

#include <algorithm>
#include <mutex>

namespace ulisse {

constexpr int kGradNT = 128;

template <typename T>
struct GradDevArgs {
  const T* xhat;
  long long n, ldn;
  int d;
  const T* A;
  const int* amap;
  const T* sa;
  const T* B;
  const int* bmap;
  long long ld;
  int M;
  const DevParams* params;
  int nsplit, tiles_per_split, ntiles;
  double* partials;
  int* counter;
  double* g_out;
  int* status;
};

template <typename T, int DP, int M, int TM, int NT>
__global__ void __launch_bounds__(NT) grad_kernel(const GradDevArgs<T> a) {
  constexpr int BM = NT * TM;
  constexpr int NW = NT / 32;
  constexpr int NACC = DP + 2;  // DP lengthscale slots, sigma^2, lambda
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* sX = reinterpret_cast<T*>(smem_raw);
  T* sB = sX + kStages * kBN * DP;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sB + kStages * M * kBN);
  __shared__ int s_bcol[M];
  __shared__ double s_red[NW][NACC];
  __shared__ int s_last;

  const int tid = threadIdx.x;
  const int rb = blockIdx.x / a.nsplit;
  const int sp = blockIdx.x - rb * a.nsplit;
  const long long row0 = (long long)rb * BM;
  const int tile_begin = sp * a.tiles_per_split;
  const int tile_end = min(tile_begin + a.tiles_per_split, a.ntiles);
  const int nt_local = max(0, tile_end - tile_begin);
  const int Ma = a.M;
  const float c0 = a.params->c0f, c1 = a.params->c1f;
  const double sigma2 = a.params->sigma2;

  if (tid < M) s_bcol[tid] = (tid < Ma) ? a.bmap[tid] : 0;
  for (int idx = tid; idx < kStages * (M - Ma) * kBN; idx += NT) {
    const int st = idx / ((M - Ma) * kBN);
    const int rem = idx - st * (M - Ma) * kBN;
    sB[(st * M + Ma) * kBN + rem] = T(0);
  }
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
    fence_barrier_init();
  }
  __syncthreads();

  const uint32_t tile_bytes = (uint32_t)(kBN * DP * sizeof(T) + Ma * kBN * sizeof(T));
  auto issue = [&](int lt) {
    const int s = lt % kStages;
    const long long j0 = (long long)(tile_begin + lt) * kBN;
    mbar_arrive_expect_tx(&bar[s], tile_bytes);
    bulk_g2s(sX + s * kBN * DP, a.xhat + j0 * DP, kBN * DP * sizeof(T), &bar[s]);
    for (int m = 0; m < Ma; ++m)
      bulk_g2s(sB + (s * M + m) * kBN, a.B + (long long)s_bcol[m] * a.ld + j0,
               kBN * sizeof(T), &bar[s]);
  };
  int issued = 0;
  if (tid == 0)
    for (; issued < min(kStages, nt_local); ++issued) issue(issued);

  T xi[TM][DP];
  T av[TM][M];
#pragma unroll
  for (int t = 0; t < TM; ++t) {
    const long long i = row0 + t * NT + tid;
    if (i < a.n) {
      load_row<T, DP>(a.xhat + i * DP, xi[t]);
    } else {
#pragma unroll
      for (int k = 0; k < DP; ++k) xi[t][k] = T(0);
    }
#pragma unroll
    for (int m = 0; m < M; ++m)
      av[t][m] = (m < Ma && i < a.n) ? a.sa[m] * a.A[(long long)a.amap[m] * a.ld + i] : T(0);
  }

  double acc[NACC];
#pragma unroll
  for (int k = 0; k < NACC; ++k) acc[k] = 0.0;

  bool timed_out = false;
  for (int lt = 0; lt < nt_local; ++lt) {
    const int s = lt % kStages;
    const bool ok = mbar_wait_bounded(&bar[s], (uint32_t)((lt / kStages) & 1));
    if (ok) {
      const T* tX = sX + s * kBN * DP;
      const T* tB = sB + s * M * kBN;
      T gl[DP];
      T gs = T(0);
#pragma unroll
      for (int k = 0; k < DP; ++k) gl[k] = T(0);
#pragma unroll 1
      for (int jq = 0; jq < kBN; jq += 4) {
        T W[TM][4];
#pragma unroll
        for (int t = 0; t < TM; ++t)
#pragma unroll
          for (int q = 0; q < 4; ++q) W[t][q] = T(0);
#pragma unroll
        for (int m = 0; m < M; ++m) {
          T b[4];
          if constexpr (sizeof(T) == 4) {
            const float4 b4 = *reinterpret_cast<const float4*>(tB + m * kBN + jq);
            b[0] = b4.x; b[1] = b4.y; b[2] = b4.z; b[3] = b4.w;
          } else {
            const double2 b0 = *reinterpret_cast<const double2*>(tB + m * kBN + jq);
            const double2 b1 = *reinterpret_cast<const double2*>(tB + m * kBN + jq + 2);
            b[0] = b0.x; b[1] = b0.y; b[2] = b1.x; b[3] = b1.y;
          }
#pragma unroll
          for (int t = 0; t < TM; ++t)
#pragma unroll
            for (int q = 0; q < 4; ++q) W[t][q] = fma(av[t][m], b[q], W[t][q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          T xj[DP];
          load_row<T, DP>(tX + (jq + q) * DP, xj);
#pragma unroll
          for (int t = 0; t < TM; ++t) {
            T sq[DP];
            T dist = T(0);
#pragma unroll
            for (int k = 0; k < DP; ++k) {
              const T df = xi[t][k] - xj[k];
              sq[k] = df * df;
              dist += sq[k];
            }
            const T P = kernel_from_dist<T>(dist, c0, c1, sigma2) * W[t][q];
            gs += P;
#pragma unroll
            for (int k = 0; k < DP; ++k) gl[k] = fma(P, sq[k], gl[k]);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < DP; ++k) acc[k] += (double)gl[k];
      acc[DP] += (double)gs;
    }
    if (__syncthreads_or(!ok)) { timed_out = true; break; }
    if (tid == 0 && issued < nt_local) issue(issued++);
  }
  if (timed_out) {
    if (tid == 0) {
      atomicOr(a.status, kStatusTimeout);
      for (int lt2 = max(0, issued - kStages); lt2 < issued; ++lt2)
        (void)mbar_wait_bounded(&bar[lt2 % kStages], (uint32_t)((lt2 / kStages) & 1));
    }
    return;
  }

  // Diagonal W_aa for the lambda component: once per row (split 0 only).
  if (sp == 0) {
#pragma unroll
    for (int t = 0; t < TM; ++t) {
      const long long i = row0 + t * NT + tid;
      if (i >= a.n) continue;
      T w = T(0);
#pragma unroll
      for (int m = 0; m < M; ++m)
        if (m < Ma) w = fma(av[t][m], a.B[(long long)s_bcol[m] * a.ld + i], w);
      acc[DP + 1] += (double)w;
    }
  }

  // CTA reduction in a fixed order, then the last CTA sums all CTAs' partials in order.
  const int w = tid >> 5, lane = tid & 31;
#pragma unroll
  for (int k = 0; k < NACC; ++k) {
    const double v = warp_sum(acc[k]);
    if (lane == 0) s_red[w][k] = v;
  }
  __syncthreads();
  double* part = a.partials + (long long)blockIdx.x * kMaxP;
  if (tid < NACC) {
    double v = 0.0;
    for (int ww = 0; ww < NW; ++ww) v += s_red[ww][tid];
    // slots: lengthscales 0..d-1, then sigma^2 at d, lambda at d+1
    if (tid < a.d) part[tid] = v;
    else if (tid == DP) part[a.d] = v;
    else if (tid == DP + 1) part[a.d + 1] = v;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(a.counter, 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (tid < a.d + 2) {
    double v = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) v += __ldcg(a.partials + (long long)b * kMaxP + tid);
    if (tid == a.d + 1) v *= a.params->lambda;
    a.g_out[tid] = v;
  }
  if (tid == 0) *a.counter = 0;
}

template <typename T, int DP, int M, int TM>
struct GradInst {
  static constexpr int BM = kGradNT * TM;
  static size_t smem_bytes() {
    return (size_t)kStages * (kBN * DP + M * kBN) * sizeof(T) + kStages * sizeof(uint64_t);
  }
  static int occupancy() {
    static int occ = -1;
    static std::once_flag once;
    std::call_once(once, [] {
      auto fn = grad_kernel<T, DP, M, TM, kGradNT>;
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes());
      int o = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, kGradNT, smem_bytes()) !=
          cudaSuccess)
        o = 1;
      occ = std::max(o, 1);
    });
    return occ;
  }
  static cudaError_t launch(GradLaunch& L, cudaStream_t s) {
    KmvPlan p = plan_split(L.n, BM, M, (int)sizeof(T), L.num_sms * occupancy());
    const size_t need = (size_t)p.n_rb * p.nsplit * kMaxP;
    if (L.plan_only) {
      L.need_partials_len = need;
      return cudaSuccess;
    }
    if (need > L.partials_len) {
      L.need_partials_len = need;
      return cudaErrorMemoryAllocation;
    }
    GradDevArgs<T> a;
    a.xhat = static_cast<const T*>(L.xhat);
    a.n = L.n;
    a.ldn = L.ldn;
    a.d = L.d;
    a.A = static_cast<const T*>(L.A);
    a.amap = L.amap;
    a.sa = static_cast<const T*>(L.sa);
    a.B = static_cast<const T*>(L.B);
    a.bmap = L.bmap;
    a.ld = L.ld;
    a.M = L.M;
    a.params = L.params;
    a.nsplit = p.nsplit;
    a.tiles_per_split = p.tiles_per_split;
    a.ntiles = p.ntiles;
    a.partials = L.partials;
    a.counter = L.counter;
    a.g_out = L.g_out;
    a.status = L.status;
    grad_kernel<T, DP, M, TM, kGradNT><<<p.n_rb * p.nsplit, kGradNT, smem_bytes(), s>>>(a);
    return cudaGetLastError();
  }
};

template <typename T, int DP>
static cudaError_t grad_dispatch_m(GradLaunch& L, cudaStream_t s) {
  constexpr int TMs = sizeof(T) == 4 ? 2 : 1;
  if (L.M <= 5) return GradInst<T, DP, 5, TMs>::launch(L, s);
  if (L.M <= 9) return GradInst<T, DP, 9, TMs>::launch(L, s);
  if (L.M <= 17) return GradInst<T, DP, 17, TMs>::launch(L, s);
  if (L.M <= 33) return GradInst<T, DP, 33, 1>::launch(L, s);
  if (L.M <= 64) return GradInst<T, DP, 64, 1>::launch(L, s);
  return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t grad_dispatch(GradLaunch& L, cudaStream_t s) {
  switch (L.DP) {
    case 2: return grad_dispatch_m<T, 2>(L, s);
    case 4: return grad_dispatch_m<T, 4>(L, s);
    case 8: return grad_dispatch_m<T, 8>(L, s);
    case 16: return grad_dispatch_m<T, 16>(L, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_grad_f32(GradLaunch& L, cudaStream_t s) { return grad_dispatch<float>(L, s); }
cudaError_t launch_grad_f64(GradLaunch& L, cudaStream_t s) { return grad_dispatch<double>(L, s); }

}  // namespace ulisse
