// Tile-generating covariance matrix-vector product (Sec. 3: K V without storing K).
//
// One CTA owns BM = NT * TM output rows and a contiguous range of j-tiles (a "split").
// For every j-tile of kBN points, one thread issues bulk asynchronous copies (TMA unit) of
// the prescaled inputs x^_J (kBN x DP, contiguous) and of each right-hand side's segment
// V[J, r] (kBN contiguous values per column) into a kStages-deep shared-memory ring guarded
// by mbarriers.  Every thread then generates k(x_i, x_j) for its TM rows and four j's at a
// time -- ARD squared distance on x^ = x / l, then sigma^2 exp(-dist / 2) as one FMA and one
// ex2 -- and applies it to all R right-hand sides from registers (vectorised 16-byte shared
// loads of four consecutive j's per column).
//
// When the j range is split over several CTAs, each writes its partial rows to scratch and
// the last CTA of a row block (an atomic arrival count; nobody waits) sums the partials in
// split order, adds the lambda V diagonal term and writes U: deterministic, one launch.
#pragma once

#include "ulisse_internal.cuh"

namespace ulisse {

template <typename T>
struct KmvDevArgs {
  const T* xhat;
  long long n, ldn;
  const T* V;
  long long ldv;
  const int* vmap;
  int R;
  T* U;
  long long ldu;
  const int* umap;
  const DevParams* params;
  int mode, which;
  int nsplit, tiles_per_split, ntiles;
  T* partials;
  int* counters;
  int* status;
};

template <typename T, int DP>
__device__ __forceinline__ void load_row(const T* __restrict__ p, T (&x)[DP]) {
  if constexpr (sizeof(T) == 4 && DP % 4 == 0) {
#pragma unroll
    for (int k = 0; k < DP; k += 4) {
      const float4 v = *reinterpret_cast<const float4*>(p + k);
      x[k] = v.x; x[k + 1] = v.y; x[k + 2] = v.z; x[k + 3] = v.w;
    }
  } else if constexpr (DP % 2 == 0) {
    using V2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
#pragma unroll
    for (int k = 0; k < DP; k += 2) {
      const V2 v = *reinterpret_cast<const V2*>(p + k);
      x[k] = v.x; x[k + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < DP; ++k) x[k] = p[k];
  }
}

// Signal covariance from the squared prescaled distance.
template <typename T>
__device__ __forceinline__ T kernel_from_dist(T dist, float c0, float c1, double sigma2) {
  if constexpr (sizeof(T) == 4) {
    return ex2_approx(fmaf(-c1, dist, c0));
  } else {
    return sigma2 * exp(-0.5 * dist);
  }
}

// MODE (compile time): kModeK (K), kModeDLen (dK/dlog l_which), kModeDSig (dK/dlog sigma^2),
// kModeDLam (dK/dlog lambda = lambda I: no tiles, only the diagonal term).
template <typename T, int DP, int R, int TM, int NT, int MODE>
__global__ void __launch_bounds__(NT) kmv_kernel(const KmvDevArgs<T> a) {
  constexpr int BM = NT * TM;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* sX = reinterpret_cast<T*>(smem_raw);
  T* sV = sX + kStages * kBN * DP;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sV + kStages * R * kBN);
  __shared__ int s_vcol[R];
  __shared__ int s_last;

  const int tid = threadIdx.x;
  const int rb = blockIdx.x / a.nsplit;
  const int sp = blockIdx.x - rb * a.nsplit;
  const long long row0 = (long long)rb * BM;
  const int tile_begin = sp * a.tiles_per_split;
  const int tile_end = min(tile_begin + a.tiles_per_split, a.ntiles);
  const int nt_local = (MODE == kModeDLam) ? 0 : max(0, tile_end - tile_begin);
  const int Ra = a.R;

  const float c0 = a.params->c0f, c1 = a.params->c1f;
  const double sigma2 = a.params->sigma2;
  const T lam = (T)a.params->lambda;

  if (tid < R) s_vcol[tid] = (tid < Ra) ? a.vmap[tid] : 0;
  // Columns beyond the live count stay zero in every stage (never copied into).
  for (int idx = tid; idx < kStages * (R - Ra) * kBN; idx += NT) {
    const int st = idx / ((R - Ra) * kBN);
    const int rem = idx - st * (R - Ra) * kBN;
    sV[(st * R + Ra) * kBN + rem] = T(0);
  }
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
    fence_barrier_init();
  }
  __syncthreads();

  const uint32_t tile_bytes = (uint32_t)(kBN * DP * sizeof(T) + Ra * kBN * sizeof(T));
  auto issue = [&](int lt) {
    const int s = lt % kStages;
    const long long j0 = (long long)(tile_begin + lt) * kBN;
    mbar_arrive_expect_tx(&bar[s], tile_bytes);
    bulk_g2s(sX + s * kBN * DP, a.xhat + j0 * DP, kBN * DP * sizeof(T), &bar[s]);
    for (int r = 0; r < Ra; ++r)
      bulk_g2s(sV + (s * R + r) * kBN, a.V + (long long)s_vcol[r] * a.ldv + j0,
               kBN * sizeof(T), &bar[s]);
  };
  int issued = 0;  // meaningful in thread 0 only
  if (tid == 0)
    for (; issued < min(kStages, nt_local); ++issued) issue(issued);

  // Own rows: prescaled inputs in registers.
  T xi[TM][DP];
  T xiw[TM];
#pragma unroll
  for (int t = 0; t < TM; ++t) {
    const long long i = row0 + t * NT + tid;
    if (i < a.n) {
      load_row<T, DP>(a.xhat + i * DP, xi[t]);
    } else {
#pragma unroll
      for (int k = 0; k < DP; ++k) xi[t][k] = T(0);
    }
    xiw[t] = (MODE == kModeDLen && i < a.n) ? a.xhat[i * DP + a.which] : T(0);
  }

  T acc[TM][R];
#pragma unroll
  for (int t = 0; t < TM; ++t)
#pragma unroll
    for (int r = 0; r < R; ++r) acc[t][r] = T(0);

  bool timed_out = false;
  for (int lt = 0; lt < nt_local; ++lt) {
    const int s = lt % kStages;
    const bool ok = mbar_wait_bounded(&bar[s], (uint32_t)((lt / kStages) & 1));
    if (ok) {
      const T* tX = sX + s * kBN * DP;
      const T* tV = sV + s * R * kBN;
#pragma unroll 1
      for (int jq = 0; jq < kBN; jq += 4) {
        T kq[TM][4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          T xj[DP];
          load_row<T, DP>(tX + (jq + q) * DP, xj);
#pragma unroll
          for (int t = 0; t < TM; ++t) {
            T dist = T(0);
#pragma unroll
            for (int k = 0; k < DP; ++k) {
              const T df = xi[t][k] - xj[k];
              dist = fma(df, df, dist);
            }
            T kv = kernel_from_dist<T>(dist, c0, c1, sigma2);
            if constexpr (MODE == kModeDLen) {
              const T dw = xiw[t] - tX[(jq + q) * DP + a.which];
              kv *= dw * dw;
            }
            kq[t][q] = kv;
          }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
          T v[4];
          if constexpr (sizeof(T) == 4) {
            const float4 w = *reinterpret_cast<const float4*>(tV + r * kBN + jq);
            v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w;
          } else {
            const double2 w0 = *reinterpret_cast<const double2*>(tV + r * kBN + jq);
            const double2 w1 = *reinterpret_cast<const double2*>(tV + r * kBN + jq + 2);
            v[0] = w0.x; v[1] = w0.y; v[2] = w1.x; v[3] = w1.y;
          }
#pragma unroll
          for (int t = 0; t < TM; ++t) {
            T u = acc[t][r];
            u = fma(kq[t][0], v[0], u);
            u = fma(kq[t][1], v[1], u);
            u = fma(kq[t][2], v[2], u);
            u = fma(kq[t][3], v[3], u);
            acc[t][r] = u;
          }
        }
      }
    }
    if (__syncthreads_or(!ok)) { timed_out = true; break; }
    if (tid == 0 && issued < nt_local) issue(issued++);
  }
  if (timed_out) {
    if (tid == 0) {
      atomicOr(a.status, kStatusTimeout);
      // Let copies still in flight land before the CTA's shared memory is released.
      for (int lt2 = max(0, issued - kStages); lt2 < issued; ++lt2)
        (void)mbar_wait_bounded(&bar[lt2 % kStages], (uint32_t)((lt2 / kStages) & 1));
    }
    return;
  }

  // Diagonal term lambda V (K) or the whole product (dK/dlog lambda = lambda I).
  constexpr bool add_diag = (MODE == kModeK || MODE == kModeDLam);
  if (a.nsplit == 1) {
#pragma unroll
    for (int t = 0; t < TM; ++t) {
      const long long i = row0 + t * NT + tid;
      if (i >= a.n) continue;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (r >= Ra) break;
        T u = acc[t][r];
        if constexpr (add_diag) u = fma(lam, a.V[(long long)s_vcol[r] * a.ldv + i], u);
        a.U[(long long)a.umap[r] * a.ldu + i] = u;
      }
    }
    return;
  }

  // Split j range: publish the partial rows, then the last CTA of the row block reduces.
  T* part = a.partials + ((long long)rb * a.nsplit + sp) * (long long)R * BM;
#pragma unroll
  for (int t = 0; t < TM; ++t)
#pragma unroll
    for (int r = 0; r < R; ++r) part[(long long)r * BM + t * NT + tid] = acc[t][r];
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(&a.counters[rb], 1) == a.nsplit - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const T* base = a.partials + (long long)rb * a.nsplit * (long long)R * BM;
#pragma unroll
  for (int t = 0; t < TM; ++t) {
    const long long i = row0 + t * NT + tid;
    if (i >= a.n) continue;
    for (int r = 0; r < Ra; ++r) {
      T u = T(0);
      for (int s2 = 0; s2 < a.nsplit; ++s2)
        u += __ldcg(base + ((long long)s2 * R + r) * BM + t * NT + tid);
      if constexpr (add_diag) u = fma(lam, a.V[(long long)s_vcol[r] * a.ldv + i], u);
      a.U[(long long)a.umap[r] * a.ldu + i] = u;
    }
  }
  if (tid == 0) a.counters[rb] = 0;
}

// Host-side plan for one launch: how many CTAs split each row block's j range.
struct KmvPlan {
  int nsplit, tiles_per_split, ntiles, n_rb;
  size_t partial_bytes;
};

inline KmvPlan plan_split(long long n, int BM, int R, int elem, int slots) {
  KmvPlan p;
  p.ntiles = (int)((n + kBN - 1) / kBN);
  p.n_rb = (int)((n + BM - 1) / BM);
  long long best_cost = -1;
  int best = 1;
  const int smax = max(1, min(p.ntiles, 64));
  for (int s = 1; s <= smax; ++s) {
    const long long items = (long long)p.n_rb * s;
    if (s > 1 && items > 4LL * slots) break;
    const long long waves = (items + slots - 1) / slots;
    const long long tiles = (p.ntiles + s - 1) / s;
    // time ~ waves * tiles per item, plus a small cost per extra split (fix-up pass)
    const long long cost = waves * tiles * 64 + (s > 1 ? 2 * s : 0);
    if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = s; }
  }
  p.nsplit = best;
  p.tiles_per_split = (p.ntiles + best - 1) / best;
  p.nsplit = (p.ntiles + p.tiles_per_split - 1) / p.tiles_per_split;
  p.partial_bytes = p.nsplit > 1 ? (size_t)p.n_rb * p.nsplit * R * BM * elem : 0;
  return p;
}

// The same plan with the split count given (a tuned choice), clamped to 1..min(64, tiles).
inline KmvPlan plan_split_forced(long long n, int BM, int R, int elem, int nsplit) {
  KmvPlan p;
  p.ntiles = (int)((n + kBN - 1) / kBN);
  p.n_rb = (int)((n + BM - 1) / BM);
  const int s = max(1, min(nsplit, min(p.ntiles, 64)));
  p.tiles_per_split = (p.ntiles + s - 1) / s;
  p.nsplit = (p.ntiles + p.tiles_per_split - 1) / p.tiles_per_split;
  p.partial_bytes = p.nsplit > 1 ? (size_t)p.n_rb * p.nsplit * R * BM * elem : 0;
  return p;
}

// Tensor-core K V accumulates a CTA's whole j range in FP32 in tensor memory, so its rounding
// grows with the range: at most kTcMaxSplitTiles 32-point tiles per CTA (20,480 points).  At
// n = 50,000 a range of 16,700 points kept the two cross-term forms within 2e-6 of each other
// (relative to max |U|), the whole range (50,000) gave 1.4e-4.
constexpr int kTcMaxSplitTiles = 640;

inline KmvPlan tc_bound_split(KmvPlan p, long long n, int BM, int R, int BN) {
  const long long nt = (n + BN - 1) / BN;
  const long long tps = (nt + p.nsplit - 1) / p.nsplit;
  if (tps <= kTcMaxSplitTiles) return p;
  const int s = (int)((nt + kTcMaxSplitTiles - 1) / kTcMaxSplitTiles);
  p.nsplit = s;
  p.partial_bytes = (size_t)p.n_rb * s * R * BM * 4;
  return p;
}

}  // namespace ulisse
