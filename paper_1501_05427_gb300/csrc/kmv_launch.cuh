// Host launcher for the tile-generating K V kernel: picks the instantiation for (DP, R),
// sizes the split of the j range to the SM count and occupancy, and launches.
#pragma once

#include <algorithm>
#include <mutex>
#include <utility>

#include "kmv_kernel.cuh"

namespace ulisse {

constexpr int kKmvNT = 128;

template <typename T, int DP, int R, int TM, int MODE>
struct KmvInst {
  static constexpr int BM = kKmvNT * TM;
  static size_t smem_bytes() {
    return (size_t)kStages * (kBN * DP + R * kBN) * sizeof(T) + kStages * sizeof(uint64_t);
  }
  static int occupancy() {
    static int occ = -1;
    static std::once_flag once;
    std::call_once(once, [] {
      auto fn = kmv_kernel<T, DP, R, TM, kKmvNT, MODE>;
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes());
      int o = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, kKmvNT, smem_bytes()) !=
          cudaSuccess)
        o = 1;
      occ = std::max(o, 1);
    });
    return occ;
  }
  static KmvPlan plan(const KmvLaunch& L) {
    if (L.nsplit > 0) return plan_split_forced(L.n, BM, R, (int)sizeof(T), L.nsplit);
    return plan_split(L.n, BM, R, (int)sizeof(T), L.num_sms * occupancy());
  }
  static cudaError_t launch(KmvLaunch& L, cudaStream_t s) {
    KmvPlan p = plan(L);
    if (MODE == kModeDLam) {  // dK/dlog lambda = lambda I: no tiles, one CTA per row block
      p.nsplit = 1;
      p.tiles_per_split = 0;
      p.partial_bytes = 0;
    }
    L.planned_nsplit = p.nsplit;
    if (L.plan_only) {
      L.need_partials_bytes = p.partial_bytes;
      L.need_counters = p.nsplit > 1 ? p.n_rb : 0;
      return cudaSuccess;
    }
    if (p.partial_bytes > L.partials_bytes || (p.nsplit > 1 && p.n_rb > L.counters_len)) {
      // Scratch too small: report what this launch needs; the caller grows it and retries.
      L.need_partials_bytes = p.partial_bytes;
      L.need_counters = p.n_rb;
      return cudaErrorMemoryAllocation;
    }
    KmvDevArgs<T> a;
    a.xhat = static_cast<const T*>(L.xhat);
    a.n = L.n;
    a.ldn = L.ldn;
    a.V = static_cast<const T*>(L.V);
    a.ldv = L.ldv;
    a.vmap = L.vmap;
    a.R = L.R;
    a.U = static_cast<T*>(L.U);
    a.ldu = L.ldu;
    a.umap = L.umap;
    a.params = L.params;
    a.mode = L.mode;
    a.which = L.which;
    a.nsplit = p.nsplit;
    a.tiles_per_split = p.tiles_per_split;
    a.ntiles = p.ntiles;
    a.partials = static_cast<T*>(L.partials);
    a.counters = L.counters;
    a.status = L.status;
    (void)occupancy();
    kmv_kernel<T, DP, R, TM, kKmvNT, MODE><<<p.n_rb * p.nsplit, kKmvNT, smem_bytes(), s>>>(a);
    return cudaGetLastError();
  }
};

// Smallest instantiated R >= r, from a sorted list.
template <int... Rs>
struct RList {};

template <typename T, int DP, int TM, int MODE, int R0, int... Rs>
cudaError_t dispatch_r(KmvLaunch& L, cudaStream_t s, RList<R0, Rs...>) {
  if ((L.R <= R0 && L.r_min <= R0) || sizeof...(Rs) == 0)
    return KmvInst<T, DP, R0, TM, MODE>::launch(L, s);
  if constexpr (sizeof...(Rs) > 0) return dispatch_r<T, DP, TM, MODE>(L, s, RList<Rs...>{});
  return cudaErrorInvalidValue;
}

// Mode and rows-per-thread dispatch for one DP.  K uses the tuned rows per thread
// (L.tm: 2 or 4); the derivative products use 2 rows per thread and a shorter R list.
template <typename T, int DP, int TMK, int TMK2, typename RK, typename RD>
cudaError_t dispatch_mode(KmvLaunch& L, cudaStream_t s) {
  switch (L.mode) {
    case kModeK:
      if (L.tm == TMK2) return dispatch_r<T, DP, TMK2, kModeK>(L, s, RK{});
      return dispatch_r<T, DP, TMK, kModeK>(L, s, RK{});
    case kModeDLen: return dispatch_r<T, DP, TMK, kModeDLen>(L, s, RD{});
    case kModeDSig: return dispatch_r<T, DP, TMK, kModeDSig>(L, s, RD{});
    case kModeDLam: return dispatch_r<T, DP, TMK, kModeDLam>(L, s, RD{});
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ulisse
