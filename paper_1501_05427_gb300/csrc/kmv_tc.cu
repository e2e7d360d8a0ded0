// Mixed-precision tile-generating K V: the contraction on the 5th-generation tensor cores.
//
// For a block of 128 output rows I and a 32-point tile J:
//   1. kernel values on the FP32 pipe: with b_j = -c1 |x^_j|^2 (c1 = log2(e)/2) and
//      a_i = log2(sigma^2) + b_i,   k_ij = sigma^2 exp(-|x^_i - x^_j|^2 / 2)
//                                        = exp2(min(a_i + b_j + 2 c1 x^_i . x^_j, log2 sigma^2)),
//      i.e. d FMAs for the cross term, one FFMA, one min and one ex2 per entry; each value is
//      split into BF16 high and low parts and written to tensor memory (tcgen05.st) as the
//      A operand of the contraction;
//   2. contraction on the tensor cores: U_I += K_IJ V_J with V split into BF16 high + low
//      parts (3 products: Kh Vh + Kh Vl + Kl Vh), FP32 accumulation in tensor memory.
// The cross term stays on the FP32 pipe: with d <= 16 it is a K = d product, too thin for a
// tensor-core pass to pay for its round trip through tensor memory.  Warp 0 streams x^_J,
// b_J and the split V_J into a 4-stage shared-memory ring with bulk copies; one thread of
// warp 1 issues the MMAs (A from tensor memory, B from shared memory); eight epilogue warps
// (a tensor-memory lane quadrant and half of the tile's 32 columns each) make the kernel
// values.  K tiles are double-buffered and each tile is handed to the MMA issuer one tile
// late so the tensor-memory stores overlap the next tile's arithmetic.  Every wait is
// bounded.  The split j range and the fixed-order fix-up of partial sums are those of the
// SIMT kernel; the diagonal term lambda V is added in FP32 from the unsplit operand.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "kmv_kernel.cuh"
#include "tc_common.cuh"

namespace ulisse {

constexpr int kTcBN = 32;
constexpr int kTcBM = 128;
constexpr int kTcThreads = 320;   // warp 0 producer, warp 1 MMA issuer, warps 2-9 epilogue
constexpr uint32_t kTcCols = 128;  // tensor-memory columns per CTA (layout in TcShape)

// ------------------------------------------------------------------------------------
// Operand preparation
// ------------------------------------------------------------------------------------
// b_i = -c1 |x^_i|^2 with c1 = log2(e)/2 (0 for the padding rows).
__global__ void prescale_tc_kernel(const float* __restrict__ xhat, int DP, int d, long long n,
                                   long long ld, float* __restrict__ bneg) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ld;
       i += (long long)gridDim.x * blockDim.x) {
    double s2 = 0.0;
    if (i < n)
      for (int q = 0; q < d; ++q) {
        const double v = xhat[i * DP + q];
        s2 += v * v;
      }
    bneg[i] = (float)(-0.5 * 1.4426950408889634 * s2);
  }
}

// V columns vmap[0..R) -> BF16 high and low parts, one K-major canonical image of N rows
// (right-hand sides) x 32 points per j-tile; rows r >= R and points >= n are zero.
__global__ void pack_v_kernel(const float* __restrict__ V, long long ldv,
                              const int* __restrict__ vmap, int R, int N, long long n,
                              long long ntiles, __nv_bfloat16* __restrict__ Vhi,
                              __nv_bfloat16* __restrict__ Vlo) {
  const long long per_tile = (long long)N * kTcBN;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < ntiles * per_tile;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long t = idx / per_tile;
    const int rem = (int)(idx - t * per_tile);
    const int r = rem / kTcBN, jj = rem - r * kTcBN;
    const long long j = t * kTcBN + jj;
    const float v = (r < R && j < n) ? V[(long long)vmap[r] * ldv + j] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
    const long long off = t * per_tile + tc::canon_offset(r, jj, 2, kTcBN / 8) / 2;
    Vhi[off] = h;
    Vlo[off] = l;
  }
}

// ------------------------------------------------------------------------------------
// Main kernel
// ------------------------------------------------------------------------------------
struct TcDevArgs {
  const float* xhat;     // x^ rows (ld x DP, row-major)
  const float* bneg;     // -c1 |x^|^2
  const __nv_bfloat16* V_hi;
  const __nv_bfloat16* V_lo;
  const float* V;        // FP32 operand columns (diagonal term)
  long long ldv;
  const int* vmap;
  int R;
  float* U;
  long long ldu;
  const int* umap;
  long long n;
  const DevParams* params;
  int nsplit, tiles_per_split, ntiles;
  float* partials;
  int* counters;
  int* status;
};

template <int DP, int N>
struct TcShape {
  static constexpr int kStages = 4;
  static constexpr uint32_t X_BYTES = kTcBN * DP * 4;     // x^ tile, row-major
  static constexpr uint32_t B_BYTES = kTcBN * 4;          // -c1 |x^_j|^2
  static constexpr uint32_t V_BYTES = N * kTcBN * 2;      // BF16 operand tile (one part)
  static constexpr uint32_t STAGE_BYTES = X_BYTES + B_BYTES + 2 * V_BYTES;
  static constexpr uint32_t OFF_BARS = kStages * STAGE_BYTES;
  static constexpr int NBARS = 2 * kStages + 4 + 1;
  static constexpr uint32_t SMEM = OFF_BARS + NBARS * 8 + 64;
  // tensor-memory columns: K tiles (2 buffers x [high 16 | low 16]) then the accumulator
  static constexpr uint32_t COL_K = 0;
  static constexpr uint32_t COL_U = 64;
  static_assert(COL_U + N <= kTcCols, "tensor memory layout exceeds the allocation");
};

// Bounded wait, uniform across the warp.
__device__ inline bool warp_wait(uint64_t* bar, uint32_t parity) {
  const bool ok = mbar_wait_spin(bar, parity);
  return __all_sync(0xffffffffu, ok);
}

template <int NH>
__device__ inline void tmem_ld_cols(uint32_t taddr, float (&v)[NH]) {
  if constexpr (NH == 8) {
    tc::tmem_ld8(taddr, v);
  } else if constexpr (NH == 16) {
    tc::tmem_ld16(taddr, v);
  } else {
    tc::tmem_ld32(taddr, v);
  }
}

template <int DP, int N>
__global__ void __launch_bounds__(kTcThreads, 3) kmv_tc_kernel(const TcDevArgs a) {
  using S = TcShape<DP, N>;
  constexpr int ST = S::kStages;
  constexpr int NH = N / 2;   // accumulator columns read back per column half
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S::OFF_BARS);
  uint64_t* full = bars;
  uint64_t* empty = bars + ST;
  uint64_t* k_full = bars + 2 * ST;
  uint64_t* k_empty = k_full + 2;
  uint64_t* done = k_full + 4;
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + S::OFF_BARS + S::NBARS * 8);
  volatile int* s_fail = reinterpret_cast<volatile int*>(s_tmem + 1);
  int* s_last = reinterpret_cast<int*>(s_tmem + 2);
  auto stage = [&](int s) -> unsigned char* { return smem + s * S::STAGE_BYTES; };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rb = blockIdx.x / a.nsplit;
  const int sp = blockIdx.x - rb * a.nsplit;
  const long long row0 = (long long)rb * kTcBM;
  const int tile_begin = sp * a.tiles_per_split;
  const int nt = max(0, min(tile_begin + a.tiles_per_split, a.ntiles) - tile_begin);

  if (tid == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1 + 8);    // MMA commit + the eight epilogue warps
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&k_full[b], 8);
      mbar_init(&k_empty[b], 1);
    }
    mbar_init(done, 1);
    fence_barrier_init();
    *s_fail = 0;
  }
  if (warp == 1) tc::tmem_alloc(s_tmem, kTcCols);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *s_tmem;

  if (warp == 0) {
    // ---------------- producer: x^_J, b_J and V_J tiles into the ring ----------------
    if (lane == 0) {
      for (int lt = 0; lt < nt; ++lt) {
        const int s = lt % ST;
        if (lt >= ST && !mbar_wait_spin(&empty[s], (uint32_t)(((lt / ST) - 1) & 1))) {
          *s_fail = 1;
          break;
        }
        if (*s_fail) break;
        const long long t = tile_begin + lt;
        unsigned char* st = stage(s);
        mbar_arrive_expect_tx(&full[s], S::STAGE_BYTES);
        bulk_g2s(st, a.xhat + t * kTcBN * DP, S::X_BYTES, &full[s]);
        bulk_g2s(st + S::X_BYTES, a.bneg + t * kTcBN, S::B_BYTES, &full[s]);
        bulk_g2s(st + S::X_BYTES + S::B_BYTES, a.V_hi + t * N * kTcBN, S::V_BYTES, &full[s]);
        bulk_g2s(st + S::X_BYTES + S::B_BYTES + S::V_BYTES, a.V_lo + t * N * kTcBN,
                 S::V_BYTES, &full[s]);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: U += K_hi V_hi + K_hi V_lo + K_lo V_hi ----------------
    if (lane == 0) {
      constexpr uint32_t idesc_k = tc::instr_desc(1, kTcBM, N);
      bool ok = true;
      for (int p = 0; p < nt; ++p) {
        if (*s_fail) { ok = false; break; }
        const int s = p % ST, b = p & 1;
        ok = mbar_wait_spin(&full[s], (uint32_t)((p / ST) & 1)) &&
             mbar_wait_spin(&k_full[b], (uint32_t)((p / 2) & 1));
        if (!ok) break;
        tc::fence_after();
        const uint32_t kH = tbase + S::COL_K + (uint32_t)(b * 32);
        const uint32_t kL = kH + 16;
        const uint32_t vH = smem_u32(stage(s) + S::X_BYTES + S::B_BYTES);
        const uint32_t vL = vH + S::V_BYTES;
#pragma unroll
        for (int term = 0; term < 3; ++term) {
          const uint32_t A = term == 2 ? kL : kH;
          const uint32_t B = term == 1 ? vL : vH;
#pragma unroll
          for (int ks = 0; ks < kTcBN / 16; ++ks)
            tc::mma_bf16_ts(tbase + S::COL_U, A + ks * 8, tc::smem_desc(B + ks * 256, 128, 512),
                            idesc_k, (p | term | ks) != 0);
        }
        tc::commit(&k_empty[b]);
        tc::commit(&empty[s]);
      }
      if (!ok) *s_fail = 1;
      tc::commit(done);
    }
  } else {
    // ---------------- epilogue: 8 warps, (lane quadrant, column half) each ----------------
    const int eq = warp & 3;
    const int half = (warp - 2) >> 2;
    const int il = eq * 32 + lane;
    const long long i = row0 + il;
    const uint32_t lane_base = (uint32_t)(eq * 32) << 16;
    // x^_i pre-scaled by 2 c1, so that the cross-term chain started at a_i + b_j is the
    // whole exponent: a_i + b_j + 2 c1 x^_i . x^_j
    const float c0 = a.params->c0f, c1 = a.params->c1f;
    const float two_c1 = 2.f * c1;
    float xi[DP];
#pragma unroll
    for (int k = 0; k < DP; ++k) xi[k] = (i < a.n) ? two_c1 * a.xhat[i * DP + k] : 0.f;
    const float ai = c0 + ((i < a.n) ? a.bneg[i] : 0.f);   // log2(sigma^2) - c1 |x^_i|^2
    bool ok = true;
    int pending = -1;   // tile whose K stores are in flight (signalled one tile late)
    for (int lt = 0; lt < nt; ++lt) {
      const int s = lt % ST, b = lt & 1;
      const bool ready = warp_wait(&full[s], (uint32_t)((lt / ST) & 1));
      if (!__all_sync(0xffffffffu, ready && !*s_fail)) { ok = false; break; }
      const float* tx = reinterpret_cast<const float*>(stage(s));
      const float* tb = reinterpret_cast<const float*>(stage(s) + S::X_BYTES);
      uint32_t hi[8], lo[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float kk[2];
        const float2 bj = *reinterpret_cast<const float2*>(tb + half * 16 + 2 * q);
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const int j = half * 16 + 2 * q + h2;
          float xj[DP];
          load_row<float, DP>(tx + j * DP, xj);
          float ex = ai + (h2 == 0 ? bj.x : bj.y);
#pragma unroll
          for (int k = 0; k < DP; ++k) ex = fmaf(xi[k], xj[k], ex);
          kk[h2] = ex2_approx(fminf(ex, c0));
        }
        const __nv_bfloat162 h = __floats2bfloat162_rn(kk[0], kk[1]);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(kk[0] - hf.x, kk[1] - hf.y);
        hi[q] = *reinterpret_cast<const uint32_t*>(&h);
        lo[q] = *reinterpret_cast<const uint32_t*>(&l);
      }
      // the stage's x^ and b are consumed; the MMA releases V
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&empty[s]);
      // previous tile's K stores: complete them, hand the tile to the MMA issuer
      if (pending >= 0) {
        tc::tmem_wait_st();
        tc::fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&k_full[pending & 1]);
        pending = -1;
      }
      if (lt >= 2 && !warp_wait(&k_empty[b], (uint32_t)(((lt / 2) - 1) & 1))) { ok = false; break; }
      const uint32_t kcol = tbase + lane_base + S::COL_K + (uint32_t)(b * 32 + half * 8);
      tc::tmem_st8(kcol, hi);
      tc::tmem_st8(kcol + 16, lo);
      pending = lt;
    }
    if (pending >= 0) {
      tc::tmem_wait_st();
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&k_full[pending & 1]);
    }
    if (!ok) *s_fail = 1;
    const bool fin = ok && warp_wait(done, 0);
    ok = __all_sync(0xffffffffu, fin && !*s_fail);
    if (ok) {
      tc::fence_after();
      float u[NH];
      tmem_ld_cols<NH>(tbase + lane_base + S::COL_U + (uint32_t)(half * NH), u);
      if (a.nsplit == 1) {
        if (i < a.n) {
          const float lam = (float)a.params->lambda;
#pragma unroll
          for (int q = 0; q < NH; ++q) {
            const int r = half * NH + q;
            if (r < a.R)
              a.U[(long long)a.umap[r] * a.ldu + i] =
                  fmaf(lam, a.V[(long long)a.vmap[r] * a.ldv + i], u[q]);
          }
        }
      } else {
        float* part = a.partials + (long long)blockIdx.x * N * kTcBM;
#pragma unroll
        for (int q = 0; q < NH; ++q) part[(half * NH + q) * kTcBM + il] = u[q];
      }
    }
  }

  // -------- all roles: release tensor memory; last CTA of the row block reduces --------
  if (warp == 1) {
    // the MMAs this CTA issued are complete once `done` has fired
    if (lane == 0) (void)mbar_wait_spin(done, 0);
    __syncwarp();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 1) tc::tmem_dealloc(tbase, kTcCols);
  if (*s_fail) {
    if (tid == 0) atomicOr(a.status, kStatusTimeout);
    return;
  }
  if (a.nsplit == 1) return;
  __threadfence();
  __syncthreads();
  if (tid == 0) *s_last = (atomicAdd(&a.counters[rb], 1) == a.nsplit - 1);
  __syncthreads();
  if (!*s_last) return;
  __threadfence();
  const float* base = a.partials + (long long)rb * a.nsplit * N * kTcBM;
  const float lam = (float)a.params->lambda;
  for (int idx = tid; idx < a.R * kTcBM; idx += kTcThreads) {
    const int r = idx / kTcBM, il = idx - r * kTcBM;
    const long long i = row0 + il;
    if (i >= a.n) continue;
    float u = 0.f;
    for (int s2 = 0; s2 < a.nsplit; ++s2) u += __ldcg(base + ((long long)s2 * N + r) * kTcBM + il);
    a.U[(long long)a.umap[r] * a.ldu + i] = fmaf(lam, a.V[(long long)a.vmap[r] * a.ldv + i], u);
  }
  if (tid == 0) a.counters[rb] = 0;
}

// The BF16 high/low images of the operand columns for an N-column MMA (every K V launch).
void launch_pack_v(const TcLaunch& L, int N, long long ntiles, cudaStream_t s) {
  const long long total = ntiles * N * kTcBN;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 8LL * L.num_sms);
  pack_v_kernel<<<blocks, 256, 0, s>>>(static_cast<const float*>(L.V), L.ldv, L.vmap, L.R, N,
                                       L.n, ntiles, static_cast<__nv_bfloat16*>(L.V_hi),
                                       static_cast<__nv_bfloat16*>(L.V_lo));
}

template <int DP, int N>
struct TcInst {
  // CTAs per SM: shared memory (the runtime's occupancy query may assume a smaller
  // carveout than the one the launch gets), at most four by tensor memory (512 columns).
  static int occupancy() {
    static int occ = -1;
    static std::once_flag once;
    std::call_once(once, [] {
      auto fn = kmv_tc_kernel<DP, N>;
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)TcShape<DP, N>::SMEM);
      cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      int dev = 0, smem_sm = 0;
      cudaGetDevice(&dev);
      if (cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
          cudaSuccess)
        smem_sm = 228 * 1024;
      const int by_smem = smem_sm / (int)(TcShape<DP, N>::SMEM + 1024);
      occ = std::max(1, std::min(by_smem, (int)(512 / kTcCols)));
    });
    return occ;
  }
  static cudaError_t launch(TcLaunch& L, cudaStream_t s) {
    KmvPlan p = L.nsplit > 0 ? plan_split_forced(L.n, kTcBM, N, 4, L.nsplit)
                             : plan_split(L.n, kTcBM, N, 4, L.num_sms * occupancy());
    p = tc_bound_split(p, L.n, kTcBM, N, kTcBN);
    const size_t pbytes = p.nsplit > 1 ? (size_t)p.n_rb * p.nsplit * N * kTcBM * 4 : 0;
    L.planned_nsplit = p.nsplit;
    if (L.plan_only) {
      L.need_partials_bytes = pbytes;
      L.need_counters = p.nsplit > 1 ? p.n_rb : 0;
      return cudaSuccess;
    }
    if (pbytes > L.partials_bytes || (p.nsplit > 1 && p.n_rb > L.counters_len)) {
      L.need_partials_bytes = pbytes;
      L.need_counters = p.n_rb;
      return cudaErrorMemoryAllocation;
    }
    const long long ntiles = (L.n + kTcBN - 1) / kTcBN;
    launch_pack_v(L, N, ntiles, s);
    TcDevArgs a;
    a.xhat = L.xhat;
    a.bneg = L.bneg;
    a.V_hi = static_cast<const __nv_bfloat16*>(L.V_hi);
    a.V_lo = static_cast<const __nv_bfloat16*>(L.V_lo);
    a.V = static_cast<const float*>(L.V);
    a.ldv = L.ldv;
    a.vmap = L.vmap;
    a.R = L.R;
    a.U = static_cast<float*>(L.U);
    a.ldu = L.ldu;
    a.umap = L.umap;
    a.n = L.n;
    a.params = L.params;
    a.nsplit = p.nsplit;
    a.tiles_per_split = (int)((ntiles + p.nsplit - 1) / p.nsplit);
    a.nsplit = (int)((ntiles + a.tiles_per_split - 1) / a.tiles_per_split);
    a.ntiles = (int)ntiles;
    a.partials = static_cast<float*>(L.partials);
    a.counters = L.counters;
    a.status = L.status;
    (void)occupancy();
    const int nrb = (int)((L.n + kTcBM - 1) / kTcBM);
    kmv_tc_kernel<DP, N><<<nrb * a.nsplit, kTcThreads, TcShape<DP, N>::SMEM, s>>>(a);
    return cudaGetLastError();
  }
};

template <int DP>
static cudaError_t tc_dispatch_n(TcLaunch& L, cudaStream_t s) {
  const int r = std::max(L.R, L.n_min);
  if (r <= 16) return TcInst<DP, 16>::launch(L, s);
  if (r <= 32) return TcInst<DP, 32>::launch(L, s);
  if (r <= 64) return TcInst<DP, 64>::launch(L, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_kmv_tc(TcLaunch& L, cudaStream_t s) {
  if (L.R < 1 || L.R > 64) return cudaErrorInvalidValue;
  switch (L.DP) {
    case 2: return tc_dispatch_n<2>(L, s);
    case 4: return tc_dispatch_n<4>(L, s);
    case 8: return tc_dispatch_n<8>(L, s);
    case 16: return tc_dispatch_n<16>(L, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_prescale_tc(const float* xhat, int DP, int d, long long n, long long ld,
                               float* bneg, int num_sms, cudaStream_t s) {
  const int blocks = (int)std::min<long long>((ld + 255) / 256, 8LL * num_sms);
  prescale_tc_kernel<<<blocks, 256, 0, s>>>(xhat, DP, d, n, ld, bneg);
  return cudaGetLastError();
}

}  // namespace ulisse
