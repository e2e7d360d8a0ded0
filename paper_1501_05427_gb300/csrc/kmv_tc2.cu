// Mixed-precision tile-generating K V with the cross term on the tensor cores too.
//
// For a block of 128 output rows I and a 32-point tile J:
//   1. C_IJ = A_I B_J^T on the tensor cores (kind::tf32).  With padded d = 2 or 4 the rows
//      carry the column term too,
//          A_i = [x^_i, 1],  B_j = [2 c1 x^_j, b_j],   b_j = -c1 |x^_j|^2, c1 = log2(e)/2,
//      so that C_ij = 2 c1 x^_i . x^_j + b_j in one 8-wide K step; with padded d = 8 or 16
//      the rows are A_i = x^_i, B_j = 2 c1 x^_j (K = d: the augmented column would cost a
//      whole further K step, three MMAs per tile on the one issuing thread that paces the
//      kernel) and the epilogue adds b_j.  Both sides split into a TF32 high part and the
//      remainder, three products (Ah Bh + Ah Bl + Al Bh), FP32 accumulation into a 32-column
//      tensor-memory buffer;
//   2. the epilogue warps read C back (tcgen05.ld) and form
//          k_ij = exp2(a_i + C_ij)  or  exp2((a_i + b_j) + C_ij),
//          a_i = log2(sigma^2) - c1 |x^_i|^2
//      (one or two FADDs and one ex2 per entry), split k into BF16 high and low parts and
//      store them over C's own columns (tcgen05.st);
//   3. U_I += K_IJ V_J on the tensor cores with V split into BF16 high + low parts (three
//      products), FP32 accumulation in tensor memory, as in the FP32-pipe variant.
// The TF32 images of A and B (high and low parts, K-major canonical, 32-point tiles back to
// back so that four tiles form the 128-row A operand) are written once per parameter value by
// pack_x_tf32_kernel.  Roles: warp 0 streams the A image once, then the B_J image and V_J
// into a 3- or 4-stage ring with bulk copies; one thread of warp 1 issues the MMAs; eight
// epilogue warps make the kernel values, in two sets of four (one per tensor-memory lane
// quadrant) that take alternate tiles whole, so that each wait and hand-off covers 32
// entries per thread.  Three C/K buffers (two when the accumulator takes 64 columns); a buffer
// is refilled only after the MMAs that read it have completed.  Every wait is bounded.  The split j range, the fixed-order fix-up of the
// partial sums and the FP32 diagonal term lambda V are those of the FP32-pipe variant.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "kmv_kernel.cuh"
#include "tc_common.cuh"

namespace ulisse {

constexpr int kT2BN = 32;
constexpr int kT2BM = 128;
constexpr int kT2Threads = 320;    // warp 0 producer, warp 1 MMA issuer, warps 2-9 epilogue
constexpr uint32_t kT2Cols = 128;  // tensor-memory columns per CTA

// The rows A_j = [x^_j, 1, 0...] and B_j = [2 c1 x^_j, b_j, 0...] for j in [0, rows) as TF32
// high part and remainder, K8 columns, in 32-row K-major canonical tiles; rows >= n are zero.
// When K8 == DP there is no slot for the augmented column (A_j = x^_j, B_j = 2 c1 x^_j); the
// batched launches leave it out for every d (aug = 0) and add b_j in the epilogue.
// b_j = -c1 |x^_j|^2 is read from the row norms of launch_prescale_tc.
__global__ void pack_x_tf32_kernel(const float* __restrict__ xhat, const float* __restrict__ bneg,
                                   const DevParams* __restrict__ params, int DP, int K8, int aug,
                                   long long n, long long rows, float* __restrict__ Ahi,
                                   float* __restrict__ Alo, float* __restrict__ Bhi,
                                   float* __restrict__ Blo) {
  const float two_c1 = 2.f * params->c1f;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < rows * K8;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long j = idx / K8;
    const int k = (int)(idx - j * K8);
    float va = 0.f, vb = 0.f;
    if (j < n) {
      if (k < DP) {
        va = xhat[j * DP + k];
        vb = two_c1 * va;
      } else if (k == DP && aug) {
        va = 1.f;
        vb = bneg[j];
      }
    }
    const long long t = j / kT2BN;
    const int jj = (int)(j - t * kT2BN);
    const long long off = t * kT2BN * K8 + tc::canon_offset(jj, k, 4, K8 / 4) / 4;
    const float ha = tc::tf32_round(va), hb = tc::tf32_round(vb);
    Ahi[off] = ha;
    Alo[off] = va - ha;
    Bhi[off] = hb;
    Blo[off] = vb - hb;
  }
}

struct Tc2DevArgs {
  const float* A_hi;     // TF32 image of the augmented A rows (high part)
  const float* A_lo;     // remainder
  const float* B_hi;     // TF32 image of the augmented B rows
  const float* B_lo;
  const float* bneg;     // -c1 |x^|^2
  const __nv_bfloat16* V_hi;
  const __nv_bfloat16* V_lo;
  const float* V;        // FP32 operand columns (diagonal term)
  long long ldv;
  const int* vmap;
  int R;
  const int* R_dev;      // batched launches: the live column count on the device (else null)
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

// BJ: the epilogue adds b_j (the rows are not augmented); the stage then carries b_J.
template <int K8, int N, bool BJ>
struct Tc2Shape {
  static constexpr uint32_t A_BYTES = kT2BM * K8 * 4;   // one part of the A_I image
  static constexpr uint32_t XB_BYTES = kT2BN * K8 * 4;  // one part of the B_J image
  static constexpr uint32_t V_BYTES = N * kT2BN * 2;    // one part of the BF16 V_J tile
  static constexpr uint32_t BN_BYTES = BJ ? kT2BN * 4 : 0;   // b_J
  static constexpr uint32_t OFF_BN = 2 * XB_BYTES + 2 * V_BYTES;   // within a stage
  static constexpr uint32_t STAGE_BYTES = 2 * XB_BYTES + 2 * V_BYTES + BN_BYTES;
  // four stages while four CTAs still fit in shared memory (~54 KB each), else three
  static constexpr int ST = (2 * A_BYTES + 4 * STAGE_BYTES <= 54 * 1024) ? 4 : 3;
  static constexpr uint32_t OFF_STAGES = 2 * A_BYTES;
  static constexpr uint32_t OFF_BARS = OFF_STAGES + ST * STAGE_BYTES;
  // C/K buffers of 32 columns: three while they fit beside the accumulator, else two
  static constexpr int NB = (3 * 32 + N <= (int)kT2Cols) ? 3 : 2;
  // full, empty per stage; a_full; c_full per tile mod 6 (so that each barrier serves one
  // epilogue set and its phases are waited in order); k_full, b_free per buffer; done
  static constexpr int NCF = 6;
  static constexpr int NBARS = 2 * ST + 1 + NCF + 2 * NB + 1;
  static constexpr uint32_t SMEM = OFF_BARS + NBARS * 8 + 64;
  static constexpr uint32_t COL_U = NB * 32;   // after the C/K buffers
  static_assert(COL_U + N <= kT2Cols, "tensor memory layout exceeds the allocation");
  static_assert(STAGE_BYTES % 16 == 0 && A_BYTES % 16 == 0 && XB_BYTES % 16 == 0,
                "bulk copies and descriptors need 16-byte alignment");
};

__device__ inline bool t2_warp_wait(uint64_t* bar, uint32_t parity) {
  const bool ok = mbar_wait_spin(bar, parity);
  return __all_sync(0xffffffffu, ok);
}

template <int NH>
__device__ inline void t2_ld_cols(uint32_t taddr, float (&v)[NH]) {
  if constexpr (NH == 8) {
    tc::tmem_ld8(taddr, v);
  } else if constexpr (NH == 16) {
    tc::tmem_ld16(taddr, v);
  } else {
    // two 16-column loads: a 32-register load does not fit the 48-register budget
    float v0[16], v1[16];
    tc::tmem_ld16(taddr, v0);
    tc::tmem_ld16(taddr + 16, v1);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      v[q] = v0[q];
      v[16 + q] = v1[q];
    }
  }
}

// One CTA's work: row block rb, j-range split sp, R live columns.  Shared by the
// single-problem kernel (rb, sp from the block index) and the batched one (from its work list).
template <int K8, int N, bool BJ>
__device__ __forceinline__ void tc2_body(const Tc2DevArgs& a, const int rb, const int sp,
                                         const int R) {
  using S = Tc2Shape<K8, N, BJ>;
  constexpr int ST = S::ST;
  constexpr int NB = S::NB;
  constexpr int NH = N / 2;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sAh = smem;
  unsigned char* sAl = smem + S::A_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S::OFF_BARS);
  uint64_t* full = bars;
  uint64_t* empty = bars + ST;
  uint64_t* a_full = bars + 2 * ST;
  uint64_t* c_full = a_full + 1;
  uint64_t* k_full = c_full + S::NCF;
  uint64_t* b_free = k_full + NB;
  uint64_t* done = b_free + NB;
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + S::OFF_BARS + S::NBARS * 8);
  volatile int* s_fail = reinterpret_cast<volatile int*>(s_tmem + 1);
  int* s_last = reinterpret_cast<int*>(s_tmem + 2);
  auto stage = [&](int s) -> unsigned char* { return smem + S::OFF_STAGES + s * S::STAGE_BYTES; };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long slot = (long long)rb * a.nsplit + sp;   // this CTA's partial-sum slot
  const long long row0 = (long long)rb * kT2BM;
  const int tile_begin = sp * a.tiles_per_split;
  const int nt = max(0, min(tile_begin + a.tiles_per_split, a.ntiles) - tile_begin);

  if (tid == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);   // the MMA commit: only the tensor cores read a stage
    }
    mbar_init(a_full, 1);
    for (int c = 0; c < S::NCF; ++c) mbar_init(&c_full[c], 1);
    for (int b = 0; b < NB; ++b) {
      mbar_init(&k_full[b], 4);   // the four epilogue warps of the tile's set
      mbar_init(&b_free[b], 1);
    }
    mbar_init(done, 1);
    fence_barrier_init();
    *s_fail = 0;
  }
  if (warp == 1) tc::tmem_alloc(s_tmem, kT2Cols);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *s_tmem;
  int issued = 0;   // tiles whose copies the producer started (lane 0 of warp 0)

  if (warp == 0) {
    // ---------------- producer: the x^_I image, then x^_J, b_J, V_J into the ring ----------
    if (lane == 0) {
      mbar_arrive_expect_tx(a_full, 2 * S::A_BYTES);
      bulk_g2s(sAh, a.A_hi + row0 * K8, S::A_BYTES, a_full);
      bulk_g2s(sAl, a.A_lo + row0 * K8, S::A_BYTES, a_full);
      for (int lt = 0; lt < nt; ++lt) {
        const int s = lt % ST;
        if (lt >= ST && !mbar_wait_backoff(&empty[s], (uint32_t)(((lt / ST) - 1) & 1))) {
          *s_fail = 1;
          break;
        }
        if (*s_fail) break;
        const long long t = tile_begin + lt;
        unsigned char* st = stage(s);
        mbar_arrive_expect_tx(&full[s], S::STAGE_BYTES);
        bulk_g2s(st, a.B_hi + t * kT2BN * K8, S::XB_BYTES, &full[s]);
        bulk_g2s(st + S::XB_BYTES, a.B_lo + t * kT2BN * K8, S::XB_BYTES, &full[s]);
        unsigned char* sv = st + 2 * S::XB_BYTES;
        bulk_g2s(sv, a.V_hi + t * N * kT2BN, S::V_BYTES, &full[s]);
        bulk_g2s(sv + S::V_BYTES, a.V_lo + t * N * kT2BN, S::V_BYTES, &full[s]);
        if constexpr (BJ) bulk_g2s(st + S::OFF_BN, a.bneg + t * kT2BN, S::BN_BYTES, &full[s]);
        issued = lt + 1;
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: C = x^_I x^_J^T, then U += K V ----------------
    if (lane == 0) {
      constexpr uint32_t idesc_c = tc::instr_desc(2, kT2BM, kT2BN);   // TF32
      constexpr uint32_t idesc_u = tc::instr_desc(1, kT2BM, N);       // BF16
      constexpr uint32_t sbo_x = (K8 / 4) * 128;
      const uint32_t aH = smem_u32(sAh), aL = smem_u32(sAl);
      const uint64_t dAh = tc::smem_desc(aH, 128, sbo_x), dAl = tc::smem_desc(aL, 128, sbo_x);
      const uint64_t dB0 = tc::smem_desc(smem_u32(stage(0)), 128, sbo_x);
      const uint64_t dV0 = tc::smem_desc(smem_u32(stage(0)) + 2 * S::XB_BYTES, 128, 512);
      bool ok = mbar_wait_spin(a_full, 0);
      auto issue_c = [&](int p) -> bool {
        const int s = p % ST, b = p % NB;
        if (!mbar_wait_spin(&full[s], (uint32_t)((p / ST) & 1))) return false;
        tc::fence_after();
        const uint64_t dBh = dB0 + (uint64_t)s * (S::STAGE_BYTES >> 4), dBl = dBh + (S::XB_BYTES >> 4);
        const uint32_t dC = tbase + (uint32_t)(b * 32);
#pragma unroll
        for (int term = 0; term < 3; ++term) {
          const uint64_t A = term == 2 ? dAl : dAh;
          const uint64_t B = term == 1 ? dBl : dBh;
#pragma unroll
          for (int ks = 0; ks < K8 / 8; ++ks)
            tc::mma_tf32(dC, A + 16u * ks, B + 16u * ks, idesc_c, (term | ks) != 0);
        }
        tc::commit(&c_full[p % S::NCF]);
        return true;
      };
      if (ok) tc::fence_after();
      for (int p = 0; p < min(NB, nt) && ok; ++p) ok = issue_c(p);
      for (int p = 0; p < nt && ok; ++p) {
        if (*s_fail) { ok = false; break; }
        const int s = p % ST, b = p % NB;
        if (!mbar_wait_spin(&k_full[b], (uint32_t)((p / NB) & 1))) { ok = false; break; }
        tc::fence_after();
        const uint64_t dVh = dV0 + (uint64_t)s * (S::STAGE_BYTES >> 4), dVl = dVh + (S::V_BYTES >> 4);
        const uint32_t kcol = tbase + (uint32_t)(b * 32);
#pragma unroll
        for (int term = 0; term < 3; ++term) {
          const uint32_t A = kcol + (term == 2 ? 8u : 0u);   // K high | K low per 16 points
          const uint64_t B = term == 1 ? dVl : dVh;
#pragma unroll
          for (int ks = 0; ks < kT2BN / 16; ++ks)
            tc::mma_bf16_ts(tbase + S::COL_U, A + ks * 16, B + 16u * ks, idesc_u, (p | term | ks) != 0);
        }
        tc::commit(&empty[s]);
        if (p + NB < nt) {
          // buffer b takes tile p + NB's C only after these MMAs have read its K
          tc::commit(&b_free[b]);
          if (!mbar_wait_spin(&b_free[b], (uint32_t)((p / NB) & 1))) { ok = false; break; }
          tc::fence_after();
          ok = issue_c(p + NB);
        }
      }
      if (!ok) *s_fail = 1;
      tc::commit(done);
    }
  } else {
    // ------ epilogue: 8 warps; warp (lane quadrant eq, set h) takes the tiles h, h + 2, ...
    //        with all 32 of their columns, in two 16-column halves ------
    const int eq = warp & 3;
    const int half = (warp - 2) >> 2;   // tile set; also the half of U it reads back
    const int il = eq * 32 + lane;
    const long long i = row0 + il;
    const uint32_t lane_base = (uint32_t)(eq * 32) << 16;
    const float ai = a.params->c0f + a.bneg[i];   // bneg covers the padded rows (zero there)
    bool ok = true;
    for (int lt = half; lt < nt; lt += 2) {
      const int b = lt % NB;
      // b_J is read from the stage: wait for its copy too (the stage is refilled only after
      // this tile's contraction, which waits for this warp's K)
      const bool ready =
          t2_warp_wait(&c_full[lt % S::NCF], (uint32_t)((lt / S::NCF) & 1)) &&
          (!BJ || t2_warp_wait(&full[lt % ST], (uint32_t)((lt / ST) & 1)));
      if (!__all_sync(0xffffffffu, ready && !*s_fail)) { ok = false; break; }
      tc::fence_after();
      const float* bj = reinterpret_cast<const float*>(stage(lt % ST) + S::OFF_BN);
      // all 32 columns of C in one tensor-memory round trip; each pair's K high and low parts
      // are written back into the pair's own registers (no extra registers live)
      const uint32_t ccol = tbase + lane_base + (uint32_t)(b * 32);
      uint32_t c[32];
      tc::tmem_ld16x2(ccol, c);
      // two entries per packed FP32x2 instruction (FADD2 / FFMA2, the same rounding as the
      // scalar forms)
      const float2 ai2 = make_float2(ai, ai);
      const float2 minus1 = make_float2(-1.f, -1.f);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        // the exponent is <= log2 sigma^2 up to rounding (about 1e-6 relative in k)
        float2 e = ai2;
        if constexpr (BJ) e = __fadd2_rn(e, *reinterpret_cast<const float2*>(bj + 2 * q));
        e = __fadd2_rn(e, make_float2(__uint_as_float(c[2 * q]), __uint_as_float(c[2 * q + 1])));
        const float2 k = make_float2(ex2_approx(e.x), ex2_approx(e.y));
        const __nv_bfloat162 h = __floats2bfloat162_rn(k.x, k.y);
        const float2 r = __ffma2_rn(__bfloat1622float2(h), minus1, k);   // k - high part
        const __nv_bfloat162 l = __floats2bfloat162_rn(r.x, r.y);
        c[2 * q] = *reinterpret_cast<const uint32_t*>(&h);
        c[2 * q + 1] = *reinterpret_cast<const uint32_t*>(&l);
      }
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        // columns [16 hh, 16 hh + 16): high parts, then low parts (the A operand of the
        // contraction's k-step hh)
        const uint32_t hi[8] = {c[16 * hh + 0], c[16 * hh + 2], c[16 * hh + 4], c[16 * hh + 6],
                                c[16 * hh + 8], c[16 * hh + 10], c[16 * hh + 12], c[16 * hh + 14]};
        const uint32_t lo[8] = {c[16 * hh + 1], c[16 * hh + 3], c[16 * hh + 5], c[16 * hh + 7],
                                c[16 * hh + 9], c[16 * hh + 11], c[16 * hh + 13], c[16 * hh + 15]};
        tc::tmem_st8(ccol + 16 * hh, hi);
        tc::tmem_st8(ccol + 16 * hh + 8, lo);
      }
      tc::tmem_wait_st();
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&k_full[b]);
    }
    if (!ok) *s_fail = 1;
    const bool fin = ok && t2_warp_wait(done, 0);
    ok = __all_sync(0xffffffffu, fin && !*s_fail);
    if (ok && nt > 0) {
      tc::fence_after();
      float u[NH];
      t2_ld_cols<NH>(tbase + lane_base + S::COL_U + (uint32_t)(half * NH), u);
      if (a.nsplit == 1) {
        if (i < a.n) {
          const float lam = (float)a.params->lambda;
#pragma unroll
          for (int q = 0; q < NH; ++q) {
            const int r = half * NH + q;
            if (r < R)
              a.U[(long long)a.umap[r] * a.ldu + i] =
                  fmaf(lam, a.V[(long long)a.vmap[r] * a.ldv + i], u[q]);
          }
        }
      } else {
        float* part = a.partials + slot * N * kT2BM;
#pragma unroll
        for (int q = 0; q < NH; ++q) part[(half * NH + q) * kT2BM + il] = u[q];
      }
    } else if (ok && a.nsplit > 1) {
      float* part = a.partials + slot * N * kT2BM;
#pragma unroll
      for (int q = 0; q < NH; ++q) part[(half * NH + q) * kT2BM + il] = 0.f;
    }
  }

  // -------- all roles: release tensor memory; last CTA of the row block reduces --------
  if (warp == 1) {
    if (lane == 0) (void)mbar_wait_backoff(done, 0);
    __syncwarp();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 1) tc::tmem_dealloc(tbase, kT2Cols);
  if (*s_fail) {
    if (tid == 0) {
      atomicOr(a.status, kStatusTimeout);
      // let the copies still in flight land before the CTA's shared memory goes away
      (void)mbar_wait_bounded(a_full, 0);
      for (int lt2 = max(0, issued - S::ST); lt2 < issued; ++lt2)
        (void)mbar_wait_bounded(&full[lt2 % S::ST], (uint32_t)((lt2 / S::ST) & 1));
    }
    return;
  }
  if (a.nsplit == 1) return;
  __threadfence();
  __syncthreads();
  if (tid == 0) *s_last = (atomicAdd(&a.counters[rb], 1) == a.nsplit - 1);
  __syncthreads();
  if (!*s_last) return;
  __threadfence();
  const float* base = a.partials + (long long)rb * a.nsplit * N * kT2BM;
  const float lam = (float)a.params->lambda;
  for (int idx = tid; idx < R * kT2BM; idx += kT2Threads) {
    const int r = idx / kT2BM, il = idx - r * kT2BM;
    const long long i = row0 + il;
    if (i >= a.n) continue;
    float u = 0.f;
    for (int s2 = 0; s2 < a.nsplit; ++s2) u += __ldcg(base + ((long long)s2 * N + r) * kT2BM + il);
    a.U[(long long)a.umap[r] * a.ldu + i] = fmaf(lam, a.V[(long long)a.vmap[r] * a.ldv + i], u);
  }
  if (tid == 0) a.counters[rb] = 0;
}

template <int K8, int N, bool BJ>
__global__ void __launch_bounds__(kT2Threads, 4) kmv_tc2_kernel(const Tc2DevArgs a) {
  const int rb = blockIdx.x / a.nsplit;
  tc2_body<K8, N, BJ>(a, rb, blockIdx.x - rb * a.nsplit, a.R);
}

// Many problems in one launch: CTA b takes work item items[b] = (problem, row block, split)
// with that problem's arguments; a problem with no live columns is skipped.
template <int K8, int N, bool BJ>
__global__ void __launch_bounds__(kT2Threads, 4) kmv_tc2_batch_kernel(
    const Tc2DevArgs* __restrict__ args, const int4* __restrict__ items) {
  __shared__ Tc2DevArgs s_a;
  const int4 it = items[blockIdx.x];
  if (threadIdx.x == 0) s_a = args[it.x];
  __syncthreads();
  const int R = s_a.R_dev ? *s_a.R_dev : s_a.R;
  if (R <= 0) return;
  tc2_body<K8, N, BJ>(s_a, it.y, it.z, R);
}

// The BF16 high and low parts of every problem's live V columns (as pack_v_kernel, one
// problem per grid row): K-major canonical images of N rows (columns of V) x 32 points.
__global__ void pack_v_batch_kernel(const Tc2DevArgs* __restrict__ args, int N) {
  const Tc2DevArgs& a = args[blockIdx.y];
  const int R = a.R_dev ? *a.R_dev : a.R;
  if (R <= 0) return;
  const long long ntiles = a.ntiles;
  const long long per_tile = (long long)N * kT2BN;
  __nv_bfloat16* Vhi = const_cast<__nv_bfloat16*>(a.V_hi);
  __nv_bfloat16* Vlo = const_cast<__nv_bfloat16*>(a.V_lo);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < ntiles * per_tile;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long t = idx / per_tile;
    const int rem = (int)(idx - t * per_tile);
    const int r = rem / kT2BN, jj = rem - r * kT2BN;
    const long long j = t * kT2BN + jj;
    const float v = (r < R && j < a.n) ? a.V[(long long)a.vmap[r] * a.ldv + j] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
    const long long off = t * per_tile + tc::canon_offset(r, jj, 2, kT2BN / 8) / 2;
    Vhi[off] = h;
    Vlo[off] = l;
  }
}

template <int K8, int N, bool BJ>
struct Tc2Inst {
  using S = Tc2Shape<K8, N, BJ>;
  // CTAs per SM: shared memory, tensor memory (512 columns) and the launch bound.
  static int occupancy() {
    static int occ = -1;
    static std::once_flag once;
    std::call_once(once, [] {
      auto fn = kmv_tc2_kernel<K8, N, BJ>;
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
      cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      int dev = 0, smem_sm = 0;
      cudaGetDevice(&dev);
      if (cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
          cudaSuccess)
        smem_sm = 228 * 1024;
      const int by_smem = smem_sm / (int)(S::SMEM + 1024);
      occ = std::max(1, std::min({by_smem, (int)(512 / kT2Cols), 4}));
    });
    return occ;
  }
  static cudaError_t launch(TcLaunch& L, cudaStream_t s) {
    KmvPlan p = L.nsplit > 0 ? plan_split_forced(L.n, kT2BM, N, 4, L.nsplit)
                             : plan_split(L.n, kT2BM, N, 4, L.num_sms * occupancy());
    p = tc_bound_split(p, L.n, kT2BM, N, kT2BN);
    const size_t pbytes = p.nsplit > 1 ? (size_t)p.n_rb * p.nsplit * N * kT2BM * 4 : 0;
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
    const long long ntiles = (L.n + kT2BN - 1) / kT2BN;
    launch_pack_v(L, N, ntiles, s);
    Tc2DevArgs a;
    a.A_hi = L.X_hi;
    a.A_lo = L.X_lo;
    a.B_hi = L.X_hi + L.X_off;
    a.B_lo = L.X_lo + L.X_off;
    a.bneg = L.bneg;
    a.V_hi = static_cast<const __nv_bfloat16*>(L.V_hi);
    a.V_lo = static_cast<const __nv_bfloat16*>(L.V_lo);
    a.V = static_cast<const float*>(L.V);
    a.ldv = L.ldv;
    a.vmap = L.vmap;
    a.R = L.R;
    a.R_dev = nullptr;
    a.U = static_cast<float*>(L.U);
    a.ldu = L.ldu;
    a.umap = L.umap;
    a.n = L.n;
    a.params = L.params;
    a.tiles_per_split = (int)((ntiles + p.nsplit - 1) / p.nsplit);
    a.nsplit = (int)((ntiles + a.tiles_per_split - 1) / a.tiles_per_split);
    a.ntiles = (int)ntiles;
    a.partials = static_cast<float*>(L.partials);
    a.counters = L.counters;
    a.status = L.status;
    (void)occupancy();
    const int nrb = (int)((L.n + kT2BM - 1) / kT2BM);
    kmv_tc2_kernel<K8, N, BJ><<<nrb * a.nsplit, kT2Threads, S::SMEM, s>>>(a);
    return cudaGetLastError();
  }
};

template <int K8, bool BJ>
static cudaError_t tc2_dispatch_n(TcLaunch& L, cudaStream_t s) {
  const int r = std::max(L.R, L.n_min);
  if (r <= 16) return Tc2Inst<K8, 16, BJ>::launch(L, s);
  if (r <= 32) return Tc2Inst<K8, 32, BJ>::launch(L, s);
  if (r <= 64) return Tc2Inst<K8, 64, BJ>::launch(L, s);
  return cudaErrorInvalidValue;
}

// K8, the TF32 MMA's K (a multiple of 8), from the padded d: padded d 2 and 4 take the
// augmented column within one K step (K8 = 8); padded d 8 and 16 leave it to the epilogue
// (K8 = d).
static int tc2_k8(int DP) { return DP >= 8 ? DP : 8; }

cudaError_t launch_kmv_tc2(TcLaunch& L, cudaStream_t s) {
  if (L.R < 1 || L.R > 64 || !L.X_hi || !L.X_lo) return cudaErrorInvalidValue;
  switch (L.DP) {
    case 2:
    case 4: return tc2_dispatch_n<8, false>(L, s);
    case 8: return tc2_dispatch_n<8, true>(L, s);
    case 16: return tc2_dispatch_n<16, true>(L, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pack_x_tf32(const float* xhat, const float* bneg, const DevParams* params,
                               int DP, long long n, long long ld128, float* X_hi, float* X_lo,
                               long long X_off, int num_sms, cudaStream_t s, bool aug) {
  const int K8 = tc2_k8(DP);
  const long long total = ld128 * K8;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 8LL * num_sms);
  pack_x_tf32_kernel<<<blocks, 256, 0, s>>>(xhat, bneg, params, DP, K8, aug ? 1 : 0, n, ld128,
                                            X_hi, X_lo, X_hi + X_off, X_lo + X_off);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Batched launches: many problems' K V in one launch (padded d <= 8, K8 = 8, b_j in the
// epilogue, the rows packed without the augmented column).
// ---------------------------------------------------------------------------------------
size_t tc2_batch_args_bytes(int B) { return sizeof(Tc2DevArgs) * (size_t)B; }

cudaError_t tc2_batch_upload_args(const TcLaunch* L, int B, void* args_dev, cudaStream_t s) {
  std::vector<Tc2DevArgs> h((size_t)B);
  for (int b = 0; b < B; ++b) {
    const TcLaunch& l = L[b];
    if (l.DP > 8 || l.nsplit < 1) return cudaErrorInvalidValue;
    Tc2DevArgs& a = h[b];
    const long long ntiles = (l.n + kT2BN - 1) / kT2BN;
    a.A_hi = l.X_hi;
    a.A_lo = l.X_lo;
    a.B_hi = l.X_hi + l.X_off;
    a.B_lo = l.X_lo + l.X_off;
    a.bneg = l.bneg;
    a.V_hi = static_cast<const __nv_bfloat16*>(l.V_hi);
    a.V_lo = static_cast<const __nv_bfloat16*>(l.V_lo);
    a.V = static_cast<const float*>(l.V);
    a.ldv = l.ldv;
    a.vmap = l.vmap;
    a.R = l.R;
    a.R_dev = l.R_dev;
    a.U = static_cast<float*>(l.U);
    a.ldu = l.ldu;
    a.umap = l.umap;
    a.n = l.n;
    a.params = l.params;
    a.tiles_per_split = (int)((ntiles + l.nsplit - 1) / l.nsplit);
    a.nsplit = (int)((ntiles + a.tiles_per_split - 1) / a.tiles_per_split);
    if (a.nsplit != l.nsplit || a.tiles_per_split > kTcMaxSplitTiles) return cudaErrorInvalidValue;
    a.ntiles = (int)ntiles;
    a.partials = static_cast<float*>(l.partials);
    a.counters = l.counters;
    a.status = l.status;
  }
  return cudaMemcpyAsync(args_dev, h.data(), sizeof(Tc2DevArgs) * (size_t)B,
                         cudaMemcpyHostToDevice, s);
}

template <int N>
static void tc2_batch_prime() {
  static std::once_flag once;
  std::call_once(once, [] {
    auto fn = kmv_tc2_batch_kernel<8, N, true>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)Tc2Shape<8, N, true>::SMEM);
    cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  });
}

void prime_kmv_tc2_batch() {
  tc2_batch_prime<16>();
  tc2_batch_prime<32>();
}

template <int N>
static cudaError_t tc2_batch_launch(const Tc2DevArgs* args, int B, const int4* items,
                                    int n_items, cudaStream_t s) {
  tc2_batch_prime<N>();
  pack_v_batch_kernel<<<dim3(64, (unsigned)B), 256, 0, s>>>(args, N);
  if (n_items > 0)
    kmv_tc2_batch_kernel<8, N, true><<<n_items, kT2Threads, Tc2Shape<8, N, true>::SMEM, s>>>(
        args, items);
  return cudaGetLastError();
}

cudaError_t launch_kmv_tc2_batch(const void* args_dev, int B, const int4* items, int n_items,
                                 int R_max, cudaStream_t s) {
  const Tc2DevArgs* args = static_cast<const Tc2DevArgs*>(args_dev);
  if (B < 1 || R_max < 1 || R_max > 32) return cudaErrorInvalidValue;
  return R_max <= 16 ? tc2_batch_launch<16>(args, B, items, n_items, s)
                     : tc2_batch_launch<32>(args, B, items, n_items, s);
}

}  // namespace ulisse
