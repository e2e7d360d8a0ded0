// Mixed-precision fused gradient pass on the 5th-generation tensor cores (Eq. gradient:unbiased,
// Sec. 4.1): the components of
//     g~_i = sum_m a_m^T dK_i b_m
// for all parameters at once, through W_ij = sum_m a_m[i] b_m[j] and P_ij = k_s(i,j) W_ij:
//     g~_{log l_k}     = sum_ij P_ij (x^_ik - x^_jk)^2
//     g~_{log sigma^2} = sum_ij P_ij
//     g~_{log lambda}  = lambda sum_i W_ii.
// Both double sums weigh the pair (i, j) by a symmetric function (k_s and the squared
// difference), so they take each unordered pair once with the symmetric weight
//     W'_ij = W_ij + W_ji = [A^_i | b_i] . [b_j | A^_j]     (A^ = the scaled a-columns),
// a product over 2M factors: the pass visits, for the block of 128 rows I, only the 32-point
// tiles J at or after the block's own points (J >= I), with weight 1/2 on the four tiles of
// I itself (there both (i, j) and (j, i) are visited).  With P'_ij = k_s(i,j) W'_ij on the
// visited pairs,
//     g~_{log l_k}     = sum_i [ x^_ik^2 S_i - 2 x^_ik G_ik + H_ik ],
//                        S_i = sum_j P'_ij,  G_ik = sum_j P'_ij x^_jk,  H_ik = sum_j P'_ij x^_jk^2
//     g~_{log sigma^2} = sum_i S_i,
// so half the kernel values of the full square are formed.  Nothing is written per point j,
// which is why the symmetry is free here (a K V product would have to add K_IJ^T V_I to the
// rows of J).  For a block of 128 rows I and each visited 32-point tile J:
//   1. W'_IJ = [A^ | B]_I [B | A^]_J^T on the tensor cores (K = 2M factors, both operands
//      split into BF16 high + low parts: three products), into tensor memory;
//   2. for padded d <= 8, C_IJ = A_I B_J^T on the tensor cores as in the K V pass (the TF32
//      row images A_j = x^_j, B_j = 2 c1 x^_j, three TF32 products) into its own tensor-memory
//      buffer; the epilogue warps read W and C back (tcgen05.ld), form the kernel values as the
//      K V kernel does (exponent (a_i + b_j) + C_ij from the row norms, one ex2; for d = 16
//      the cross term on the FP32 pipe), multiply, split P into BF16 high + low parts and
//      store them over W's own tensor-memory columns;
//   3. [S | G | H]_I += P_IJ Z_J on the tensor cores, Z_j = [x^_j, x^_j^2, 1] split the same
//      way, accumulated in tensor memory across all tiles of the CTA's j range.
// The per-row combination and the diagonal sum run in FP64 at the end; CTA partials are summed
// in a fixed order by the last CTA to arrive (as in the SIMT gradient kernel).  Warp 0 streams
// B_J's TF32 image (x^_J for d = 16), the row norms, B^_J and Z_J into a 3- or 4-stage ring
// with bulk copies; one thread of warp 1 issues the MMAs; eight epilogue warps (a tensor-memory
// lane quadrant and half of the tile's 32 columns each) make P.  W/P tiles are double-buffered;
// a buffer is refilled only after the MMAs that read it have completed.  The single C buffer
// takes the next tile's product as soon as the eight warps have read it, so those MMAs run
// during the current tile's arithmetic.  Every wait is bounded.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "kmv_kernel.cuh"
#include "tc_common.cuh"

namespace ulisse {

constexpr int kGtBN = 32;
constexpr int kGtBM = 128;
constexpr int kGtThreads = 320;    // warp 0 producer, warp 1 MMA issuer, warps 2-9 epilogue
constexpr uint32_t kGtCols = 128;  // tensor-memory columns per CTA
constexpr int kGtZOff = 128;       // Z image offset in the packed scratch, in units of ld128
static_assert(16 * 8 <= kGtZOff && kGtZOff + 48 <= kGtScratchRows,
              "operand images exceed the gradient scratch");

__device__ inline void split_bf16(float v, __nv_bfloat16& h, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(v);
  l = __float2bfloat16_rn(v - __bfloat162float(h));
}

// Right operand [b_j | A^_j] of every 32-point tile as BF16 high and low parts: a K-major
// canonical image of 32 points (rows) x K1 factor slots, slot m < M holding b_m[j] and slot
// M + m holding sa[m] a_m[j]; slots >= 2M and points j >= n are zero.
__global__ void pack_bt_kernel(const float* __restrict__ B, const int* __restrict__ bmap,
                               const float* __restrict__ A, const int* __restrict__ amap,
                               const float* __restrict__ sa, long long ld, int M, int K1,
                               long long n, long long ntiles, __nv_bfloat16* __restrict__ Bhi,
                               __nv_bfloat16* __restrict__ Blo) {
  const long long per_tile = (long long)kGtBN * K1;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < ntiles * per_tile;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long t = idx / per_tile;
    const int rem = (int)(idx - t * per_tile);
    const int m = rem / kGtBN, j = rem - m * kGtBN;
    const long long jj = t * kGtBN + j;
    float v = 0.f;
    if (jj < n) {
      if (m < M) v = B[(long long)bmap[m] * ld + jj];
      else if (m < 2 * M) v = sa[m - M] * A[(long long)amap[m - M] * ld + jj];
    }
    __nv_bfloat16 h, l;
    split_bf16(v, h, l);
    const long long off = t * per_tile + tc::canon_offset(j, m, 2, K1 / 8) / 2;
    Bhi[off] = h;
    Blo[off] = l;
  }
}

// Z_j = [x^_j (DP), x^_j^2 (DP), 1, 0...] for every tile as BF16 high and low parts: a
// K-major canonical image of N2 rows (accumulator columns) x 32 points; points j >= n are zero.
__global__ void pack_z_kernel(const float* __restrict__ xhat, int DP, long long n, int N2,
                              long long ntiles, __nv_bfloat16* __restrict__ Zhi,
                              __nv_bfloat16* __restrict__ Zlo) {
  const long long per_tile = (long long)N2 * kGtBN;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < ntiles * per_tile;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long t = idx / per_tile;
    const int rem = (int)(idx - t * per_tile);
    const int c = rem / kGtBN, j = rem - c * kGtBN;
    const long long jj = t * kGtBN + j;
    float v = 0.f;
    if (jj < n) {
      if (c < DP) {
        v = xhat[jj * DP + c];
      } else if (c < 2 * DP) {
        const float x = xhat[jj * DP + (c - DP)];
        v = x * x;
      } else if (c == 2 * DP) {
        v = 1.f;
      }
    }
    __nv_bfloat16 h, l;
    split_bf16(v, h, l);
    const long long off = t * per_tile + tc::canon_offset(c, j, 2, kGtBN / 8) / 2;
    Zhi[off] = h;
    Zlo[off] = l;
  }
}

struct GtDevArgs {
  const float* xhat;   // x^ rows (ld x DP, row-major)
  const float* bneg;   // -c1 |x^|^2
  const __nv_bfloat16* Bt_hi;
  const __nv_bfloat16* Bt_lo;
  const __nv_bfloat16* Zt_hi;
  const __nv_bfloat16* Zt_lo;
  const float* A;      // left factors: column amap[m], scaled by sa[m]
  const int* amap;
  const float* sa;
  const float* B;      // right factors (the diagonal term reads them unsplit)
  const int* bmap;
  long long ld;
  int M;
  long long n;
  int d;
  const DevParams* params;
  int nsplit, ntiles;
  int n_cta;           // CTAs of this problem (row blocks x nsplit): the last one reduces
  // padded d <= 8: the TF32 row images of the tensor-core K V pass (8 columns, 32-row
  // K-major canonical tiles; high part and remainder), A_j = [x^_j, 1?] and
  // B_j = [2 c1 x^_j, b_j?]; c_has_bj when the augmented column carries b_j
  const float* XA_hi;
  const float* XA_lo;
  const float* XB_hi;
  const float* XB_lo;
  int c_has_bj;
  double* partials;
  int* counter;
  double* g_out;
  int* status;
};

// XC (padded d <= 8): the exponent's cross term C = A_I B_J^T on the tensor cores from the
// TF32 row images (three TF32 products, as the K V pass); the stage carries B_J's image instead
// of x^_J.  Padded d = 16 keeps the FP32 cross term (its accumulator leaves no room for C).
template <int DP, int KS>
struct GtShape {
  static constexpr bool XC = DP <= 8;
  static constexpr int K1 = 16 * KS;                   // factor slots (2M), padded
  static constexpr int N2 = (2 * DP + 1 + 15) / 16 * 16;
  static constexpr int K8 = 8;                         // columns of the TF32 row images
  static constexpr uint32_t A_BYTES = kGtBM * K1 * 2;  // one part of A^_I
  static constexpr uint32_t XA_BYTES = XC ? kGtBM * K8 * 4 : 0;   // one part of A_I (TF32)
  static constexpr uint32_t X_BYTES = XC ? 2 * kGtBN * K8 * 4 : kGtBN * DP * 4;
  static constexpr uint32_t XB_BYTES = kGtBN * K8 * 4;  // one part of B_J (TF32)
  static constexpr uint32_t BN_BYTES = kGtBN * 4;
  static constexpr uint32_t BT_BYTES = kGtBN * K1 * 2;
  static constexpr uint32_t Z_BYTES = N2 * kGtBN * 2;
  // stage: x^_J (FP32) or B_J (TF32 high | remainder), b_J, B^_J high | low, Z_J high | low
  static constexpr uint32_t OFF_BN = X_BYTES;
  static constexpr uint32_t OFF_BT = OFF_BN + BN_BYTES;
  static constexpr uint32_t OFF_Z = OFF_BT + 2 * BT_BYTES;
  static constexpr uint32_t STAGE_BYTES = OFF_Z + 2 * Z_BYTES;
  static constexpr int NBARS_FIXED = 2 + 2 + 2 + 1 + 2;  // w_full, p_full, free, done, c_full/free
  static constexpr uint32_t FIXED = 2 * A_BYTES + 2 * XA_BYTES + (8 + NBARS_FIXED) * 8 + 64;
  // four stages unless three keep one more CTA per SM (228 KB of shared memory per SM)
  static constexpr int occ_with(int st) {
    const int o = (int)((228u * 1024u) / (FIXED + st * STAGE_BYTES + 2048u));
    const int cap = DP >= 16 ? 2 : 3;   // the launch bounds' CTAs per SM
    return o < cap ? o : cap;
  }
  static constexpr int ST = occ_with(4) >= occ_with(3) ? 4 : 3;
  static constexpr uint32_t OFF_XA = 2 * A_BYTES;
  static constexpr uint32_t OFF_STAGES = OFF_XA + 2 * XA_BYTES;
  static constexpr uint32_t OFF_BARS = OFF_STAGES + ST * STAGE_BYTES;
  static constexpr int NBARS = 2 * ST + NBARS_FIXED;    // full, empty, then the fixed ones
  static constexpr uint32_t SMEM = OFF_BARS + NBARS * 8 + 64;
  // tensor-memory columns: two W/P buffers of 32, the C buffer of 32 (XC), then the
  // [G | H | S] accumulator
  static constexpr uint32_t COL_C = 64;
  static constexpr uint32_t COL_D2 = XC ? 96 : 64;
  static_assert(COL_D2 + N2 <= kGtCols, "tensor memory layout exceeds the allocation");
  static_assert(X_BYTES % 16 == 0 && STAGE_BYTES % 16 == 0 && A_BYTES % 16 == 0 &&
                    OFF_BT % 16 == 0 && OFF_Z % 16 == 0 && OFF_STAGES % 16 == 0,
                "bulk copies and descriptors need 16-byte alignment");
};

// Two 16-column tensor-memory loads at independent addresses and one wait.
__device__ inline void gt_tmem_ld16_two(uint32_t ta, uint32_t tb, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%32];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,"
      "%27,%28,%29,%30,%31}, [%33];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(ta), "r"(tb)
      : "memory");
}

__device__ inline bool gt_warp_wait(uint64_t* bar, uint32_t parity) {
  const bool ok = mbar_wait_spin(bar, parity);
  return __all_sync(0xffffffffu, ok);
}

// One CTA's work: row block rb, split sp of its tile range.  Shared by the single-problem
// kernel and the batched one.
template <int DP, int KS>
__device__ __forceinline__ void gt_body(const GtDevArgs& a, const int rb, const int sp) {
  using S = GtShape<DP, KS>;
  constexpr int ST = S::ST, K1 = S::K1, N2 = S::N2;
  constexpr int NACC = DP + 2;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ double s_red[8][NACC];
  unsigned char* sAh = smem;
  unsigned char* sAl = smem + S::A_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S::OFF_BARS);
  uint64_t* full = bars;
  uint64_t* empty = bars + ST;
  uint64_t* w_full = bars + 2 * ST;
  uint64_t* p_full = w_full + 2;
  uint64_t* b_free = p_full + 2;
  uint64_t* done = b_free + 2;
  uint64_t* c_full = done + 1;   // XC: C_J formed (MMA commit)
  uint64_t* c_free = done + 2;   // XC: the eight epilogue warps have read C_J
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + S::OFF_BARS + S::NBARS * 8);
  volatile int* s_fail = reinterpret_cast<volatile int*>(s_tmem + 1);
  int* s_last = reinterpret_cast<int*>(s_tmem + 2);
  auto stage = [&](int s) -> unsigned char* { return smem + S::OFF_STAGES + s * S::STAGE_BYTES; };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // Row block rb visits the tiles [4 rb, ntiles) (its own four tiles, then every later
  // one), cut into nsplit equal ranges; CTAs start in row-block order, longest ranges first.
  constexpr int kTilesPerBlock = kGtBM / kGtBN;
  const long long slot = (long long)rb * a.nsplit + sp;   // this CTA's partial-sum slot
  const long long row0 = (long long)rb * kGtBM;
  const int diag_end = min(kTilesPerBlock * (rb + 1), a.ntiles);   // tiles of I itself
  const int span = a.ntiles - kTilesPerBlock * rb;
  const int per = (span + a.nsplit - 1) / a.nsplit;
  const int tile_begin = kTilesPerBlock * rb + sp * per;
  const int nt = max(0, min(tile_begin + per, a.ntiles) - tile_begin);

  // [A^_I | B_I]: slot m < M holds sa[m] a_m[i], slot M + m holds b_m[i]; split into BF16
  // high and low parts (K-major canonical image).
  for (int idx = tid; idx < kGtBM * K1; idx += kGtThreads) {
    const int m = idx / kGtBM, il = idx - m * kGtBM;
    const long long i = row0 + il;
    float v = 0.f;
    if (i < a.n) {
      if (m < a.M) v = a.sa[m] * a.A[(long long)a.amap[m] * a.ld + i];
      else if (m < 2 * a.M) v = a.B[(long long)a.bmap[m - a.M] * a.ld + i];
    }
    __nv_bfloat16 h, l;
    split_bf16(v, h, l);
    const uint32_t off = tc::canon_offset(il, m, 2, K1 / 8);
    *reinterpret_cast<__nv_bfloat16*>(sAh + off) = h;
    *reinterpret_cast<__nv_bfloat16*>(sAl + off) = l;
  }
  if constexpr (S::XC) {
    // A_I's TF32 image (high part, then remainder): 128 rows of the packed images, which
    // are zero beyond n
    constexpr int kQ = kGtBM * S::K8 / 4;   // float4 per part
    float4* sx = reinterpret_cast<float4*>(smem + S::OFF_XA);
    const float4* gh = reinterpret_cast<const float4*>(a.XA_hi + row0 * S::K8);
    const float4* gl = reinterpret_cast<const float4*>(a.XA_lo + row0 * S::K8);
    for (int idx = tid; idx < 2 * kQ; idx += kGtThreads)
      sx[idx] = idx < kQ ? gh[idx] : gl[idx - kQ];
  }
  tc::fence_async_smem();
  if (tid == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1 + 8);   // MMA commit + the eight epilogue warps
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&w_full[b], 1);
      mbar_init(&p_full[b], 8);
      mbar_init(&b_free[b], 1);
    }
    mbar_init(done, 1);
    mbar_init(c_full, 1);
    mbar_init(c_free, 8);
    fence_barrier_init();
    *s_fail = 0;
  }
  if (warp == 1) tc::tmem_alloc(s_tmem, kGtCols);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *s_tmem;
  int issued = 0;   // tiles whose copies the producer started (lane 0 of warp 0)

  double acc[NACC];
#pragma unroll
  for (int k = 0; k < NACC; ++k) acc[k] = 0.0;

  if (warp == 0) {
    // ---------- producer: x^_J (or B_J's TF32 image), b_J, B^_J and Z_J into the ring ----------
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
        if constexpr (S::XC) {
          bulk_g2s(st, a.XB_hi + t * kGtBN * S::K8, S::XB_BYTES, &full[s]);
          bulk_g2s(st + S::XB_BYTES, a.XB_lo + t * kGtBN * S::K8, S::XB_BYTES, &full[s]);
        } else {
          bulk_g2s(st, a.xhat + t * kGtBN * DP, S::X_BYTES, &full[s]);
        }
        bulk_g2s(st + S::OFF_BN, a.bneg + t * kGtBN, S::BN_BYTES, &full[s]);
        unsigned char* bt = st + S::OFF_BT;
        bulk_g2s(bt, a.Bt_hi + t * kGtBN * K1, S::BT_BYTES, &full[s]);
        bulk_g2s(bt + S::BT_BYTES, a.Bt_lo + t * kGtBN * K1, S::BT_BYTES, &full[s]);
        unsigned char* zt = st + S::OFF_Z;
        bulk_g2s(zt, a.Zt_hi + t * N2 * kGtBN, S::Z_BYTES, &full[s]);
        bulk_g2s(zt + S::Z_BYTES, a.Zt_lo + t * N2 * kGtBN, S::Z_BYTES, &full[s]);
        issued = lt + 1;
      }
    }
  } else if (warp == 1) {
    // ------------- MMA issuer: W = A^ B^T and C = A B^T, then [G | H | S] += P Z -------------
    if (lane == 0) {
      constexpr uint32_t idesc_w = tc::instr_desc(1, kGtBM, kGtBN);
      constexpr uint32_t idesc_g = tc::instr_desc(1, kGtBM, N2);
      constexpr uint32_t sbo_k1 = (K1 / 8) * 128;
      const uint32_t aH = smem_u32(sAh), aL = smem_u32(sAl);
      auto issue_w = [&](int p) -> bool {
        const int s = p % ST, b = p & 1;
        if (!mbar_wait_spin(&full[s], (uint32_t)((p / ST) & 1))) return false;
        tc::fence_after();
        const uint32_t bH = smem_u32(stage(s) + S::OFF_BT);
        const uint32_t bL = bH + S::BT_BYTES;
        const uint32_t dW = tbase + (uint32_t)(b * 32);
#pragma unroll
        for (int term = 0; term < 3; ++term) {
          const uint32_t A = term == 2 ? aL : aH;
          const uint32_t B = term == 1 ? bL : bH;
#pragma unroll
          for (int ks = 0; ks < KS; ++ks)
            tc::mma_bf16(dW, tc::smem_desc(A + ks * 256, 128, sbo_k1),
                         tc::smem_desc(B + ks * 256, 128, sbo_k1), idesc_w, (term | ks) != 0);
        }
        tc::commit(&w_full[b]);
        return true;
      };
      // C_J = A_I B_J^T into the single C buffer (three TF32 products, K = 8)
      auto issue_c = [&](int p) -> bool {
        const int s = p % ST;
        if (!mbar_wait_spin(&full[s], (uint32_t)((p / ST) & 1))) return false;
        tc::fence_after();
        constexpr uint32_t idesc_c = tc::instr_desc(2, kGtBM, kGtBN);   // TF32
        constexpr uint32_t sbo_x = (S::K8 / 4) * 128;
        const uint32_t xa = smem_u32(smem + S::OFF_XA), xb = smem_u32(stage(s));
#pragma unroll
        for (int term = 0; term < 3; ++term) {
          const uint32_t A = term == 2 ? xa + S::XA_BYTES : xa;
          const uint32_t B = term == 1 ? xb + S::XB_BYTES : xb;
          tc::mma_tf32(tbase + S::COL_C, tc::smem_desc(A, 128, sbo_x),
                       tc::smem_desc(B, 128, sbo_x), idesc_c, term != 0);
        }
        tc::commit(c_full);
        return true;
      };
      bool ok = true;
      for (int p = 0; p < min(2, nt) && ok; ++p) ok = issue_w(p);
      if constexpr (S::XC) {
        if (ok && nt > 0) ok = issue_c(0);
      }
      for (int p = 0; p < nt && ok; ++p) {
        if (*s_fail) { ok = false; break; }
        const int s = p % ST, b = p & 1;
        if constexpr (S::XC) {
          // the C buffer takes tile p + 1 once the epilogue has read tile p's
          if (p + 1 < nt) {
            if (!mbar_wait_spin(c_free, (uint32_t)(p & 1))) { ok = false; break; }
            tc::fence_after();
            if (!issue_c(p + 1)) { ok = false; break; }
          }
        }
        if (!mbar_wait_spin(&p_full[b], (uint32_t)((p / 2) & 1))) { ok = false; break; }
        tc::fence_after();
        const uint32_t zH = smem_u32(stage(s) + S::OFF_Z);
        const uint32_t zL = zH + S::Z_BYTES;
        const uint32_t pcol = tbase + (uint32_t)(b * 32);
#pragma unroll
        for (int term = 0; term < 3; ++term) {
          const uint32_t A = pcol + (term == 2 ? 8u : 0u);   // P high | P low per 16 points
          const uint32_t B = term == 1 ? zL : zH;
#pragma unroll
          for (int ks = 0; ks < kGtBN / 16; ++ks)
            tc::mma_bf16_ts(tbase + S::COL_D2, A + ks * 16, tc::smem_desc(B + ks * 256, 128, 512),
                            idesc_g, (p | term | ks) != 0);
        }
        tc::commit(&empty[s]);
        if (p + 2 < nt) {
          // buffer b is rewritten by tile p + 2's W only after these MMAs have read P
          tc::commit(&b_free[b]);
          if (!mbar_wait_spin(&b_free[b], (uint32_t)((p / 2) & 1))) { ok = false; break; }
          tc::fence_after();
          ok = issue_w(p + 2);
        }
      }
      if (!ok) *s_fail = 1;
      if (nt > 0) tc::commit(done);   // a CTA with an empty range issues nothing and waits on nothing
    }
  } else {
    // ------------- epilogue: 8 warps, (lane quadrant, column half) each -------------
    const int eq = warp & 3;
    const int half = (warp - 2) >> 2;
    const int il = eq * 32 + lane;
    const long long i = row0 + il;
    const uint32_t lane_base = (uint32_t)(eq * 32) << 16;
    const float c0 = a.params->c0f, c1 = a.params->c1f;
    const float two_c1 = 2.f * c1;
    float xi[S::XC ? 1 : DP];
    if constexpr (!S::XC) {
#pragma unroll
      for (int k = 0; k < DP; ++k) xi[k] = (i < a.n) ? two_c1 * a.xhat[i * DP + k] : 0.f;
    }
    const float ai = c0 + ((i < a.n) ? a.bneg[i] : 0.f);
    const bool add_bj = !S::XC || !a.c_has_bj;   // else the augmented C carries b_j
    bool ok = true;
    for (int lt = 0; lt < nt; ++lt) {
      const int s = lt % ST, b = lt & 1;
      bool ready = gt_warp_wait(&full[s], (uint32_t)((lt / ST) & 1)) &&
                   gt_warp_wait(&w_full[b], (uint32_t)((lt / 2) & 1));
      if constexpr (S::XC) ready = ready && gt_warp_wait(c_full, (uint32_t)(lt & 1));
      if (!__all_sync(0xffffffffu, ready && !*s_fail)) { ok = false; break; }
      tc::fence_after();
      const uint32_t wcol = tbase + lane_base + (uint32_t)(b * 32 + half * 16);
      float w[16], cx[16];
      if constexpr (S::XC) {
        uint32_t r[32];
        gt_tmem_ld16_two(wcol, tbase + lane_base + S::COL_C + (uint32_t)(half * 16), r);
        tc::fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(c_free);   // the C buffer may take the next tile
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          w[q] = __uint_as_float(r[q]);
          cx[q] = __uint_as_float(r[16 + q]);
        }
      } else {
        tc::tmem_ld16(wcol, w);
      }
      if (tile_begin + lt < diag_end) {   // a tile of I itself: (i, j) and (j, i) both visited
#pragma unroll
        for (int q = 0; q < 16; ++q) w[q] *= 0.5f;
      }
      const float* tx = reinterpret_cast<const float*>(stage(s));
      const float* tb = reinterpret_cast<const float*>(stage(s) + S::OFF_BN);
      uint32_t hi[8], lo[8];
      // packed FP32x2 instructions: the cross term two coordinates at a time (FP32 pipe) or
      // the exponent two entries at a time (tensor-core C), the weight and the high/low split
      // two entries at a time
      const float2 minus1 = make_float2(-1.f, -1.f);
      const float2 ai2 = make_float2(ai, ai);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float ex[2];
        const float2 bj = *reinterpret_cast<const float2*>(tb + half * 16 + 2 * q);
        if constexpr (S::XC) {
          // (a_i + b_j) + C_ij, the order of the K V pass
          const float2 base = add_bj ? __fadd2_rn(ai2, bj) : ai2;
          const float2 e2 = __fadd2_rn(base, make_float2(cx[2 * q], cx[2 * q + 1]));
          ex[0] = e2.x;
          ex[1] = e2.y;
        } else {
#pragma unroll
          for (int h2 = 0; h2 < 2; ++h2) {
            const int j = half * 16 + 2 * q + h2;
            float xj[DP];
            load_row<float, DP>(tx + j * DP, xj);
            float2 acc = make_float2(ai + (h2 == 0 ? bj.x : bj.y), 0.f);
#pragma unroll
            for (int k = 0; k < DP; k += 2)
              acc = __ffma2_rn(make_float2(xi[k], xi[k + 1]), make_float2(xj[k], xj[k + 1]), acc);
            ex[h2] = acc.x + acc.y;
          }
        }
        const float2 pk = __fmul2_rn(make_float2(ex2_approx(fminf(ex[0], c0)),
                                                 ex2_approx(fminf(ex[1], c0))),
                                     make_float2(w[2 * q], w[2 * q + 1]));
        const __nv_bfloat162 h = __floats2bfloat162_rn(pk.x, pk.y);
        const float2 r = __ffma2_rn(__bfloat1622float2(h), minus1, pk);   // pk - high part
        const __nv_bfloat162 l = __floats2bfloat162_rn(r.x, r.y);
        hi[q] = *reinterpret_cast<const uint32_t*>(&h);
        lo[q] = *reinterpret_cast<const uint32_t*>(&l);
      }
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&empty[s]);   // x^_J (or nothing) and b_J consumed
      // P over this warp's own 16 W columns: high parts first, then low parts
      tc::tmem_st8(wcol, hi);
      tc::tmem_st8(wcol + 8, lo);
      tc::tmem_wait_st();
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&p_full[b]);
    }
    if (!ok) *s_fail = 1;
    const bool fin = ok && (nt == 0 || gt_warp_wait(done, 0));
    ok = __all_sync(0xffffffffu, fin && !*s_fail);
    if (ok && nt > 0) {
      tc::fence_after();
      if (half == 0) {
        float g[N2];
#pragma unroll
        for (int c = 0; c < N2 / 16; ++c) {
          float v[16];
          tc::tmem_ld16(tbase + lane_base + S::COL_D2 + (uint32_t)(c * 16), v);
#pragma unroll
          for (int q = 0; q < 16; ++q) g[c * 16 + q] = v[q];
        }
        if (i < a.n) {
          const double Ssum = g[2 * DP];
#pragma unroll
          for (int k = 0; k < DP; ++k) {
            const double x = a.xhat[i * DP + k];
            acc[k] = x * x * Ssum - 2.0 * x * (double)g[k] + (double)g[DP + k];
          }
          acc[DP] = Ssum;
        }
      } else if (sp == 0 && i < a.n) {
        // diagonal W_ii for the lambda component, once per row
        float wii = 0.f;
        for (int m = 0; m < a.M; ++m)
          wii = fmaf(a.sa[m] * a.A[(long long)a.amap[m] * a.ld + i],
                     a.B[(long long)a.bmap[m] * a.ld + i], wii);
        acc[DP + 1] = wii;
      }
    }
  }

  // -------- all roles: release tensor memory; CTA reduction; last CTA sums the partials -------
  if (warp == 1) {
    if (lane == 0 && nt > 0) (void)mbar_wait_spin(done, 0);
    __syncwarp();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 1) tc::tmem_dealloc(tbase, kGtCols);
  if (*s_fail) {
    if (tid == 0) {
      atomicOr(a.status, kStatusTimeout);
      // let the copies still in flight land before the CTA's shared memory goes away
      for (int lt2 = max(0, issued - S::ST); lt2 < issued; ++lt2)
        (void)mbar_wait_bounded(&full[lt2 % S::ST], (uint32_t)((lt2 / S::ST) & 1));
    }
    return;
  }
  if (warp >= 2) {
#pragma unroll
    for (int k = 0; k < NACC; ++k) {
      const double v = warp_sum(acc[k]);
      if (lane == 0) s_red[warp - 2][k] = v;
    }
  }
  __syncthreads();
  double* part = a.partials + slot * kMaxP;
  if (tid < NACC) {
    double v = 0.0;
    for (int ww = 0; ww < 8; ++ww) v += s_red[ww][tid];
    // slots: lengthscales 0..d-1, then sigma^2 at d, lambda at d+1
    if (tid < a.d) part[tid] = v;
    else if (tid == DP) part[a.d] = v;
    else if (tid == DP + 1) part[a.d + 1] = v;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) *s_last = (atomicAdd(a.counter, 1) == a.n_cta - 1);
  __syncthreads();
  if (!*s_last) return;
  __threadfence();
  if (tid < a.d + 2) {
    double v = 0.0;
    for (int b = 0; b < a.n_cta; ++b) v += __ldcg(a.partials + (long long)b * kMaxP + tid);
    if (tid == a.d + 1) v *= a.params->lambda;
    a.g_out[tid] = v;
  }
  if (tid == 0) *a.counter = 0;
}

template <int DP, int KS>
__global__ void __launch_bounds__(kGtThreads, DP >= 16 ? 2 : 3) grad_tc_kernel(const GtDevArgs a) {
  const int rb = blockIdx.x / a.nsplit;
  gt_body<DP, KS>(a, rb, blockIdx.x - rb * a.nsplit);
}

// Many problems of one input width in one launch: CTA b takes work item items[b] =
// (problem, row block, split) with that problem's arguments.
template <int DP, int KS>
__global__ void __launch_bounds__(kGtThreads, DP >= 16 ? 2 : 3) grad_tc_batch_kernel(
    const GtDevArgs* __restrict__ args, const int4* __restrict__ items) {
  __shared__ GtDevArgs s_a;
  const int4 it = items[blockIdx.x];
  if (threadIdx.x == 0) s_a = args[it.x];
  __syncthreads();
  gt_body<DP, KS>(s_a, it.y, it.z);
}

// The operand images of every problem of a batched launch (one problem per grid row), as
// pack_bt_kernel and pack_z_kernel.
template <int DP, int KS>
__global__ void pack_gt_batch_kernel(const GtDevArgs* __restrict__ args) {
  using S = GtShape<DP, KS>;
  constexpr int K1 = S::K1, N2 = S::N2;
  const GtDevArgs& a = args[blockIdx.y];
  const long long ntiles = a.ntiles;
  __nv_bfloat16* Bhi = const_cast<__nv_bfloat16*>(a.Bt_hi);
  __nv_bfloat16* Blo = const_cast<__nv_bfloat16*>(a.Bt_lo);
  __nv_bfloat16* Zhi = const_cast<__nv_bfloat16*>(a.Zt_hi);
  __nv_bfloat16* Zlo = const_cast<__nv_bfloat16*>(a.Zt_lo);
  const long long per_b = (long long)kGtBN * K1, per_z = (long long)N2 * kGtBN;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
       idx < ntiles * (per_b + per_z); idx += (long long)gridDim.x * blockDim.x) {
    __nv_bfloat16 h, l;
    if (idx < ntiles * per_b) {
      const long long t = idx / per_b;
      const int rem = (int)(idx - t * per_b);
      const int m = rem / kGtBN, j = rem - m * kGtBN;
      const long long jj = t * kGtBN + j;
      float v = 0.f;
      if (jj < a.n) {
        if (m < a.M) v = a.B[(long long)a.bmap[m] * a.ld + jj];
        else if (m < 2 * a.M) v = a.sa[m - a.M] * a.A[(long long)a.amap[m - a.M] * a.ld + jj];
      }
      split_bf16(v, h, l);
      const long long off = t * per_b + tc::canon_offset(j, m, 2, K1 / 8) / 2;
      Bhi[off] = h;
      Blo[off] = l;
    } else {
      const long long z = idx - ntiles * per_b;
      const long long t = z / per_z;
      const int rem = (int)(z - t * per_z);
      const int c = rem / kGtBN, j = rem - c * kGtBN;
      const long long jj = t * kGtBN + j;
      float v = 0.f;
      if (jj < a.n) {
        if (c < DP) {
          v = a.xhat[jj * DP + c];
        } else if (c < 2 * DP) {
          const float x = a.xhat[jj * DP + (c - DP)];
          v = x * x;
        } else if (c == 2 * DP) {
          v = 1.f;
        }
      }
      split_bf16(v, h, l);
      const long long off = t * per_z + tc::canon_offset(c, j, 2, kGtBN / 8) / 2;
      Zhi[off] = h;
      Zlo[off] = l;
    }
  }
}

// Split of each row block's tile range into s CTAs.  The SMs share the visited tiles plus a
// fixed cost per CTA (the operand image, the pipeline fill and the reduction, about six
// tiles' worth); a CTA shares its SM with occ - 1 others, so the longest range (row block 0,
// ntiles / s tiles) takes about occ x its length and must not end the pass.
static int plan_gt_split(long long n_rb, long long ntiles, int num_sms, int occ) {
  const long long per_block = kGtBM / kGtBN;
  const long long visited = n_rb * ntiles - per_block * n_rb * (n_rb - 1) / 2;
  // no more than kTcMaxSplitTiles tiles per CTA: the sums accumulate in FP32 in tensor memory
  const int s_min = (int)((ntiles + kTcMaxSplitTiles - 1) / kTcMaxSplitTiles);
  long long best = -1;
  int best_s = s_min;
  for (int s = s_min; s <= std::max(64, s_min) && s <= ntiles; ++s) {
    const long long shared = (visited + 6 * n_rb * s + num_sms - 1) / num_sms;
    const long long longest = ((ntiles + s - 1) / s + 6) * occ;
    const long long cost = std::max(shared, longest);
    if (best < 0 || cost < best) {
      best = cost;
      best_s = s;
    }
  }
  return best_s;
}

// The TF32 row images of the K V pass (A rows at X_hi / X_lo, B rows X_off floats on).
static void gt_set_images(GtDevArgs& a, const GradLaunch& L) {
  a.XA_hi = L.X_hi;
  a.XA_lo = L.X_lo;
  a.XB_hi = L.X_hi ? L.X_hi + L.X_off : nullptr;
  a.XB_lo = L.X_lo ? L.X_lo + L.X_off : nullptr;
  a.c_has_bj = L.c_has_bj ? 1 : 0;
}

template <int DP, int KS>
struct GtInst {
  using S = GtShape<DP, KS>;
  static int occupancy() {
    static int occ = -1;
    static std::once_flag once;
    std::call_once(once, [] {
      auto fn = grad_tc_kernel<DP, KS>;
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
      cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      int dev = 0, smem_sm = 0;
      cudaGetDevice(&dev);
      if (cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
          cudaSuccess)
        smem_sm = 228 * 1024;
      const int by_smem = smem_sm / (int)(S::SMEM + 2048);
      occ = std::max(1, std::min({by_smem, (int)(512 / kGtCols), DP >= 16 ? 2 : 3}));
    });
    return occ;
  }
  static cudaError_t launch(GradLaunch& L, cudaStream_t s) {
    const int occ = occupancy();
    const long long ntiles = (L.n + kGtBN - 1) / kGtBN;
    const int n_rb = (int)((L.n + kGtBM - 1) / kGtBM);
    const int nsplit = plan_gt_split(n_rb, ntiles, L.num_sms, occ);
    const size_t need = (size_t)n_rb * nsplit * kMaxP;
    if (L.plan_only) {
      L.need_partials_len = need;
      return cudaSuccess;
    }
    if (need > L.partials_len) {
      L.need_partials_len = need;
      return cudaErrorMemoryAllocation;
    }
    __nv_bfloat16* hi = static_cast<__nv_bfloat16*>(L.tc_hi);
    __nv_bfloat16* lo = static_cast<__nv_bfloat16*>(L.tc_lo);
    const long long zoff = (long long)kGtZOff * L.tc_ld;
    {
      const long long total = ntiles * kGtBN * S::K1;
      const int blocks = (int)std::min<long long>((total + 255) / 256, 8LL * L.num_sms);
      pack_bt_kernel<<<blocks, 256, 0, s>>>(static_cast<const float*>(L.B), L.bmap,
                                            static_cast<const float*>(L.A), L.amap,
                                            static_cast<const float*>(L.sa), L.ld, L.M, S::K1,
                                            L.n, ntiles, hi, lo);
    }
    {
      const long long total = ntiles * S::N2 * kGtBN;
      const int blocks = (int)std::min<long long>((total + 255) / 256, 8LL * L.num_sms);
      pack_z_kernel<<<blocks, 256, 0, s>>>(static_cast<const float*>(L.xhat), DP, L.n, S::N2,
                                           ntiles, hi + zoff, lo + zoff);
    }
    GtDevArgs a;
    a.xhat = static_cast<const float*>(L.xhat);
    a.bneg = L.bneg;
    a.Bt_hi = hi;
    a.Bt_lo = lo;
    a.Zt_hi = hi + zoff;
    a.Zt_lo = lo + zoff;
    a.A = static_cast<const float*>(L.A);
    a.amap = L.amap;
    a.sa = static_cast<const float*>(L.sa);
    a.B = static_cast<const float*>(L.B);
    a.bmap = L.bmap;
    a.ld = L.ld;
    a.M = L.M;
    a.n = L.n;
    a.d = L.d;
    a.params = L.params;
    a.nsplit = nsplit;
    a.n_cta = n_rb * nsplit;
    a.ntiles = (int)ntiles;
    gt_set_images(a, L);
    a.partials = L.partials;
    a.counter = L.counter;
    a.g_out = L.g_out;
    a.status = L.status;
    grad_tc_kernel<DP, KS><<<n_rb * nsplit, kGtThreads, S::SMEM, s>>>(a);
    return cudaGetLastError();
  }
};

// KS = 16-wide steps of the 2M factor slots.
template <int DP>
static cudaError_t grad_tc_dispatch_m(GradLaunch& L, cudaStream_t s) {
  if (L.M <= 8) return GtInst<DP, 1>::launch(L, s);
  if (L.M <= 16) return GtInst<DP, 2>::launch(L, s);
  if (L.M <= 24) return GtInst<DP, 3>::launch(L, s);
  if (L.M <= 32) return GtInst<DP, 4>::launch(L, s);
  if (L.M <= 64) return GtInst<DP, 8>::launch(L, s);
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------------------
// Batched launches: many problems of one padded width in one launch.
// ---------------------------------------------------------------------------------------
size_t gt_batch_args_bytes(int B) { return sizeof(GtDevArgs) * (size_t)B; }

cudaError_t gt_batch_upload_args(const GradLaunch* L, const int* nsplit, int B, void* args_dev,
                                 cudaStream_t s) {
  std::vector<GtDevArgs> h((size_t)B);
  for (int b = 0; b < B; ++b) {
    const GradLaunch& l = L[b];
    const long long ntiles = (l.n + kGtBN - 1) / kGtBN;
    const long long n_rb = (l.n + kGtBM - 1) / kGtBM;
    if (l.M < 1 || l.M > kMaxM || nsplit[b] < 1 || l.DP != L[0].DP || !l.tc_hi || !l.tc_lo ||
        !l.X_hi || !l.X_lo ||
        (ntiles + nsplit[b] - 1) / nsplit[b] > kTcMaxSplitTiles)
      return cudaErrorInvalidValue;
    GtDevArgs& a = h[b];
    __nv_bfloat16* hi = static_cast<__nv_bfloat16*>(l.tc_hi);
    __nv_bfloat16* lo = static_cast<__nv_bfloat16*>(l.tc_lo);
    const long long zoff = (long long)kGtZOff * l.tc_ld;
    a.xhat = static_cast<const float*>(l.xhat);
    a.bneg = l.bneg;
    a.Bt_hi = hi;
    a.Bt_lo = lo;
    a.Zt_hi = hi + zoff;
    a.Zt_lo = lo + zoff;
    a.A = static_cast<const float*>(l.A);
    a.amap = l.amap;
    a.sa = static_cast<const float*>(l.sa);
    a.B = static_cast<const float*>(l.B);
    a.bmap = l.bmap;
    a.ld = l.ld;
    a.M = l.M;
    a.n = l.n;
    a.d = l.d;
    a.params = l.params;
    a.nsplit = nsplit[b];
    a.ntiles = (int)ntiles;
    a.n_cta = (int)(n_rb * nsplit[b]);
    gt_set_images(a, l);
    a.partials = l.partials;
    a.counter = l.counter;
    a.g_out = l.g_out;
    a.status = l.status;
  }
  return cudaMemcpyAsync(args_dev, h.data(), sizeof(GtDevArgs) * (size_t)B,
                         cudaMemcpyHostToDevice, s);
}

template <int DP, int KS>
static void gt_batch_prime() {
  static std::once_flag once;
  std::call_once(once, [] {
    auto fn = grad_tc_batch_kernel<DP, KS>;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)GtShape<DP, KS>::SMEM);
    cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  });
}

template <int DP, int KS>
static cudaError_t gt_batch_launch(const GtDevArgs* args, int B, const int4* items, int n_items,
                                   bool prime_only, cudaStream_t s) {
  gt_batch_prime<DP, KS>();
  if (prime_only) return cudaSuccess;
  pack_gt_batch_kernel<DP, KS><<<dim3(64, (unsigned)B), 256, 0, s>>>(args);
  if (n_items > 0)
    grad_tc_batch_kernel<DP, KS><<<n_items, kGtThreads, GtShape<DP, KS>::SMEM, s>>>(args, items);
  return cudaGetLastError();
}

template <int DP>
static cudaError_t gt_batch_dispatch_m(const GtDevArgs* args, int B, const int4* items,
                                       int n_items, int M, bool prime_only, cudaStream_t s) {
  if (M <= 8) return gt_batch_launch<DP, 1>(args, B, items, n_items, prime_only, s);
  if (M <= 16) return gt_batch_launch<DP, 2>(args, B, items, n_items, prime_only, s);
  if (M <= 24) return gt_batch_launch<DP, 3>(args, B, items, n_items, prime_only, s);
  if (M <= 32) return gt_batch_launch<DP, 4>(args, B, items, n_items, prime_only, s);
  if (M <= 64) return gt_batch_launch<DP, 8>(args, B, items, n_items, prime_only, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_grad_tc_batch(const void* args_dev, int B, const int4* items, int n_items,
                                 int DP, int M, cudaStream_t s, bool prime_only) {
  const GtDevArgs* args = static_cast<const GtDevArgs*>(args_dev);
  if (B < 1 && !prime_only) return cudaErrorInvalidValue;
  switch (DP) {
    case 2: return gt_batch_dispatch_m<2>(args, B, items, n_items, M, prime_only, s);
    case 4: return gt_batch_dispatch_m<4>(args, B, items, n_items, M, prime_only, s);
    case 8: return gt_batch_dispatch_m<8>(args, B, items, n_items, M, prime_only, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_grad_tc(GradLaunch& L, cudaStream_t s) {
  if (L.M < 1 || L.M > kMaxM || !L.tc_hi || !L.tc_lo || !L.bneg) return cudaErrorInvalidValue;
  if (L.DP <= 8 && (!L.X_hi || !L.X_lo)) return cudaErrorInvalidValue;
  switch (L.DP) {
    case 2: return grad_tc_dispatch_m<2>(L, s);
    case 4: return grad_tc_dispatch_m<4>(L, s);
    case 8: return grad_tc_dispatch_m<8>(L, s);
    case 16: return grad_tc_dispatch_m<16>(L, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ulisse
