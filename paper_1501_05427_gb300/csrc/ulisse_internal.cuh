// Internal declarations of libulisse: device helpers, shared structs and launchers.
// Nothing here is part of the public ABI (include/ulisse.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ulisse {

constexpr int kMaxD = 16;
constexpr int kMaxP = kMaxD + 2;
constexpr int kBN = 64;          // points per staged j-tile
constexpr int kStages = 3;       // staged j-tiles in flight per CTA
constexpr int kMaxRChunk = 32;   // right-hand sides per K V launch
constexpr int kMaxM = 64;        // rank of the gradient's bilinear form per launch
constexpr int kGtScratchRows = 128 + 48;   // tensor-core gradient operand scratch (x tc_ld)

// Device status bits (OR-ed into the context's status word).
constexpr int kStatusBreakdown = 1;
constexpr int kStatusMaxIter = 2;
constexpr int kStatusTimeout = 4;
constexpr int kStatusBadM = 8;

// Random-stream purposes (fourth Philox counter word, estimator index in bits 8..15).
constexpr uint64_t kPurposeProbe = 1;
constexpr uint64_t kPurposeUlisse = 2;
constexpr uint64_t kPurposeSgld = 3;
constexpr uint64_t kPurposeWsRows = 4;

// Scalars derived from psi on the device (written by the prescale kernel).
struct DevParams {
  double psi[kMaxP];
  double inv_l[kMaxD];   // 1 / l_d
  double sigma2;         // sigma^2
  double lambda;         // lambda (noise variance)
  float c0f;             // log2(sigma^2)
  float c1f;             // log2(e) / 2, so k_s = exp2(c0 - c1 * dist)
  float lambdaf;
  float pad;
};

// Per-column solver state (Algorithm 1 + ULISSE truncation, Sec. 4).
enum ColPhase { kPre = 0, kTail = 1, kDone = 2 };
struct ColState {
  double ee;      // e_m^T e_m
  int phase;      // ColPhase
  int l;          // early-stop iteration (0 until reached)
  int m;          // CG iterations done
  int outcome;    // 0 ok, 3 breakdown, 4 max_iter
  int J[2];       // accepted steps after the early stop, per estimator
  int n_est;      // 1 or 2 estimators
  int est_off;    // first estimator column in the estimate buffer
  int colid;      // random-stream column index
  int pad;
  double best_ee; // warm-started solves: smallest e^T e seen (its iterate is kept in Sbest)
};

// ------------------------------------------------------------------------------------
// Philox4x64-10 (Salmon et al., SC'11), from the published round function.
// ------------------------------------------------------------------------------------
__host__ __device__ inline void philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2,
                                              uint64_t c3, uint64_t k0, uint64_t k1,
                                              uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
#ifdef __CUDA_ARCH__
    const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
#else
    const unsigned __int128 p0 = (unsigned __int128)M0 * c0;
    const unsigned __int128 p1 = (unsigned __int128)M1 * c2;
    const uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    const uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
#endif
    const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += W0; k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Uniform on [0,1) from the top 53 bits.
__host__ __device__ inline double u01_53(uint64_t w) {
  return (double)(w >> 11) * (1.0 / 9007199254740992.0);
}

// Standard normal from two words (Box-Muller, first of the pair), in double.
__device__ inline double box_muller(uint64_t w0, uint64_t w1) {
  const double u1 = u01_53(w0), u2 = u01_53(w1);
  return sqrt(-2.0 * log(1.0 - u1)) * cos(6.283185307179586 * u2);
}

// ------------------------------------------------------------------------------------
// Bulk asynchronous copies (TMA unit) into shared memory, tracked by an mbarrier.
// ------------------------------------------------------------------------------------
__device__ inline uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ inline void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ inline void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(
          smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

// 1-D bulk copy global -> shared; dst, src 16-byte aligned, bytes a multiple of 16.
__device__ inline void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ inline bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: about a second at most, then false (the caller reports a timeout).
__device__ inline bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (it > 16) __nanosleep(256);
  }
  return false;
}

// Bounded wait for short, latency-critical handoffs (about a second at most).
__device__ inline bool mbar_wait_spin(uint64_t* bar, uint32_t parity) {
  for (int it = 0; it < (1 << 25); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (it > (1 << 16)) __nanosleep(32);
  }
  return false;
}

// Bounded wait for a single thread with nothing else to do meanwhile (a producer or an MMA
// issuer): it sleeps between polls so that polling takes no issue slots from the warps that
// compute (about a second at most, then false).
__device__ inline bool mbar_wait_backoff(uint64_t* bar, uint32_t parity) {
  for (int it = 0; it < (1 << 24); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    __nanosleep(64);
  }
  return false;
}

__device__ inline float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ------------------------------------------------------------------------------------
// Block reductions (fixed order: deterministic).
// ------------------------------------------------------------------------------------
__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int NT>
__device__ inline double block_sum(double v, double* scratch /* >= NT/32 */) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) scratch[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < NT / 32; ++i) t += scratch[i];
    scratch[0] = t;
  }
  __syncthreads();
  t = scratch[0];
  __syncthreads();
  return t;
}

// ------------------------------------------------------------------------------------
// Launch descriptors.
// ------------------------------------------------------------------------------------
// kModeDLam: dK/dlog lambda = lambda I (no tiles, only the diagonal term).
enum KmvMode { kModeK = 0, kModeDLen = 1, kModeDSig = 2, kModeDLam = 3 };

// Where the mixed path forms the cross term x^_i . x^_j (ulisse_config.tc_cross_term).
constexpr int kCrossPipe = 1;     // FP32 FMAs in the epilogue (kmv_tc_kernel)
constexpr int kCrossTensor = 2;   // 3xTF32 on the tensor cores (kmv_tc2_kernel)

struct KmvLaunch {
  const void* xhat;      // ldn x DP prescaled inputs (x / l), zero padded
  long long n, ldn;
  int d, DP;
  const void* V;         // column c of the operand at V + c * ldv
  long long ldv;
  const int* vmap;       // operand columns, R entries
  int R;                 // right-hand sides (<= kMaxRChunk)
  void* U;               // result column c at U + c * ldu
  long long ldu;
  const int* umap;       // result columns, R entries
  const DevParams* params;
  int mode;              // KmvMode
  int which;             // dimension for kModeDLen
  int tm;                // rows per thread for K (0 = default)
  int r_min;             // compiled column count at least this (0: the smallest >= R)
  int nsplit;            // j-range split count (0: the launch plan's choice)
  int planned_nsplit;    // out: the split count used (or planned)
  void* partials;        // split-j scratch
  size_t partials_bytes;
  int* counters;         // one per row block, zero between launches
  int counters_len;
  int* status;
  int num_sms;
  // Set by the launcher when the scratch above is too small (it then returns
  // cudaErrorMemoryAllocation without launching).
  size_t need_partials_bytes;
  int need_counters;
  bool plan_only;        // only fill need_* (no launch): sizing scratch ahead of a capture
};

struct GradLaunch {
  const void* xhat;
  long long n, ldn;
  int d, DP;
  const void* A;         // left factors: column amap[m] of A, scaled by sa[m]
  const int* amap;
  const void* sa;        // device, M scales (element type of A)
  const void* B;         // right factors: column bmap[m] of B
  const int* bmap;
  long long ld;
  int M;
  const DevParams* params;
  double* partials;      // per-CTA FP64 partial sums, kMaxP each
  size_t partials_len;   // doubles
  int* counter;          // single counter, zero between launches
  double* g_out;         // device, d + 2 doubles
  int* status;
  int num_sms;
  size_t need_partials_len;  // set when partials_len is too small
  bool plan_only;            // only fill need_partials_len (no launch)
  // tensor-core pass (launch_grad_tc) only: row norms (launch_prescale_tc) and BF16 packed
  // scratch, high and low parts, kGtScratchRows x tc_ld elements each (tc_ld = n rounded up
  // to 128): the right operand image (2M <= 128 factor slots), then the point features Z
  const float* bneg;
  void* tc_hi;
  void* tc_lo;
  long long tc_ld;
  // padded d <= 8: the TF32 row images of launch_pack_x_tf32 (A rows at X_hi / X_lo, B rows
  // X_off floats further on), from which the pass forms the exponent's cross term on the
  // tensor cores; c_has_bj when they were packed with the augmented column (b_j in C)
  const float* X_hi;
  const float* X_lo;
  long long X_off;
  bool c_has_bj;
};

// Mixed-precision (tcgen05) K V launch: operands prepared by launch_prescale_tc.
struct TcLaunch {
  const float* xhat;     // prescaled inputs, ld x DP row-major (the SIMT layout)
  const float* bneg;     // -c1 |x^|^2 (launch_prescale_tc), ld128
  void* V_hi;            // BF16 packed operand tiles (written by the launch), ld128 x 64
  void* V_lo;
  const void* V;         // FP32 operand columns
  long long ldv;
  const int* vmap;
  int R;                 // right-hand sides (<= 64)
  const int* R_dev;      // batched launches: the live column count on the device (or null)
  void* U;
  long long ldu;
  const int* umap;
  long long n;
  int DP;
  const DevParams* params;
  int n_min;             // MMA N at least this (0: the smallest of 16, 32, 64 >= R)
  int nsplit;            // j-range split count (0: the launch plan's choice)
  int planned_nsplit;    // out: the split count used (or planned)
  void* partials;
  size_t partials_bytes;
  int* counters;
  int counters_len;
  int* status;
  int num_sms;
  size_t need_partials_bytes;
  int need_counters;
  bool plan_only;        // only fill need_* (no launch): sizing scratch ahead of a capture
  // tensor-core cross term (launch_kmv_tc2): TF32 images of the augmented rows
  // (launch_pack_x_tf32): A rows at X_hi / X_lo, B rows X_off floats further on
  const float* X_hi;
  const float* X_lo;
  long long X_off;
};

// Launchers (return cudaSuccess or the launch error).
cudaError_t launch_kmv_f32(KmvLaunch& L, cudaStream_t s);
cudaError_t launch_kmv_f32_dp2(KmvLaunch& L, cudaStream_t s);
cudaError_t launch_kmv_f32_dp4(KmvLaunch& L, cudaStream_t s);
cudaError_t launch_kmv_f32_dp8(KmvLaunch& L, cudaStream_t s);
cudaError_t launch_kmv_f32_dp16(KmvLaunch& L, cudaStream_t s);
cudaError_t launch_kmv_f64(KmvLaunch& L, cudaStream_t s);
cudaError_t launch_grad_f32(GradLaunch& L, cudaStream_t s);
cudaError_t launch_grad_f64(GradLaunch& L, cudaStream_t s);
cudaError_t launch_kmv_tc(TcLaunch& L, cudaStream_t s);
cudaError_t launch_grad_tc(GradLaunch& L, cudaStream_t s);
cudaError_t launch_kmv_tc2(TcLaunch& L, cudaStream_t s);
void launch_pack_v(const TcLaunch& L, int N, long long ntiles, cudaStream_t s);
// aug: rows carry the column term b_j (padded d 2 and 4 of the single-problem launches);
// false for the batched launches, whose epilogue adds it for every d.
cudaError_t launch_pack_x_tf32(const float* xhat, const float* bneg, const DevParams* params,
                               int DP, long long n, long long ld128, float* X_hi, float* X_lo,
                               long long X_off, int num_sms, cudaStream_t s, bool aug);
// Batched tensor-core K V (padded d <= 8): per problem a TcLaunch with the operand pointers,
// R or R_dev, and the forced split nsplit >= 1 (tiles per split <= kTcMaxSplitTiles);
// items: (problem, 128-row block, split) per CTA; R_max: the largest live column count.
size_t tc2_batch_args_bytes(int B);
cudaError_t tc2_batch_upload_args(const TcLaunch* L, int B, void* args_dev, cudaStream_t s);
cudaError_t launch_kmv_tc2_batch(const void* args_dev, int B, const int4* items, int n_items,
                                 int R_max, cudaStream_t s);
void prime_kmv_tc2_batch();
// Batched tensor-core gradient pass (problems of one padded width DP <= 8, M factor pairs):
// per problem a GradLaunch with the operands (as launch_grad_tc) and its split nsplit[b];
// items: (problem, 128-row block, split) per CTA.  prime_only: set the kernel attributes
// (ahead of a capture) and launch nothing.
size_t gt_batch_args_bytes(int B);
cudaError_t gt_batch_upload_args(const GradLaunch* L, const int* nsplit, int B, void* args_dev,
                                 cudaStream_t s);
cudaError_t launch_grad_tc_batch(const void* args_dev, int B, const int4* items, int n_items,
                                 int DP, int M, cudaStream_t s, bool prime_only = false);
cudaError_t launch_prescale_tc(const float* xhat, int DP, int d, long long n, long long ld,
                               float* bneg, int num_sms, cudaStream_t s);

}  // namespace ulisse
