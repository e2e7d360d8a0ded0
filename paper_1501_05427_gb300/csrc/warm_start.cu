// Learned warm start for the K s = y solve (Algorithm 1 accepts any initial iterate s_0;
// ULISSE stays unbiased for any s_0 chosen before the step's random draws).
//
// s_0 = K_s(X, Z) c,  c = MLP(psi) = W3^T tanh(W2^T tanh(W1^T z + b1) + b2) + b3,
// z = (psi - mu) / sd, Z a fixed set of anchor inputs.  The network is trained to shrink
// the initial residual e_0 = y - K s_0, which is what decides when the y solve reaches the
// early stop of Sec. 4.  Each step the chain records stores, at its parameters psi_t, m
// rows I_t drawn uniformly with replacement, y at those rows and
//     M_t = K(X_{I_t}, X; psi_t) K_s(X, Z; psi_t)          (m x A),
// so that y_{I_t} - M_t c is the initial residual on the rows I_t.  The loss is
//     1/B sum_b ( 1/m || y_{I_b} - M_b c_b ||^2 + rho || c_b ||^2 )
// over a minibatch of recorded pairs.  Kernels below: the recording (row sampling, the
// anchor columns of K_s, a tiled product of generated K rows with them), small FP32 matrix
// products, tanh and its derivative, column sums, the residual and its transpose product,
// and Adam.  Inference uses BF16 copies of the weights with FP32 accumulation.
#include <cuda_bf16.h>

#include <algorithm>

#include "warm_start.cuh"

namespace ulisse {
namespace ws {

constexpr int kTile = 16;

// C[M x N] = op(A) op(B) (+ bias[N]) (then tanh if act), FP32.  op(A) is A (M x K, row
// stride lda) or A^T (A stored K x M); op(B) is B (K x N) or B^T (B stored N x K).
template <bool TA, bool TB>
__global__ void gemm_kernel(int M, int N, int K, const float* __restrict__ A, int lda,
                            const float* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                            const float* __restrict__ bias, int act) {
  __shared__ float sA[kTile][kTile + 1];
  __shared__ float sB[kTile][kTile + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int row = blockIdx.y * kTile + ty, col = blockIdx.x * kTile + tx;
  float acc = 0.f;
  for (int k0 = 0; k0 < K; k0 += kTile) {
    const int ka = k0 + tx, kb = k0 + ty;
    float av = 0.f, bv = 0.f;
    if (row < M && ka < K) av = TA ? A[(long long)ka * lda + row] : A[(long long)row * lda + ka];
    if (col < N && kb < K) bv = TB ? B[(long long)col * ldb + kb] : B[(long long)kb * ldb + col];
    sA[ty][tx] = av;
    sB[ty][tx] = bv;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kTile; ++k) acc = fmaf(sA[ty][k], sB[k][tx], acc);
    __syncthreads();
  }
  if (row < M && col < N) {
    if (bias) acc += bias[col];
    if (act) acc = tanhf(acc);
    C[(long long)row * ldc + col] = acc;
  }
}

template <bool TA, bool TB>
static void gemm(cudaStream_t s, int M, int N, int K, const float* A, int lda, const float* B,
                 int ldb, float* C, int ldc, const float* bias, int act) {
  dim3 block(kTile, kTile), grid((N + kTile - 1) / kTile, (M + kTile - 1) / kTile);
  gemm_kernel<TA, TB><<<grid, block, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, act);
}

// dA = dH * (1 - H^2) (derivative of tanh through its output).
__global__ void tanh_back_kernel(const float* __restrict__ dH, const float* __restrict__ H,
                                 float* __restrict__ dA, long long len) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < len;
       k += (long long)gridDim.x * blockDim.x)
    dA[k] = dH[k] * (1.f - H[k] * H[k]);
}

// out[c] = sum_r Y[r, c] (fixed order).
__global__ void colsum_kernel(const float* __restrict__ Y, int rows, int cols,
                              float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += Y[(long long)r * cols + c];
  out[c] = s;
}

__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, long long len, float lr,
                            float b1, float b2, float eps, float bc1, float bc2) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < len;
       k += (long long)gridDim.x * blockDim.x) {
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    w[k] -= lr * (mk / bc1) / (sqrtf(vk / bc2) + eps);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst,
                               long long len) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < len;
       k += (long long)gridDim.x * blockDim.x)
    dst[k] = __float2bfloat16_rn(src[k]);
}

// Record pair `slot`: psi (FP32), m rows drawn uniformly with replacement from the
// counter-based stream (record number `count`, purpose kPurposeWsRows) and y at those rows.
__global__ void record_rows_kernel(const double* __restrict__ psi, int p, const float* __restrict__ y,
                                   long long n, int m, unsigned long long seed,
                                   unsigned long long count, float* __restrict__ pair_psi,
                                   int* __restrict__ pair_rows, float* __restrict__ pair_y,
                                   int slot) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < p) pair_psi[(long long)slot * p + k] = (float)psi[k];
  if (k < m) {
    uint64_t out[4];
    philox4x64_10((uint64_t)k, count, 0, kPurposeWsRows, seed, 0, out);
    long long r = (long long)(u01_53(out[0]) * (double)n);
    if (r >= n) r = n - 1;
    pair_rows[(long long)slot * m + k] = (int)r;
    pair_y[(long long)slot * m + k] = y[r];
  }
}

// cross[j * A + a] = k_s(x_j, z_a) at the current parameters (prescaled inputs).
__global__ void cross_kernel(const float* __restrict__ xhat, int DP, long long n,
                             const int* __restrict__ anch, int A, const DevParams* __restrict__ P,
                             float* __restrict__ cross) {
  extern __shared__ float sz[];   // A x DP anchors
  for (int k = threadIdx.x; k < A * DP; k += blockDim.x)
    sz[k] = xhat[(long long)anch[k / DP] * DP + k % DP];
  __syncthreads();
  const float c0 = P->c0f, c1 = P->c1f;
  const long long total = n * A;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long j = e / A;
    const int a = (int)(e - j * A);
    float s = 0.f;
    for (int q = 0; q < DP; ++q) {
      const float df = xhat[j * DP + q] - sz[a * DP + q];
      s = fmaf(df, df, s);
    }
    cross[e] = ex2_approx(fmaf(-c1, s, c0));
  }
}

// Split partial sums of the signal part of M: for the j range of split blockIdx.z,
//   Mpart[z][k][a] = sum_j k_s(x_{rows_k}, x_j) cross[j][a].
// A CTA owns a 64-row x 64-anchor tile; per 32-wide j chunk it generates the 64 x 32 kernel
// tile in shared memory, stages the 32 x 64 slice of `cross`, and each thread accumulates
// a 4 x 4 block of the tile.
constexpr int kMT = 64, kAT = 64, kJT = 32;
__global__ void __launch_bounds__(256) mrow_kernel(const float* __restrict__ xhat, int DP, long long n,
                                                   const int* __restrict__ rows, int m, int A,
                                                   const float* __restrict__ cross,
                                                   const DevParams* __restrict__ P,
                                                   long long jchunk, float* __restrict__ Mpart) {
  __shared__ float xr[kMT][kMaxD + 1];
  __shared__ float xj[kJT][kMaxD + 1];
  __shared__ __align__(16) float Kt[kJT][kMT + 4];
  __shared__ __align__(16) float Ct[kJT][kAT + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int a0 = blockIdx.x * kAT, r0 = blockIdx.y * kMT;
  const long long jb = (long long)blockIdx.z * jchunk;
  const long long je = min(n, jb + jchunk);
  const float c0 = P->c0f, c1 = P->c1f;
  for (int e = tid; e < kMT * DP; e += 256) {
    const int r = e / DP, q = e - r * DP;
    xr[r][q] = (r0 + r < m) ? xhat[(long long)rows[r0 + r] * DP + q] : 0.f;
  }
  float acc[4][4] = {};
  for (long long j0 = jb; j0 < je; j0 += kJT) {
    __syncthreads();   // previous chunk fully consumed (and xr written on the first pass)
    for (int e = tid; e < kJT * DP; e += 256) {
      const int jj = e / DP, q = e - jj * DP;
      xj[jj][q] = (j0 + jj < je) ? xhat[(j0 + jj) * DP + q] : 0.f;
    }
    for (int e = tid; e < kJT * kAT; e += 256) {
      const int jj = e / kAT, a = e - jj * kAT;
      Ct[jj][a] = (j0 + jj < je && a0 + a < A) ? cross[(j0 + jj) * A + a0 + a] : 0.f;
    }
    __syncthreads();
    for (int e = tid; e < kJT * kMT; e += 256) {
      const int jj = e / kMT, r = e - jj * kMT;
      float s = 0.f;
      for (int q = 0; q < DP; ++q) {
        const float df = xr[r][q] - xj[jj][q];
        s = fmaf(df, df, s);
      }
      Kt[jj][r] = (r0 + r < m && j0 + jj < je) ? ex2_approx(fmaf(-c1, s, c0)) : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int jj = 0; jj < kJT; ++jj) {
      const float4 kv = *reinterpret_cast<const float4*>(&Kt[jj][ty * 4]);
      const float4 cv = *reinterpret_cast<const float4*>(&Ct[jj][tx * 4]);
      const float kr[4] = {kv.x, kv.y, kv.z, kv.w}, cr[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[i][c] = fmaf(kr[i], cr[c], acc[i][c]);
    }
  }
  float* out = Mpart + (long long)blockIdx.z * m * A;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + ty * 4 + i;
    if (r >= m) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int a = a0 + tx * 4 + c;
      if (a < A) out[(long long)r * A + a] = acc[i][c];
    }
  }
}

// M[k][a] = sum over splits (fixed order) + lambda cross[rows_k][a] (the noise term of K).
__global__ void mreduce_kernel(const float* __restrict__ Mpart, int n_split, int m, int A,
                               const int* __restrict__ rows, const float* __restrict__ cross,
                               const DevParams* __restrict__ P, float* __restrict__ M) {
  const long long total = (long long)m * A;
  const float lam = P->lambdaf;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long k = e / A;
    const int a = (int)(e - k * A);
    float s = 0.f;
    for (int sp = 0; sp < n_split; ++sp) s += Mpart[sp * total + e];
    M[e] = fmaf(lam, cross[(long long)rows[k] * A + a], s);
  }
}

// Standardisation of the recorded inputs: mu, sd (sd floored) over the first T pairs.
__global__ void standardize_kernel(const float* __restrict__ pair_psi, int T, int p,
                                   float* __restrict__ mu, float* __restrict__ sd) {
  const int k = threadIdx.x;
  if (k >= p) return;
  double s = 0.0, s2 = 0.0;
  for (int t = 0; t < T; ++t) {
    const double v = pair_psi[(long long)t * p + k];
    s += v;
    s2 += v * v;
  }
  const double mean = s / T;
  const double var = fmax(s2 / T - mean * mean, 0.0);
  mu[k] = (float)mean;
  sd[k] = (float)fmax(sqrt(var), 1e-3);
}

// Z[b, k] = (pair_psi[idx[b], k] - mu[k]) / sd[k]
__global__ void gather_z_kernel(const float* __restrict__ pair_psi, const int* __restrict__ idx,
                                int B, int p, const float* __restrict__ mu,
                                const float* __restrict__ sd, float* __restrict__ Z) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= B * p) return;
  const int b = k / p, q = k - b * p;
  Z[k] = (pair_psi[(long long)idx[b] * p + q] - mu[q]) / sd[q];
}

__device__ inline float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Residual on the recorded rows: R[b][k] = y_I[k] - sum_a M[k][a] C[b][a] for pair idx[b],
// one warp per row.  Per-block sums of R^2 (block 0 of each pair adds rho m ||c_b||^2) to
// loss_part[b * gridDim.x + blockIdx.x]; the loss is their total / (B m).
__global__ void resid_kernel(const float* __restrict__ pair_M, const float* __restrict__ pair_y,
                             const int* __restrict__ idx, const float* __restrict__ C, int m,
                             int A, float ridge, float* __restrict__ R,
                             double* __restrict__ loss_part) {
  __shared__ double red[8];
  const int b = blockIdx.y, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long t = idx[b];
  const float* cb = C + (long long)b * A;
  const int k = blockIdx.x * 8 + w;
  double part = 0.0;
  if (k < m) {
    const float* Mk = pair_M + (t * m + k) * A;
    float acc = 0.f;
    for (int a = lane; a < A; a += 32) acc = fmaf(Mk[a], cb[a], acc);
    acc = warp_sum_f(acc);
    if (lane == 0) {
      const float r = pair_y[t * m + k] - acc;
      R[(long long)b * m + k] = r;
      part = (double)r * (double)r;
    }
  }
  if (blockIdx.x == 0) {
    double cc = 0.0;
    for (int a = threadIdx.x; a < A; a += blockDim.x) cc += (double)cb[a] * (double)cb[a];
    part += (double)ridge * (double)m * cc;
  }
  part = warp_sum(part);
  if (lane == 0) red[w] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < 8; ++i) s += red[i];
    loss_part[(long long)b * gridDim.x + blockIdx.x] = s;
  }
}

// dC[b][a] = sr sum_k M[k][a] R[b][k] + sc C[b][a]  (sr = -2 / (B m), sc = 2 rho / B).
__global__ void dc_kernel(const float* __restrict__ pair_M, const int* __restrict__ idx,
                          const float* __restrict__ R, const float* __restrict__ C, int m, int A,
                          float sr, float sc, float* __restrict__ dC) {
  extern __shared__ float sres[];   // m residuals of pair b
  const int b = blockIdx.y;
  const long long t = idx[b];
  for (int k = threadIdx.x; k < m; k += blockDim.x) sres[k] = R[(long long)b * m + k];
  __syncthreads();
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= A) return;
  const float* Mb = pair_M + t * m * A;
  float acc = 0.f;
  for (int k = 0; k < m; ++k) acc = fmaf(Mb[(long long)k * A + a], sres[k], acc);
  dC[(long long)b * A + a] = fmaf(sc, C[(long long)b * A + a], sr * acc);
}

// Pooled normal equations of the loss for a constant c over the first T pairs (rows
// stacked: Mall = pair_M viewed as (T m) x A):
//     G = Mall^T Mall / (T m) + rho I   (lower triangle, FP64),   gb = Mall^T y_all / (T m).
// A CTA owns a 32 x 32 block of G (blocks above the diagonal exit); per 32-row chunk each
// thread forms an FP32 partial of its entry and adds it into an FP64 accumulator.
constexpr int kGT = 32;
__global__ void __launch_bounds__(1024) gram_kernel(const float* __restrict__ Mall,
                                                    const float* __restrict__ yall,
                                                    long long rows, int A, float ridge,
                                                    double* __restrict__ G,
                                                    double* __restrict__ gb) {
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bj > bi) return;
  __shared__ float si[kGT][kGT + 1], sj[kGT][kGT + 1], sy[kGT];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int i = bi * kGT + ty, j = bj * kGT + tx;
  double acc = 0.0, accb = 0.0;
  for (long long r0 = 0; r0 < rows; r0 += kGT) {
    const long long r = r0 + ty;
    const bool ok = r < rows;
    si[ty][tx] = (ok && bi * kGT + tx < A) ? Mall[r * A + bi * kGT + tx] : 0.f;
    sj[ty][tx] = (ok && j < A) ? Mall[r * A + j] : 0.f;
    if (tx == 0) sy[ty] = ok ? yall[r] : 0.f;
    __syncthreads();
    float part = 0.f, partb = 0.f;
#pragma unroll 8
    for (int k = 0; k < kGT; ++k) {
      part = fmaf(si[k][ty], sj[k][tx], part);
      partb = fmaf(si[k][ty], sy[k], partb);
    }
    acc += part;
    accb += partb;
    __syncthreads();
  }
  if (i < A && j < A) G[(long long)i * A + j] = acc / (double)rows + (i == j ? (double)ridge : 0.0);
  if (bj == 0 && tx == 0 && i < A) gb[i] = accb / (double)rows;
}

// In-place Cholesky G = L L^T of the lower triangle (one CTA, FP64, right-looking).  A
// non-positive pivot sets *fail and leaves the factor unfinished.
__global__ void __launch_bounds__(1024) chol_kernel(double* __restrict__ G, int A,
                                                    int* __restrict__ fail) {
  __shared__ double piv;
  for (int k = 0; k < A; ++k) {
    if (threadIdx.x == 0) {
      const double dk = G[(long long)k * A + k];
      piv = dk > 0.0 ? sqrt(dk) : 0.0;
      if (dk > 0.0) G[(long long)k * A + k] = piv;
      else *fail = 1;
    }
    __syncthreads();
    if (piv == 0.0) return;
    for (int i = k + 1 + threadIdx.x; i < A; i += blockDim.x) G[(long long)i * A + k] /= piv;
    __syncthreads();
    const int w = A - k - 1;
    for (long long e = threadIdx.x; e < (long long)w * w; e += blockDim.x) {
      const int i = k + 1 + (int)(e / w), j = k + 1 + (int)(e % w);
      if (j <= i) G[(long long)i * A + j] -= G[(long long)i * A + k] * G[(long long)j * A + k];
    }
    __syncthreads();
  }
}

// P = L^{-1} (lower triangular; FP32 copy, zeros above the diagonal): thread j forward-
// substitutes column j of L X = I.
__global__ void trinv_kernel(const double* __restrict__ L, int A, double* __restrict__ X,
                             float* __restrict__ P) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= A) return;
  for (int i = 0; i < A; ++i) {
    double v = 0.0;
    if (i >= j) {
      double s = (i == j) ? 1.0 : 0.0;
      for (int k = j; k < i; ++k) s -= L[(long long)i * A + k] * X[(long long)k * A + j];
      v = s / L[(long long)i * A + i];
    }
    X[(long long)i * A + j] = v;
    P[(long long)i * A + j] = (float)v;
  }
}

__global__ void f64_to_f32_kernel(const double* __restrict__ src, float* __restrict__ dst, int len) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < len) dst[k] = (float)src[k];
}

// c = MLP(z(psi)) for one psi: one CTA; weights FP32 (w) or BF16 (wb), FP32 accumulation.
template <bool BF16>
__global__ void infer_kernel(const double* __restrict__ psi, int p, int H, int A,
                             const float* __restrict__ w, const __nv_bfloat16* __restrict__ wb,
                             const float* __restrict__ mu, const float* __restrict__ sd,
                             float* __restrict__ c) {
  extern __shared__ float buf[];   // z (p), h1 (H), h2 (H)
  float* z = buf;
  float* h1 = z + p;
  float* h2 = h1 + H;
  auto W = [&](long long k) -> float { return BF16 ? __bfloat162float(wb[k]) : w[k]; };
  const long long oW1 = 0, ob1 = oW1 + (long long)p * H, oW2 = ob1 + H, ob2 = oW2 + (long long)H * H,
                  oW3 = ob2 + H, ob3 = oW3 + (long long)H * A;
  for (int k = threadIdx.x; k < p; k += blockDim.x) z[k] = ((float)psi[k] - mu[k]) / sd[k];
  __syncthreads();
  for (int j = threadIdx.x; j < H; j += blockDim.x) {
    float s = W(ob1 + j);
    for (int k = 0; k < p; ++k) s = fmaf(z[k], W(oW1 + (long long)k * H + j), s);
    h1[j] = tanhf(s);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < H; j += blockDim.x) {
    float s = W(ob2 + j);
    for (int k = 0; k < H; ++k) s = fmaf(h1[k], W(oW2 + (long long)k * H + j), s);
    h2[j] = tanhf(s);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < A; j += blockDim.x) {
    float s = W(ob3 + j);
    for (int k = 0; k < H; ++k) s = fmaf(h2[k], W(oW3 + (long long)k * A + j), s);
    c[j] = s;
  }
}

// x0[i] = sum_a k_s(x^_i, x^_anch[a]) c[a] with the current prescaled inputs (ld x DP).
__global__ void x0_kernel(const float* __restrict__ xhat, int DP, long long n,
                          const int* __restrict__ anch, int A, const float* __restrict__ c,
                          const DevParams* __restrict__ P, float* __restrict__ x0) {
  extern __shared__ float sz[];   // A x DP anchors, then A coefficients
  for (int k = threadIdx.x; k < A * DP; k += blockDim.x)
    sz[k] = xhat[(long long)anch[k / DP] * DP + k % DP];
  float* sc = sz + A * DP;
  for (int a = threadIdx.x; a < A; a += blockDim.x) sc[a] = c[a];
  __syncthreads();
  const float c0 = P->c0f, c1 = P->c1f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    float xi[kMaxD];
    for (int q = 0; q < DP; ++q) xi[q] = xhat[i * DP + q];
    float acc = 0.f;
    for (int a = 0; a < A; ++a) {
      float s = 0.f;
      for (int q = 0; q < DP; ++q) {
        const float df = xi[q] - sz[a * DP + q];
        s = fmaf(df, df, s);
      }
      acc = fmaf(ex2_approx(fmaf(-c1, s, c0)), sc[a], acc);
    }
    x0[i] = acc;
  }
}

}  // namespace ws

// ------------------------------------------------------------------------------------------
// Host-side pieces called by the context (api.cu)
// ------------------------------------------------------------------------------------------
long long ws_param_count(int p, int H, int A) {
  return (long long)p * H + H + (long long)H * H + H + (long long)H * A + A;
}

int ws_loss_blocks(int m) { return (m + 7) / 8; }

void ws_record(const WsBuffers& b, const double* psi_dev, const float* y, const float* xhat,
               int DP, const DevParams* params, int slot, unsigned long long count,
               cudaStream_t s) {
  const int th = 256, nr = std::max(b.p, b.m);
  int* rows = b.pair_rows + (long long)slot * b.m;
  ws::record_rows_kernel<<<(nr + th - 1) / th, th, 0, s>>>(psi_dev, b.p, y, b.n, b.m, b.seed,
                                                          count, b.pair_psi, b.pair_rows,
                                                          b.pair_y, slot);
  const long long total = b.n * b.A;
  ws::cross_kernel<<<(int)std::min<long long>((total + th - 1) / th, 8192), th,
                     sizeof(float) * (size_t)b.A * DP, s>>>(xhat, DP, b.n, b.anch, b.A, params,
                                                            b.cross);
  const long long jchunk = ((b.n + b.n_split - 1) / b.n_split + ws::kJT - 1) / ws::kJT * ws::kJT;
  dim3 grid((b.A + ws::kAT - 1) / ws::kAT, (b.m + ws::kMT - 1) / ws::kMT, b.n_split);
  ws::mrow_kernel<<<grid, 256, 0, s>>>(xhat, DP, b.n, rows, b.m, b.A, b.cross, params, jchunk,
                                       b.Mpart);
  const long long mt = (long long)b.m * b.A;
  ws::mreduce_kernel<<<(int)std::min<long long>((mt + th - 1) / th, 4096), th, 0, s>>>(
      b.Mpart, b.n_split, b.m, b.A, rows, b.cross, params, b.pair_M + (long long)slot * mt);
}

void ws_standardize(const WsBuffers& b, int T, cudaStream_t s) {
  ws::standardize_kernel<<<1, 32, 0, s>>>(b.pair_psi, T, b.p, b.mu, b.sd);
}

// Loss and gradient over the B pairs listed in b.idx (already on the device).  Gradient into
// b.g; per-block partial sums into b.loss_part (their total / (B m) is the loss).
void ws_loss_grad(const WsBuffers& b, int B, int n_loss_blocks, cudaStream_t s) {
  const int p = b.p, H = b.H, A = b.A, m = b.m;
  float* W1 = b.w;
  float* b1 = W1 + (long long)p * H;
  float* W2 = b1 + H;
  float* b2 = W2 + (long long)H * H;
  float* W3 = b2 + H;
  float* b3 = W3 + (long long)H * A;
  float* gW1 = b.g;
  float* gb1 = gW1 + (long long)p * H;
  float* gW2 = gb1 + H;
  float* gb2 = gW2 + (long long)H * H;
  float* gW3 = gb2 + H;
  float* gb3 = gW3 + (long long)H * A;
  ws::gather_z_kernel<<<(B * p + 255) / 256, 256, 0, s>>>(b.pair_psi, b.idx, B, p, b.mu, b.sd, b.Z);
  ws::gemm<false, false>(s, B, H, p, b.Z, p, W1, H, b.H1, H, b1, 1);
  ws::gemm<false, false>(s, B, H, H, b.H1, H, W2, H, b.H2, H, b2, 1);
  ws::gemm<false, false>(s, B, A, H, b.H2, H, W3, A, b.C, A, b3, 0);
  {
    dim3 grid(n_loss_blocks, B);
    ws::resid_kernel<<<grid, 256, 0, s>>>(b.pair_M, b.pair_y, b.idx, b.C, m, A, b.ridge, b.R,
                                          b.loss_part);
  }
  {
    dim3 grid((A + 127) / 128, B);
    ws::dc_kernel<<<grid, 128, sizeof(float) * (size_t)m, s>>>(
        b.pair_M, b.idx, b.R, b.C, m, A, -2.f / ((float)B * (float)m), 2.f * b.ridge / (float)B,
        b.dC);
  }
  // backward through the three layers
  ws::gemm<true, false>(s, H, A, B, b.H2, H, b.dC, A, gW3, A, nullptr, 0);
  ws::colsum_kernel<<<(A + 255) / 256, 256, 0, s>>>(b.dC, B, A, gb3);
  ws::gemm<false, true>(s, B, H, A, b.dC, A, W3, A, b.dH, H, nullptr, 0);
  ws::tanh_back_kernel<<<(B * H + 255) / 256, 256, 0, s>>>(b.dH, b.H2, b.dA, (long long)B * H);
  ws::gemm<true, false>(s, H, H, B, b.H1, H, b.dA, H, gW2, H, nullptr, 0);
  ws::colsum_kernel<<<(H + 255) / 256, 256, 0, s>>>(b.dA, B, H, gb2);
  ws::gemm<false, true>(s, B, H, H, b.dA, H, W2, H, b.dH, H, nullptr, 0);
  ws::tanh_back_kernel<<<(B * H + 255) / 256, 256, 0, s>>>(b.dH, b.H1, b.dA, (long long)B * H);
  ws::gemm<true, false>(s, p, H, B, b.Z, p, b.dA, H, gW1, H, nullptr, 0);
  ws::colsum_kernel<<<(H + 255) / 256, 256, 0, s>>>(b.dA, B, H, gb1);
}

// Whitening of the output layer for the first T pairs: G = L L^T (pooled normal matrix
// plus the ridge), P = L^{-1}, and the whitened last layer set to W~3 = 0,
// b~3 = gb^T P^T (so that b3 = b~3 P = G^{-1} gb, the pooled least-squares constant).
// Returns false (nothing changed) if the Cholesky factorisation failed.
bool ws_whiten(const WsBuffers& b, int T, cudaStream_t s) {
  const int A = b.A;
  dim3 grid((A + ws::kGT - 1) / ws::kGT, (A + ws::kGT - 1) / ws::kGT);
  ws::gram_kernel<<<grid, 1024, 0, s>>>(b.pair_M, b.pair_y, (long long)T * b.m, A, b.ridge, b.G,
                                        b.gb);
  cudaMemsetAsync(b.flag, 0, sizeof(int), s);
  ws::chol_kernel<<<1, 1024, 0, s>>>(b.G, A, b.flag);
  int fail = 1;
  cudaMemcpyAsync(&fail, b.flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess || fail) return false;
  ws::trinv_kernel<<<(A + 127) / 128, 128, 0, s>>>(b.G, A, b.Ginv, b.P);
  ws::f64_to_f32_kernel<<<(A + 255) / 256, 256, 0, s>>>(b.gb, b.gbf, A);
  cudaMemsetAsync(b.wt, 0, sizeof(float) * (size_t)b.H * A, s);
  ws::gemm<false, true>(s, 1, A, A, b.gbf, A, b.P, A, b.wt + (long long)b.H * A, A, nullptr, 0);
  ws_unwhiten(b, s);
  return true;
}

// Effective last layer (W3; b3) = (W~3; b~3) P.
void ws_unwhiten(const WsBuffers& b, cudaStream_t s) {
  const long long oW3 = (long long)b.p * b.H + b.H + (long long)b.H * b.H + b.H;
  ws::gemm<false, false>(s, b.H + 1, b.A, b.A, b.wt, b.A, b.P, b.A, b.w + oW3, b.A, nullptr, 0);
}

// One Adam step with the output layer in whitened coordinates: the gradient of the last
// layer is mapped by P^T (chain rule of W3 = W~3 P), the hidden layers step as usual.
void ws_adam_whitened(const WsBuffers& b, float lr, int t, cudaStream_t s) {
  const long long oW3 = (long long)b.p * b.H + b.H + (long long)b.H * b.H + b.H;
  const long long nl = (long long)(b.H + 1) * b.A;
  ws::gemm<false, true>(s, b.H + 1, b.A, b.A, b.g + oW3, b.A, b.P, b.A, b.gt, b.A, nullptr, 0);
  const float b1 = 0.9f, b2 = 0.999f;
  const float bc1 = 1.f - powf(b1, (float)t), bc2 = 1.f - powf(b2, (float)t);
  ws::adam_kernel<<<(int)std::min<long long>((oW3 + 255) / 256, 1024), 256, 0, s>>>(
      b.w, b.g, b.adam_m, b.adam_v, oW3, lr, b1, b2, 1e-8f, bc1, bc2);
  ws::adam_kernel<<<(int)std::min<long long>((nl + 255) / 256, 1024), 256, 0, s>>>(
      b.wt, b.gt, b.adam_m + oW3, b.adam_v + oW3, nl, lr, b1, b2, 1e-8f, bc1, bc2);
  ws_unwhiten(b, s);
}

void ws_to_bf16(const WsBuffers& b, cudaStream_t s) {
  const long long len = ws_param_count(b.p, b.H, b.A);
  ws::to_bf16_kernel<<<(int)std::min<long long>((len + 255) / 256, 1024), 256, 0, s>>>(b.w, b.wb,
                                                                                       len);
}

// c = MLP(psi) (BF16 weights if bf16) then x0 = K_s(X, Z) c with the current prescale.
void ws_x0(const WsBuffers& b, const double* psi_dev, bool bf16, const float* xhat, int DP,
           long long n, const DevParams* params, float* c_out, float* x0, int num_sms,
           cudaStream_t s) {
  const size_t sh = sizeof(float) * (b.p + 2 * b.H);
  if (bf16)
    ws::infer_kernel<true><<<1, 256, sh, s>>>(psi_dev, b.p, b.H, b.A, b.w, b.wb, b.mu, b.sd, c_out);
  else
    ws::infer_kernel<false><<<1, 256, sh, s>>>(psi_dev, b.p, b.H, b.A, b.w, b.wb, b.mu, b.sd, c_out);
  const size_t sh2 = sizeof(float) * ((size_t)b.A * DP + b.A);
  const int blocks = (int)std::min<long long>((n + 255) / 256, 4LL * num_sms);
  ws::x0_kernel<<<blocks, 256, sh2, s>>>(xhat, DP, n, b.anch, b.A, c_out, params, x0);
}

}  // namespace ulisse
