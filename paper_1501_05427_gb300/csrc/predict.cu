// Posterior predictive for new inputs (Sec. 2, Eq. monte:carlo:integration): for parameters
// theta and test inputs x*_j,
//     p(y*_j | y, theta) = N(mu_j, v_j),  mu_j = k*_j^T K^{-1} y,
//     v_j = sigma^2 + lambda - k*_j^T K^{-1} k*_j,   k*_j = k_s(X, x*_j)
// (k_s the signal part of the covariance: a test input is not a training input, so the
// noise term lambda delta_ij does not enter k*_j; it enters v_j as the noise of y*).  The
// solves run in the library's solver; these kernels form the cross-covariance columns, the
// products k*_j^T s and the variance's dot products.  Averaging N(mu_j, v_j) over posterior
// samples theta^(i) is the Monte Carlo estimate of Eq. monte:carlo:integration.
#include <algorithm>

#include "predict.cuh"

namespace ulisse {

constexpr int kPredNT = 256;

// x^*_j = x*_j / l (row-major, DP columns, zero padded) for j < m.
template <typename T>
__global__ void predict_prescale_kernel(const float* __restrict__ Xs, long long m, int d, int DP,
                                        const DevParams* __restrict__ P, T* __restrict__ xs_hat) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < m * DP;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long j = idx / DP;
    const int k = (int)(idx - j * DP);
    xs_hat[idx] = k < d ? (T)((double)Xs[j * d + k] * P->inv_l[k]) : T(0);
  }
}

// Column c0 + j of B (leading dimension ld) = k*_j = k_s(X, x*_j) for rows i < n, zero on the
// padding rows [n, ld).  Grid: (row chunks, test points).
template <typename T>
__global__ void predict_cross_cols_kernel(const T* __restrict__ xhat, long long n, long long ld,
                                          int DP, const T* __restrict__ xs_hat, long long m,
                                          const DevParams* __restrict__ P, T* __restrict__ B,
                                          int c0) {
  const long long j = blockIdx.y;
  if (j >= m) return;
  const T* xs = xs_hat + j * DP;
  T* col = B + (long long)(c0 + j) * ld;
  const double s2 = P->sigma2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ld;
       i += (long long)gridDim.x * blockDim.x) {
    T v = T(0);
    if (i < n) {
      double d2 = 0.0;
      for (int k = 0; k < DP; ++k) {
        const double t = (double)xhat[i * DP + k] - (double)xs[k];
        d2 += t * t;
      }
      v = (T)(s2 * exp(-0.5 * d2));
    }
    col[i] = v;
  }
}

// mu_j = sum_i k_s(x*_j, x_i) s_i, one CTA per test point (FP64 accumulation, fixed order).
template <typename T>
__global__ void __launch_bounds__(kPredNT) predict_mean_kernel(
    const T* __restrict__ xhat, long long n, int DP, const T* __restrict__ xs_hat,
    const DevParams* __restrict__ P, const T* __restrict__ s, float* __restrict__ mean) {
  __shared__ double red[kPredNT / 32];
  const long long j = blockIdx.x;
  const T* xs = xs_hat + j * DP;
  double acc = 0.0;
  for (long long i = threadIdx.x; i < n; i += kPredNT) {
    double d2 = 0.0;
    for (int k = 0; k < DP; ++k) {
      const double t = (double)xhat[i * DP + k] - (double)xs[k];
      d2 += t * t;
    }
    acc += exp(-0.5 * d2) * (double)s[i];
  }
  acc = block_sum<kPredNT>(acc, red);
  if (threadIdx.x == 0) mean[j] = (float)(P->sigma2 * acc);
}

// v_j = sigma^2 + lambda - k*_j^T S_j, with k*_j column c0 + j of B and S_j column e0 + j of
// the estimates, one CTA per test point.
template <typename T>
__global__ void __launch_bounds__(kPredNT) predict_var_kernel(
    const T* __restrict__ B, const T* __restrict__ SE, long long n, long long ld, int c0, int e0,
    const DevParams* __restrict__ P, float* __restrict__ var) {
  __shared__ double red[kPredNT / 32];
  const long long j = blockIdx.x;
  const T* kc = B + (long long)(c0 + j) * ld;
  const T* sc = SE + (long long)(e0 + j) * ld;
  double acc = 0.0;
  for (long long i = threadIdx.x; i < n; i += kPredNT) acc += (double)kc[i] * (double)sc[i];
  acc = block_sum<kPredNT>(acc, red);
  if (threadIdx.x == 0) var[j] = (float)(P->sigma2 + P->lambda - acc);
}

template <typename T>
cudaError_t launch_predict_prescale(const float* Xs, long long m, int d, int DP,
                                    const DevParams* P, void* xs_hat, int num_sms, cudaStream_t s) {
  const int blocks = (int)std::min<long long>((m * DP + 255) / 256, 4LL * num_sms);
  predict_prescale_kernel<T><<<std::max(blocks, 1), 256, 0, s>>>(Xs, m, d, DP, P, (T*)xs_hat);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_predict_cross_cols(const void* xhat, long long n, long long ld, int DP,
                                      const void* xs_hat, long long m, const DevParams* P,
                                      void* B, int c0, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  const dim3 grid((unsigned)std::min<long long>((ld + kPredNT - 1) / kPredNT, 64), (unsigned)m);
  predict_cross_cols_kernel<T><<<grid, kPredNT, 0, s>>>((const T*)xhat, n, ld, DP,
                                                         (const T*)xs_hat, m, P, (T*)B, c0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_predict_mean(const void* xhat, long long n, int DP, const void* xs_hat,
                                long long m, const DevParams* P, const void* s, void* mean,
                                cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  predict_mean_kernel<T><<<(unsigned)m, kPredNT, 0, st>>>((const T*)xhat, n, DP,
                                                           (const T*)xs_hat, P, (const T*)s,
                                                           (float*)mean);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_predict_var(const void* B, const void* SE, long long n, long long ld, int c0,
                               int e0, long long m, const DevParams* P, void* var,
                               cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  predict_var_kernel<T><<<(unsigned)m, kPredNT, 0, st>>>((const T*)B, (const T*)SE, n, ld, c0,
                                                          e0, P, (float*)var);
  return cudaGetLastError();
}

#define ULISSE_PREDICT_INST(T)                                                                   \
  template cudaError_t launch_predict_prescale<T>(const float*, long long, int, int,             \
                                                  const DevParams*, void*, int, cudaStream_t);   \
  template cudaError_t launch_predict_cross_cols<T>(const void*, long long, long long, int,      \
                                                    const void*, long long, const DevParams*,   \
                                                    void*, int, cudaStream_t);                  \
  template cudaError_t launch_predict_mean<T>(const void*, long long, int, const void*,          \
                                              long long, const DevParams*, const void*, void*,   \
                                              cudaStream_t);                                     \
  template cudaError_t launch_predict_var<T>(const void*, const void*, long long, long long, int,\
                                             int, long long, const DevParams*, void*,            \
                                             cudaStream_t);
ULISSE_PREDICT_INST(float)
ULISSE_PREDICT_INST(double)
#undef ULISSE_PREDICT_INST

}  // namespace ulisse
