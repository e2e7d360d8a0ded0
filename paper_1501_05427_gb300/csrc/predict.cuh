// Launchers of the posterior-predictive kernels (predict.cu), T = the context's vector type.
#pragma once

#include "ulisse_internal.cuh"

namespace ulisse {
template <typename T>
cudaError_t launch_predict_prescale(const float* Xs, long long m, int d, int DP,
                                    const DevParams* P, void* xs_hat, int num_sms, cudaStream_t s);
template <typename T>
cudaError_t launch_predict_cross_cols(const void* xhat, long long n, long long ld, int DP,
                                      const void* xs_hat, long long m, const DevParams* P,
                                      void* B, int c0, cudaStream_t s);
template <typename T>
cudaError_t launch_predict_mean(const void* xhat, long long n, int DP, const void* xs_hat,
                                long long m, const DevParams* P, const void* s, void* mean,
                                cudaStream_t st);
template <typename T>
cudaError_t launch_predict_var(const void* B, const void* SE, long long n, long long ld, int c0,
                               int e0, long long m, const DevParams* P, void* var,
                               cudaStream_t st);

}  // namespace ulisse
