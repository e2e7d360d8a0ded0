// a1: parameter unpack and input prescale (shared by the context path and the
// allocation-free K V entry point).
#pragma once

#include "ulisse_internal.cuh"

namespace ulisse {

// ------------------------------------------------------------------------------------
// a1: parameters from psi, and x^ = x / l (rows >= n and dims >= d stay zero).
// ------------------------------------------------------------------------------------
template <typename T>
__global__ void prescale_kernel(const double* __restrict__ psi, const float* __restrict__ X,
                                T* __restrict__ xhat, long long n, int d, int DP,
                                DevParams* __restrict__ P) {
  double inv_l[kMaxD];
  for (int k = 0; k < d; ++k) inv_l[k] = exp(-psi[k]);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int k = 0; k < d + 2; ++k) P->psi[k] = psi[k];
    for (int k = 0; k < d; ++k) P->inv_l[k] = inv_l[k];
    const double s2 = exp(psi[d]), lam = exp(psi[d + 1]);
    P->sigma2 = s2;
    P->lambda = lam;
    P->c0f = (float)log2(s2);
    P->c1f = (float)(0.5 * 1.4426950408889634);  // log2(e) / 2
    P->lambdaf = (float)lam;
  }
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    for (int k = 0; k < DP; ++k)
      xhat[i * DP + k] = (k < d) ? (T)((double)X[i * d + k] * inv_l[k]) : T(0);
  }
}

}  // namespace ulisse
