// Learned warm start: device buffers and host launchers (warm_start.cu).
#pragma once

#include <cuda_bf16.h>

#include "ulisse_internal.cuh"

namespace ulisse {

struct WsBuffers {
  int p, H, A, m, max_pairs;
  int d;
  long long n;
  float ridge;
  unsigned long long seed;
  int* anch;               // A anchor row indices
  float* w;                // parameters (flattened W1 b1 W2 b2 W3 b3)
  float* g;                // gradient
  float* adam_m;
  float* adam_v;
  __nv_bfloat16* wb;       // BF16 copy for inference
  float* pair_psi;         // max_pairs x p
  int* pair_rows;          // max_pairs x m sampled row indices
  float* pair_y;           // max_pairs x m: y at those rows
  float* pair_M;           // max_pairs x m x A: rows of K times the anchor columns
  float* cross;            // n x A scratch: K_s(X, Z) at the recorded parameters
  float* Mpart;            // n_split x m x A scratch: split partial sums of M
  int n_split;
  float* mu;               // p
  float* sd;               // p
  int* idx;                // batch indices (max_pairs)
  float *Z, *H1, *H2, *C, *R, *dC, *dH, *dA;   // work buffers, max_pairs rows
  double* loss_part;       // max_pairs x ceil(m / 8)
  // output-layer whitening (pooled normal matrix G = L L^T, P = L^{-1})
  double *G, *Ginv, *gb;   // A x A, A x A, A
  float *P, *gbf;          // A x A, A
  float *wt, *gt;          // whitened last layer (W~3; b~3) and its gradient, (H + 1) x A
  int* flag;
  float *w_best, *wt_best;  // weights with the lowest held-out loss during training
};

long long ws_param_count(int p, int H, int A);
// Record pair `slot` (the `count`-th recorded overall) at the current parameters.
void ws_record(const WsBuffers& b, const double* psi_dev, const float* y, const float* xhat,
               int DP, const DevParams* params, int slot, unsigned long long count,
               cudaStream_t s);
int ws_loss_blocks(int m);
void ws_standardize(const WsBuffers& b, int T, cudaStream_t s);
void ws_loss_grad(const WsBuffers& b, int B, int n_loss_blocks, cudaStream_t s);
bool ws_whiten(const WsBuffers& b, int T, cudaStream_t s);
void ws_unwhiten(const WsBuffers& b, cudaStream_t s);
void ws_adam_whitened(const WsBuffers& b, float lr, int t, cudaStream_t s);
void ws_to_bf16(const WsBuffers& b, cudaStream_t s);
void ws_x0(const WsBuffers& b, const double* psi_dev, bool bf16, const float* xhat, int DP,
           long long n, const DevParams* params, float* c_out, float* x0, int num_sms,
           cudaStream_t s);

}  // namespace ulisse
