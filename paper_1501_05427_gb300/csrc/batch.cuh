// Many independent GP problems of uneven size in one persistent launch (batched contexts).
//
// The O(n^2) passes of all problems -- the covariance products of a CG round and the fused
// gradient sweep -- run as one launch each.  The work list holds one item per (problem,
// 256-row block), ordered by decreasing row length (longest items first); a fixed grid of
// CTAs takes items from a global counter until the list is exhausted.  Each item runs the
// whole j range of its problem (no split: with thousands of items the counter balances the
// load), so no partial sums cross CTAs for K V; the gradient writes one slot of partial sums
// per item, summed in row-block order per problem by a second small launch.
#pragma once

#include "ulisse_internal.cuh"

namespace ulisse {

constexpr int kBatchNT = 128;
constexpr int kBatchTM = 2;
constexpr int kBatchBM = kBatchNT * kBatchTM;   // rows per item
constexpr int kBatchMaxDP = 8;                 // input widths d <= 8

struct BatchItem {
  int prob;   // problem index
  int rb;     // 256-row block within the problem
  int slot;   // gradient partial slot (problem-major, rb order)
  int pad;
};

// K V for one problem: U[:, umap[r]] = K V[:, vmap[r]] for r < *nlive.
struct BatchKmvDesc {
  const float* xhat;     // ldn x DP prescaled inputs (padding rows zero)
  long long n;
  int DP;
  int pad0;
  const DevParams* params;
  const float* V;        // column-major, leading dimension ldv (padding rows zero)
  long long ldv;
  const int* vmap;
  float* U;
  long long ldu;
  const int* umap;
  const int* nlive;      // live column count (device), 0 = skip the problem
};

// Fused gradient for one problem (Eq. gradient:unbiased), as the single-problem pass.
struct BatchGradDesc {
  const float* xhat;
  long long n;
  int DP, d;
  const DevParams* params;
  const float* A;        // left factors: columns amap[m], scaled by sa[m]
  const int* amap;
  const float* sa;
  const float* B;        // right factors: columns bmap[m]
  const int* bmap;
  long long ld;
  int M;
  int slot0;             // first partial slot of this problem
  int n_slots;           // its row blocks
  int pad0;
  double* g_out;         // d + 2 doubles
};

// R_max: the largest live count over the problems (selects the compiled column count).
cudaError_t launch_kmv_batch(const BatchKmvDesc* descs, const BatchItem* items, int n_items,
                             int* queue, int R_max, int num_sms, int* status, cudaStream_t s);
// Occupancy queries and attributes of every compiled width, made ahead of a graph capture.
void prime_kmv_batch();
void prime_grad_batch();
constexpr int kBatchWidths[5] = {2, 4, 9, 17, 32};   // compiled widths of the batched K V
constexpr long long kBatchCgChunk = 4096;          // rows per CTA of the batched CG kernels
cudaError_t launch_grad_batch(const BatchGradDesc* descs, int n_probs, const BatchItem* items,
                              int n_items, int* queue, double* partials, int M, int num_sms,
                              int* status, cudaStream_t s);

}  // namespace ulisse
