// Vector kernels of the solver path: parameter unpack + prescale, Hutchinson probes,
// batched CG (Algorithm 1) with the ULISSE truncation and reweighting (Sec. 4), and the
// SGLD update (Sec. 2.1).  Vectors are T (float or double); every scalar recurrence --
// e^T e, d^T K d, alpha, beta, the early-stop test and the ULISSE weights -- is FP64.
#pragma once

#include "prescale.cuh"
#include "ulisse_internal.cuh"

namespace ulisse {

constexpr int kCgChunkNT = 256;   // threads of the chunked CG kernels

// ------------------------------------------------------------------------------------
// a2: probes r_j (column j = 1..nr of B): +-1 from the top bit, or N(0,1) by Box-Muller,
// element i of probe j from Philox counter (i, j, epoch, 1) keyed by (seed, 0).
// ------------------------------------------------------------------------------------
// Step of a chain run from a CUDA graph: the kernels of the graph read the step number,
// the step size and the trace slot from here (one graph serves every step of the chain);
// the SGLD update, the graph's last kernel, advances k.
struct ChainSlot {
  long long k;                  // index of the step within the chain call
  unsigned long long step0;     // step number of k = 0
  const double* eps;            // step sizes, one per k
  double* trace;                // NULL or p doubles per k
};

template <typename T>
__global__ void probes_kernel(T* __restrict__ B, long long ld, long long n, int nr, int kind,
                              unsigned long long seed, unsigned long long epoch,
                              const ChainSlot* __restrict__ cs = nullptr, int refresh = 1) {
  if (cs) epoch = (cs->step0 + (unsigned long long)cs->k) / (unsigned long long)refresh;
  const int j = blockIdx.y + 1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    uint64_t w[4];
    philox4x64_10((uint64_t)i, (uint64_t)j, epoch, kPurposeProbe, seed, 0, w);
    T v;
    if (kind == 0) v = (w[0] >> 63) ? T(-1) : T(1);
    else v = (T)box_muller(w[0], w[1]);
    B[(long long)j * ld + i] = v;
  }
}

template <typename T>
struct CgArgs {
  T* S;          // iterates s_m
  T* E;          // residuals e_m
  T* D;          // directions d_m
  const T* KD;   // K d_m (or K s_0 before the first iteration)
  const T* B;    // right-hand sides
  T* SE;         // ULISSE estimates
  long long n, ld;
  ColState* st;
  ColState* st_next;     // state written by an iteration, committed by compact_kernel
  const int* live;
  double* part1;         // per (column, chunk) partial d^T K d
  double* part2;         // per (column, chunk) partial e^T e
  int nchunk;            // CTAs per column
  long long chunk;       // rows per CTA
  double alpha_thr, eps, beta;
  int max_iter;
  int has_s0;
  unsigned long long seed, step;
  const ChainSlot* cs;   // when set, the step number comes from the chain slot
  const int* n_live;     // batched launches: this problem's live column count
  // Warm-started solves (Sec. 5.1's probe reuse): when warm_refresh > 0, S holds the final
  // CG iterates of the previous step's solve of every column (valid while *warm_valid is
  // nonzero).  Column 0 (y, never changes) starts from its iterate -- or from the learned
  // warm start when y_learned -- and probe columns start from theirs while the probes are
  // unchanged (step % warm_refresh != 0).  The keep-if-better rule still applies.
  int warm_refresh;
  const int* warm_valid;
  int y_learned;
  T* Sbest;              // warm-started solves: per column, the iterate of smallest residual
                         // seen (the start of the next step's solve)
  int* status;
};

// Accepted steps after the early stop: j = 1, 2, ... while u_j < 1/w_j = exp(-beta j).
__device__ inline int draw_J(unsigned long long seed, unsigned long long step, int colid,
                             int est, double beta, int jcap) {
  int J = 0;
  for (int j = 1; j <= jcap; ++j) {
    uint64_t w[4];
    philox4x64_10((uint64_t)j, (uint64_t)colid, step, kPurposeUlisse | ((uint64_t)est << 8),
                  seed, 0, w);
    if (u01_53(w[0]) < exp(-beta * (double)j)) J = j;
    else break;
  }
  return J;
}

// prod_{r=0}^{j} w_r, w_r = exp(beta r).
__device__ inline double weight_product(int j, double beta) {
  double W = 1.0;
  for (int r = 0; r <= j; ++r) W *= exp(beta * (double)r);
  return W;
}

template <typename T>
__device__ inline void chunk_range(const CgArgs<T>& a, int ch, long long* i0, long long* i1) {
  *i0 = (long long)ch * a.chunk;
  *i1 = min(a.n, *i0 + a.chunk);
}

// Whether column c starts from its initial iterate (else from s_0 = 0): every column with
// has_s0; with warm-started solves, column 0 (y) when its start is valid or learned, and the
// probe columns while the probes are unchanged.
template <typename T>
__device__ inline bool init_use_s0(const CgArgs<T>& a, int c) {
  if (a.warm_refresh <= 0) return a.has_s0 != 0;
  const unsigned long long step = a.cs ? a.cs->step0 + (unsigned long long)a.cs->k : a.step;
  const bool valid = *a.warm_valid != 0;
  return (c == 0) ? (a.y_learned || valid)
                  : (valid && step % (unsigned long long)a.warm_refresh != 0);
}

// b^T b and, when use_s0, (b - K s_0)^T (b - K s_0) over rows [i0, i1) of column c (FP64),
// summed over the block; rr = bb otherwise.
template <typename T>
__device__ inline void init_sums(const CgArgs<T>& a, int c, bool use_s0, long long i0,
                                 long long i1, double* red, double* bb, double* rr) {
  const T* b = a.B + c * a.ld;
  const T* ks0 = a.KD + c * a.ld;
  double pb = 0.0, pr = 0.0;
  for (long long i = i0 + threadIdx.x; i < i1; i += kCgChunkNT) {
    const double bi = (double)b[i];
    pb += bi * bi;
    if (use_s0) {
      const double ri = (double)(T)(b[i] - ks0[i]);
      pr += ri * ri;
    }
  }
  *bb = block_sum<kCgChunkNT>(pb, red);
  *rr = use_s0 ? block_sum<kCgChunkNT>(pr, red) : *bb;
}

// The CG start's sums per (chunk, column) when a column spans several chunks (part2: b^T b,
// part1: the residual's); cg_init_kernel adds them in chunk order.
template <typename T>
__global__ void __launch_bounds__(kCgChunkNT) cg_init_dot_kernel(const CgArgs<T> a) {
  __shared__ double red[kCgChunkNT / 32];
  const int c = blockIdx.y, ch = blockIdx.x;
  long long i0, i1;
  chunk_range(a, ch, &i0, &i1);
  double bb, rr;
  init_sums(a, c, init_use_s0(a, c), i0, i1, red, &bb, &rr);
  if (threadIdx.x == 0) {
    a.part2[(long long)c * a.nchunk + ch] = bb;
    a.part1[(long long)c * a.nchunk + ch] = rr;
  }
}

// e_0 = b - K s_0, d_0 = e_0, draws of J; grid (chunk, column).  With one chunk per column
// the CTA forms the sums itself; with several, every CTA of the column adds the partial sums
// of cg_init_dot_kernel in chunk order, so all of them take the same decision.
template <typename T>
__global__ void __launch_bounds__(kCgChunkNT) cg_init_kernel(const CgArgs<T> a) {
  __shared__ double red[kCgChunkNT / 32];
  const int c = blockIdx.y, ch = blockIdx.x;
  ColState& st = a.st[c];
  T* s = a.S + c * a.ld;
  T* e = a.E + c * a.ld;
  T* d = a.D + c * a.ld;
  const T* b = a.B + c * a.ld;
  const T* ks0 = a.KD + c * a.ld;
  const bool warm = a.warm_refresh > 0;
  T* sb = warm ? a.Sbest + c * a.ld : nullptr;
  // with warm-started solves the start comes from Sbest (y_learned: column 0 from S)
  const T* s0 = (warm && !(c == 0 && a.y_learned)) ? sb : s;
  const bool use_s0 = init_use_s0(a, c);
  long long i0, i1;
  chunk_range(a, ch, &i0, &i1);
  // An initial iterate is kept only when it lowers the residual norm below that of s_0 = 0.
  // The choice depends on the parameters, the data and the iterate alone (no random draw),
  // so every estimator built on it stays unbiased.
  double bb, rr;
  if (a.nchunk == 1) {
    init_sums(a, c, use_s0, i0, i1, red, &bb, &rr);
  } else {
    bb = 0.0;
    rr = 0.0;
    for (int k = 0; k < a.nchunk; ++k) {
      bb += a.part2[(long long)c * a.nchunk + k];
      rr += a.part1[(long long)c * a.nchunk + k];
    }
    if (!use_s0) rr = bb;
  }
  const bool keep = use_s0 && rr < bb;
  for (long long i = i0 + threadIdx.x; i < i1; i += kCgChunkNT) {
    const T si = keep ? s0[i] : T(0);
    s[i] = si;
    if (warm) sb[i] = si;
    const T ei = keep ? b[i] - ks0[i] : b[i];
    e[i] = ei;
    d[i] = ei;
  }
  const double ee = keep ? rr : bb;
  const int n_est = st.n_est;
  const bool done = sqrt(ee) < a.eps;
  if (done) {
    for (int t = 0; t < n_est; ++t) {
      T* se = a.SE + (long long)(st.est_off + t) * a.ld;
      for (long long i = i0 + threadIdx.x; i < i1; i += kCgChunkNT) se[i] = s[i];
    }
  }
  if (ch == 0 && threadIdx.x == 0) {
    st.ee = ee;
    st.best_ee = ee;
    st.l = 0;
    st.m = 0;
    st.outcome = 0;
    const unsigned long long step = a.cs ? a.cs->step0 + (unsigned long long)a.cs->k : a.step;
    st.J[0] = draw_J(a.seed, step, st.colid, 0, a.beta, a.max_iter);
    st.J[1] = n_est > 1 ? draw_J(a.seed, step, st.colid, 1, a.beta, a.max_iter) : -1;
    st.phase = done ? kDone : kPre;
  }
}

// One CG iteration (Algorithm 1) on every live column, with the ULISSE bookkeeping, in
// three launches over a (chunk, live column) grid so that every column is spread over
// several CTAs:
//   cg_dot_kernel     partial d^T K d per chunk
//   cg_update_kernel  alpha = e^T e / d^T K d (partials summed in chunk order), s += alpha d,
//                     e -= alpha K d, the ULISSE tail term, partial e'^T e' per chunk
//   cg_finish_kernel  e'^T e' (chunk order), the early-stop / convergence / max_iter
//                     decisions (every CTA of a column reaches the same ones), the copy of
//                     s_l into the estimators at the early stop, d = e' + beta d, and the
//                     new column state (into st_next; compact_kernel commits it).
// The increment delta_{m+1} = alpha_m d_m is added with weight prod_{r<=j} w_r to every
// estimator whose J >= j (j = m+1-l) once the early stop at l has been reached.

// The bodies below take the chunk (ch) and the live-list index (li) of the CTA: the
// single-problem kernels pass their grid coordinates, the batched ones add the problem.
template <typename T>
__device__ inline void cg_dot_body(const CgArgs<T>& a, int ch, int li) {
  __shared__ double red[kCgChunkNT / 32];
  const int c = a.live[li];
  const T* d = a.D + c * a.ld;
  const T* kd = a.KD + c * a.ld;
  long long i0, i1;
  chunk_range(a, ch, &i0, &i1);
  double p = 0.0;
  for (long long i = i0 + threadIdx.x; i < i1; i += kCgChunkNT) p += (double)d[i] * (double)kd[i];
  p = block_sum<kCgChunkNT>(p, red);
  if (threadIdx.x == 0) a.part1[(long long)c * a.nchunk + ch] = p;
}

template <typename T>
__device__ inline void cg_update_body(const CgArgs<T>& a, int ch, int li) {
  __shared__ double red[kCgChunkNT / 32];
  const int c = a.live[li];
  const ColState& st = a.st[c];
  double dKd = 0.0;
  for (int k = 0; k < a.nchunk; ++k) dKd += a.part1[(long long)c * a.nchunk + k];
  if (!(dKd > 0.0) || !isfinite(dKd)) return;  // breakdown: handled in cg_finish_kernel
  T* s = a.S + c * a.ld;
  T* e = a.E + c * a.ld;
  const T* d = a.D + c * a.ld;
  const T* kd = a.KD + c * a.ld;
  const double al = st.ee / dKd;
  const T alT = (T)al;
  T w0 = T(0), w1 = T(0);
  if (st.phase == kTail) {
    const int j = st.m + 1 - st.l;
    const double Wa = weight_product(j, a.beta) * al;
    if (st.J[0] >= j) w0 = (T)Wa;
    if (st.n_est > 1 && st.J[1] >= j) w1 = (T)Wa;
  }
  T* se0 = a.SE + (long long)st.est_off * a.ld;
  T* se1 = se0 + a.ld;
  long long i0, i1;
  chunk_range(a, ch, &i0, &i1);
  double p2 = 0.0;
  for (long long i = i0 + threadIdx.x; i < i1; i += kCgChunkNT) {
    const T di = d[i];
    s[i] = fma(alT, di, s[i]);
    const T ei = fma(-alT, kd[i], e[i]);
    e[i] = ei;
    p2 += (double)ei * (double)ei;
    if (w0 != T(0)) se0[i] = fma(w0, di, se0[i]);
    if (w1 != T(0)) se1[i] = fma(w1, di, se1[i]);
  }
  p2 = block_sum<kCgChunkNT>(p2, red);
  if (threadIdx.x == 0) a.part2[(long long)c * a.nchunk + ch] = p2;
}

template <typename T>
__device__ inline void cg_finish_body(const CgArgs<T>& a, int ch, int li) {
  const int c = a.live[li];
  const ColState& st = a.st[c];
  const int phase = st.phase, l = st.l, m = st.m, n_est = st.n_est;
  const int J0 = st.J[0], J1 = st.J[1];
  T* s = a.S + c * a.ld;
  T* e = a.E + c * a.ld;
  T* d = a.D + c * a.ld;
  T* se0 = a.SE + (long long)st.est_off * a.ld;
  long long i0, i1;
  chunk_range(a, ch, &i0, &i1);
  double dKd = 0.0, ee1 = 0.0;
  for (int k = 0; k < a.nchunk; ++k) {
    dKd += a.part1[(long long)c * a.nchunk + k];
    ee1 += a.part2[(long long)c * a.nchunk + k];
  }
  ColState nx = st;
  if (!(dKd > 0.0) || !isfinite(dKd)) {
    // Breakdown: K is not positive definite along d, or a value is not finite.
    if (phase == kPre)
      for (int t = 0; t < n_est; ++t)
        for (long long i = i0 + threadIdx.x; i < i1; i += kCgChunkNT) se0[t * a.ld + i] = s[i];
    if (ch == 0 && threadIdx.x == 0) {
      nx.outcome = 3;
      nx.phase = kDone;
      a.st_next[c] = nx;
      atomicOr(a.status, kStatusBreakdown);
    }
    return;
  }
  const int m1 = m + 1;
  int ph = phase, l1 = l, outcome = st.outcome;
  bool copy_s = false, done = false;
  const int jmax = (n_est > 1 && J1 > J0) ? J1 : J0;
  if (ph == kPre && sqrt(ee1) < a.alpha_thr) {
    l1 = m1;
    ph = kTail;
    copy_s = true;
  }
  const bool conv = sqrt(ee1) < a.eps;
  if (ph == kPre && conv) {
    copy_s = true;
    done = true;
  } else if (ph == kTail && (m1 - l1 >= jmax || conv)) {
    done = true;
  } else if (m1 >= a.max_iter) {
    if (ph == kPre) copy_s = true;
    outcome = 4;
    done = true;
  }
  if (copy_s)
    for (int t = 0; t < n_est; ++t)
      for (long long i = i0 + threadIdx.x; i < i1; i += kCgChunkNT) se0[t * a.ld + i] = s[i];
  // warm-started solves: remember the iterate of smallest residual (same decision in every
  // CTA of the column)
  const bool better = a.warm_refresh > 0 && ee1 < st.best_ee;
  if (better) {
    T* sb = a.Sbest + c * a.ld;
    for (long long i = i0 + threadIdx.x; i < i1; i += kCgChunkNT) sb[i] = s[i];
  }
  if (!done) {
    const T btT = (T)(ee1 / st.ee);
    for (long long i = i0 + threadIdx.x; i < i1; i += kCgChunkNT) d[i] = fma(btT, d[i], e[i]);
  }
  if (ch == 0 && threadIdx.x == 0) {
    nx.ee = ee1;
    if (better) nx.best_ee = ee1;
    nx.m = m1;
    nx.l = l1;
    nx.outcome = outcome;
    nx.phase = done ? kDone : ph;
    a.st_next[c] = nx;
    if (outcome == 4) atomicOr(a.status, kStatusMaxIter);
  }
}

template <typename T>
__global__ void __launch_bounds__(kCgChunkNT) cg_dot_kernel(const CgArgs<T> a) {
  cg_dot_body(a, blockIdx.x, blockIdx.y);
}
template <typename T>
__global__ void __launch_bounds__(kCgChunkNT) cg_update_kernel(const CgArgs<T> a) {
  cg_update_body(a, blockIdx.x, blockIdx.y);
}
template <typename T>
__global__ void __launch_bounds__(kCgChunkNT) cg_finish_kernel(const CgArgs<T> a) {
  cg_finish_body(a, blockIdx.x, blockIdx.y);
}

// Batched forms: grid (chunk, live-list index, problem) over all problems of a batch; a
// CTA past its problem's chunk count or live count returns at once.
template <typename T>
__global__ void __launch_bounds__(kCgChunkNT) cg_dot_batch_kernel(const CgArgs<T>* __restrict__ args) {
  const CgArgs<T>& a = args[blockIdx.z];
  if ((int)blockIdx.y >= *a.n_live || (int)blockIdx.x >= a.nchunk) return;
  cg_dot_body(a, blockIdx.x, blockIdx.y);
}
template <typename T>
__global__ void __launch_bounds__(kCgChunkNT) cg_update_batch_kernel(const CgArgs<T>* __restrict__ args) {
  const CgArgs<T>& a = args[blockIdx.z];
  if ((int)blockIdx.y >= *a.n_live || (int)blockIdx.x >= a.nchunk) return;
  cg_update_body(a, blockIdx.x, blockIdx.y);
}
template <typename T>
__global__ void __launch_bounds__(kCgChunkNT) cg_finish_batch_kernel(const CgArgs<T>* __restrict__ args) {
  const CgArgs<T>& a = args[blockIdx.z];
  if ((int)blockIdx.y >= *a.n_live || (int)blockIdx.x >= a.nchunk) return;
  cg_finish_body(a, blockIdx.x, blockIdx.y);
}

// Commit the state of the columns that just iterated (the first n_prev entries of the
// live list), then rebuild the live list in column order; count to *n_live.
__global__ void compact_kernel(ColState* __restrict__ st, const ColState* __restrict__ st_next,
                               int R, int n_prev, int* __restrict__ live,
                               int* __restrict__ n_live) {
  if (threadIdx.x != 0) return;
  for (int k = 0; k < n_prev; ++k) st[live[k]] = st_next[live[k]];
  int k = 0;
  for (int c = 0; c < R; ++c)
    if (st[c].phase != kDone) live[k++] = c;
  *n_live = k;
}

// Column bookkeeping of one problem of a batch (compact_batch_kernel).
struct BatchCgProb {
  ColState* st;
  const ColState* st_next;
  int* live;
  int* n_live;
  int R;
  long long n;
};

// K V width bucket of the batched product for a largest live count r: 0..4 for r <= 2, 4,
// 9, 17, 32 (the compiled widths of the batched kernel).
__host__ __device__ inline int batch_width_bucket(int r) {
  return r <= 2 ? 0 : r <= 4 ? 1 : r <= 9 ? 2 : r <= 17 ? 3 : 4;
}

// compact_kernel for every problem of a batch in one launch (one thread per problem; the
// live lists and counts are those of the previous round, the counts 0 before the first):
// commit, rebuild, and the largest live count to *rmax.  Inside a step graph it also sets
// the loop condition (another round while any column is live) and the branch (the width
// bucket of rmax; none when 0).  A round cap stops a loop that would not end.
// stat (may be null): [rounds, sum of n_b^2 x live columns, launches, rounds this call].
__global__ void __launch_bounds__(256) compact_batch_kernel(
    const BatchCgProb* __restrict__ probs, int B, int* __restrict__ rmax, int in_graph,
    cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_branch, int max_rounds,
    long long* __restrict__ stat, int* __restrict__ status) {
  __shared__ int s_max[256];
  __shared__ long long s_ent[256];
  int mx = 0;
  long long ent = 0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const BatchCgProb P = probs[b];
    const int n_prev = *P.n_live;
    for (int k = 0; k < n_prev; ++k) P.st[P.live[k]] = P.st_next[P.live[k]];
    int k = 0;
    for (int c = 0; c < P.R; ++c)
      if (P.st[c].phase != kDone) P.live[k++] = c;
    *P.n_live = k;
    mx = max(mx, k);
    ent += P.n * P.n * (long long)k;
  }
  s_max[threadIdx.x] = mx;
  s_ent[threadIdx.x] = ent;
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int t = 1; t < (int)blockDim.x; ++t) {
    mx = max(mx, s_max[t]);
    ent += s_ent[t];
  }
  if (stat) {
    const long long it = stat[3]++;
    if (mx > 0 && it >= max_rounds) {
      atomicOr(status, kStatusMaxIter);
      for (int b = 0; b < B; ++b) *probs[b].n_live = 0;
      mx = 0;
      ent = 0;
    }
    stat[2] += 1;
    if (mx > 0) {
      stat[0] += 1;
      stat[1] += ent;
      stat[2] += 4;   // the batched K V and the three batched CG launches
    }
  }
  *rmax = mx;
  if (in_graph) {
    cudaGraphSetConditional(h_loop, mx > 0 ? 1u : 0u);
    cudaGraphSetConditional(h_branch, mx > 0 ? (unsigned)batch_width_bucket(mx) : 5u);
  }
}

// ------------------------------------------------------------------------------------
// a7: SGLD proposal psi' = psi + eps/2 M (g + grad log p) + sqrt(eps) L xi, L L^T = M,
// xi_k standard normal from Philox counter (k, 0, step, 3).  One warp: lane i owns row i of
// L and component i (p <= kMaxP <= 32); each element's sums run in the serial order.
// ------------------------------------------------------------------------------------
__device__ inline void sgld_body(double* __restrict__ psi, const double* __restrict__ g,
                                 const double* __restrict__ M, const double* __restrict__ prior,
                                 double eps, int p, unsigned long long seed,
                                 unsigned long long step, double* __restrict__ trace,
                                 int* __restrict__ status) {
  __shared__ double L[kMaxP * kMaxP];
  __shared__ double xi[kMaxP], v[kMaxP];
  const int lane = threadIdx.x & 31;
  auto Mij = [&](int i, int j) -> double {
    return M ? M[i * p + j] : (i == j ? 1.0 : 0.0);
  };
  if (lane < p) {
    uint64_t w[4];
    philox4x64_10((uint64_t)lane, 0, step, kPurposeSgld, seed, 0, w);
    xi[lane] = box_muller(w[0], w[1]);
    v[lane] = g[lane] + (prior ? prior[lane] : 0.0);
    for (int j = 0; j < p; ++j) L[lane * p + j] = 0.0;
  }
  __syncwarp();
  // Cholesky M = L L^T, column by column: the diagonal on lane 0, then the column below it
  for (int j = 0; j < p; ++j) {
    int bad = 0;
    if (lane == 0) {
      double sj = Mij(j, j);
      for (int k = 0; k < j; ++k) sj -= L[j * p + k] * L[j * p + k];
      bad = !(sj > 0.0);
      if (!bad) L[j * p + j] = sqrt(sj);
    }
    if (__shfl_sync(0xffffffffu, bad, 0)) {
      if (lane == 0) atomicOr(status, kStatusBadM);
      return;
    }
    __syncwarp();
    if (lane > j && lane < p) {
      double t = Mij(lane, j);
      for (int k = 0; k < j; ++k) t -= L[lane * p + k] * L[j * p + k];
      L[lane * p + j] = t / L[j * p + j];
    }
    __syncwarp();
  }
  if (lane < p) {
    double drift = 0.0, noise = 0.0;
    for (int j = 0; j < p; ++j) drift += Mij(lane, j) * v[j];
    for (int j = 0; j <= lane; ++j) noise += L[lane * p + j] * xi[j];
    const double out = psi[lane] + 0.5 * eps * drift + sqrt(eps) * noise;
    psi[lane] = out;
    if (trace) trace[lane] = out;
  }
}

// Launched with one warp.
__global__ void sgld_kernel(double* __restrict__ psi, const double* __restrict__ g,
                            const double* __restrict__ M, const double* __restrict__ prior,
                            const double* __restrict__ eps_arr, double eps_scalar, int p,
                            unsigned long long seed, unsigned long long step,
                            double* __restrict__ trace, int* __restrict__ status) {
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  sgld_body(psi, g, M, prior, eps_arr ? *eps_arr : eps_scalar, p, seed, step, trace, status);
}

// The same update inside a chain graph: step, step size and trace slot from the chain
// slot, which then moves on to the next step.  Launched with one warp.
__global__ void sgld_chain_kernel(double* __restrict__ psi, const double* __restrict__ g,
                                  const double* __restrict__ M, const double* __restrict__ prior,
                                  int p, unsigned long long seed, ChainSlot* __restrict__ cs,
                                  int* __restrict__ status, int advance = 1,
                                  int trace_stride = 0, int trace_off = 0) {
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  const long long k = cs->k;
  const long long stride = trace_stride > 0 ? trace_stride : p;
  sgld_body(psi, g, M, prior, cs->eps[k], p, seed, cs->step0 + (unsigned long long)k,
            cs->trace ? cs->trace + k * stride + trace_off : nullptr, status);
  __syncwarp();   // every lane has read the slot
  if (advance && threadIdx.x == 0) cs->k = k + 1;
}

// The chain slot moves on to the next step (batched step graphs: after every problem's
// update).
__global__ void chain_advance_kernel(ChainSlot* __restrict__ cs) {
  if (threadIdx.x == 0 && blockIdx.x == 0) cs->k += 1;
}

// Graph form of compact_kernel: commits the previous iteration's column states (the live
// list and count are still those of the previous iteration; the count is 0 before the
// first), rebuilds the list, and sets the graph's loop conditions -- the WHILE body runs
// again while columns are live, and the SWITCH picks the branch compiled for that many
// live columns (none when 0).  A round cap (max_iter + 2) stops a loop that would not end.
// stat: [rounds, sum of live columns over rounds, kernel launches, iterations this call].
__global__ void compact_graph_kernel(ColState* __restrict__ st, const ColState* __restrict__ st_next,
                                     int R, int* __restrict__ live, int* __restrict__ n_live,
                                     cudaGraphConditionalHandle h_loop,
                                     cudaGraphConditionalHandle h_branch, int chunk_cols,
                                     int launches_per_chunk, int launches_fixed, int max_rounds,
                                     long long* __restrict__ stat, int* __restrict__ status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int n_prev = *n_live;
  for (int k = 0; k < n_prev; ++k) st[live[k]] = st_next[live[k]];
  int k = 0;
  for (int c = 0; c < R; ++c)
    if (st[c].phase != kDone) live[k++] = c;
  const long long it = stat[3]++;
  if (k > 0 && it >= max_rounds) {
    atomicOr(status, kStatusMaxIter);
    k = 0;
  }
  *n_live = k;
  stat[2] += 1;
  if (k > 0) {
    stat[0] += 1;
    stat[1] += k;
    stat[2] += launches_fixed + (long long)launches_per_chunk * ((k + chunk_cols - 1) / chunk_cols);
  }
  cudaGraphSetConditional(h_loop, k > 0 ? 1u : 0u);
  cudaGraphSetConditional(h_branch, k > 0 ? (unsigned)(k - 1) : (unsigned)R);
}

// Element-type conversion between caller buffers and the context's (FP64 contexts).
template <typename S, typename D>
__global__ void convert_cols_kernel(const S* __restrict__ src, long long lds, D* __restrict__ dst,
                                    long long ldd, long long n) {
  const int c = blockIdx.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[c * ldd + i] = (D)src[c * lds + i];
}

}  // namespace ulisse
