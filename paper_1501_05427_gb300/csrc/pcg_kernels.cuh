// Preconditioned CG with J = K + delta I (Sec. 3, "Preconditioned CG") and the ULISSE
// truncation and reweighting on its outer iteration (Sec. 4), for the columns of a block.
//
// Outer iteration (per column; e_0 = b, s_0 = 0):
//     z_i = J^{-1} e_i                     (inner CG, below)
//     d_0 = z_0;  d_i = z_i + beta_{i-1} d_{i-1},  beta_{i-1} = e_i^T (z_i - z_{i-1}) / e_{i-1}^T z_{i-1}
//     alpha_i = e_i^T z_i / d_i^T K d_i
//     s_{i+1} = s_i + alpha_i d_i,   e_{i+1} = e_i - alpha_i K d_i
// beta is the flexible (Polak-Ribiere) form: the inexact inner solve changes the
// preconditioner from one iteration to the next; with exact inner solves it equals the usual
// e_i^T z_i / e_{i-1}^T z_{i-1}.  The increments alpha_i d_i are those ULISSE truncates: the
// early stop compares ||e_{i+1}|| with q sqrt(n), and step j after it is kept with its weight
// prod_{r<=j} w_r, exactly as for plain CG (same counter-based draws, same column state).
//
// Inner CG on J z = e (per column): x_0 = 0, r_0 = p_0 = e; x += a p, r -= a (K p + delta p),
// a = r^T r / p^T (K p + delta p); it stops at the first iteration with ||r|| <= tau ||e||, or
// after inner_max iterations.  K p is one K V product of the library (any precision).
//
// One CTA per listed column; every dot product is an FP64 block sum in a fixed order.
#pragma once

#include "solver_kernels.cuh"

namespace ulisse {

constexpr int kPcgNT = 512;

// Inner-solve state of a column.
struct PcgAux {
  double ez;      // e_i^T z_i of the current outer direction
  double rr;      // inner r^T r
  double thr;     // tau^2 e^T e (the inner stopping threshold on r^T r)
  int inner_it;   // inner iterations of the current preconditioner solve
  int inner_done;
};

template <typename T>
struct PcgArgs {
  T *S, *E, *D, *Z;        // outer iterate, residual, direction, preconditioned residual
  const T* KD;             // K d
  T *X, *Rr, *P;           // inner iterate, residual, direction
  const T* KP;             // K p
  const T* B;              // right-hand sides
  T* SE;                   // ULISSE estimates
  long long n, ld;
  ColState* st;
  PcgAux* aux;
  const int* live;         // the columns this launch works on (one CTA each)
  double alpha_thr, eps, beta, delta, tau;
  int max_iter, inner_max;
  unsigned long long seed, step;
  int* status;
};

// s = 0, e = b, the J draws (as cg_init_kernel: column c, estimators 0 and 1).
template <typename T>
__global__ void __launch_bounds__(kPcgNT) pcg_init_kernel(const PcgArgs<T> a) {
  __shared__ double red[kPcgNT / 32];
  const int c = a.live[blockIdx.x];
  ColState& st = a.st[c];
  T* s = a.S + c * a.ld;
  T* e = a.E + c * a.ld;
  const T* b = a.B + c * a.ld;
  double pe = 0.0;
  for (long long i = threadIdx.x; i < a.n; i += kPcgNT) {
    s[i] = T(0);
    const T bi = b[i];
    e[i] = bi;
    pe += (double)bi * (double)bi;
  }
  const double ee = block_sum<kPcgNT>(pe, red);
  const bool done = sqrt(ee) < a.eps;
  if (done)
    for (int t = 0; t < st.n_est; ++t) {
      T* se = a.SE + (long long)(st.est_off + t) * a.ld;
      for (long long i = threadIdx.x; i < a.n; i += kPcgNT) se[i] = T(0);
    }
  __syncthreads();
  if (threadIdx.x == 0) {
    st.ee = ee;
    st.best_ee = ee;
    st.l = 0;
    st.m = 0;
    st.outcome = 0;
    st.J[0] = draw_J(a.seed, a.step, st.colid, 0, a.beta, a.max_iter);
    st.J[1] = st.n_est > 1 ? draw_J(a.seed, a.step, st.colid, 1, a.beta, a.max_iter) : -1;
    st.phase = done ? kDone : kPre;
  }
}

// Start the inner solve J z = e: x = 0, r = p = e.
template <typename T>
__global__ void __launch_bounds__(kPcgNT) pcg_inner_init_kernel(const PcgArgs<T> a) {
  const int c = a.live[blockIdx.x];
  const T* e = a.E + c * a.ld;
  T* x = a.X + c * a.ld;
  T* r = a.Rr + c * a.ld;
  T* p = a.P + c * a.ld;
  for (long long i = threadIdx.x; i < a.n; i += kPcgNT) {
    const T ei = e[i];
    x[i] = T(0);
    r[i] = ei;
    p[i] = ei;
  }
  if (threadIdx.x == 0) {
    const double ee = a.st[c].ee;
    PcgAux& ax = a.aux[c];
    ax.rr = ee;
    ax.thr = a.tau * a.tau * ee;
    ax.inner_it = 0;
    ax.inner_done = ee > 0.0 ? 0 : 1;
  }
}

// One inner CG iteration, K p given in KP.
template <typename T>
__global__ void __launch_bounds__(kPcgNT) pcg_inner_step_kernel(const PcgArgs<T> a) {
  __shared__ double red[kPcgNT / 32];
  const int c = a.live[blockIdx.x];
  PcgAux& ax = a.aux[c];
  T* x = a.X + c * a.ld;
  T* r = a.Rr + c * a.ld;
  T* p = a.P + c * a.ld;
  const T* kp = a.KP + c * a.ld;
  const T dl = (T)a.delta;
  double pq = 0.0;
  for (long long i = threadIdx.x; i < a.n; i += kPcgNT) {
    const T pi = p[i];
    pq += (double)pi * (double)fma(dl, pi, kp[i]);
  }
  pq = block_sum<kPcgNT>(pq, red);
  const double rr = ax.rr;
  if (!(pq > 0.0) || !isfinite(pq)) {
    // J is not positive definite along p, or a value is not finite: keep x as it is
    __syncthreads();
    if (threadIdx.x == 0) {
      ax.inner_done = 1;
      a.st[c].outcome = 3;
      atomicOr(a.status, kStatusBreakdown);
    }
    return;
  }
  const double al = rr / pq;
  const T alT = (T)al;
  double p2 = 0.0;
  for (long long i = threadIdx.x; i < a.n; i += kPcgNT) {
    const T pi = p[i];
    x[i] = fma(alT, pi, x[i]);
    const T ri = fma(-alT, fma(dl, pi, kp[i]), r[i]);
    r[i] = ri;
    p2 += (double)ri * (double)ri;
  }
  const double rr1 = block_sum<kPcgNT>(p2, red);
  const int it = ax.inner_it + 1;
  const bool done = rr1 <= ax.thr || it >= a.inner_max;
  if (!done) {
    const T btT = (T)(rr1 / rr);
    for (long long i = threadIdx.x; i < a.n; i += kPcgNT) p[i] = fma(btT, p[i], r[i]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ax.rr = rr1;
    ax.inner_it = it;
    ax.inner_done = done ? 1 : 0;
  }
}

// The new preconditioned residual z' = x: the first direction d = z', later the flexible
// update d = z' + beta d; e^T z' is kept for the next alpha.
template <typename T>
__global__ void __launch_bounds__(kPcgNT) pcg_dir_kernel(const PcgArgs<T> a) {
  __shared__ double red[kPcgNT / 32];
  const int c = a.live[blockIdx.x];
  ColState& st = a.st[c];
  PcgAux& ax = a.aux[c];
  const T* x = a.X + c * a.ld;
  const T* e = a.E + c * a.ld;
  T* z = a.Z + c * a.ld;
  T* d = a.D + c * a.ld;
  const bool first = st.m == 0;
  double pn = 0.0, po = 0.0;
  for (long long i = threadIdx.x; i < a.n; i += kPcgNT) {
    const double ei = (double)e[i];
    pn += ei * (double)x[i];
    if (!first) po += ei * (double)z[i];
  }
  const double ez_new = block_sum<kPcgNT>(pn, red);
  const double ez_old = first ? 0.0 : block_sum<kPcgNT>(po, red);
  if (!(ez_new > 0.0) || !isfinite(ez_new)) {
    // the inner solve gave a z with e^T z <= 0: the outer iteration cannot continue; a
    // column still before its early stop returns its current iterate
    const bool pre = st.phase == kPre;
    if (pre) {
      const T* s = a.S + c * a.ld;
      for (int t = 0; t < st.n_est; ++t) {
        T* se = a.SE + (long long)(st.est_off + t) * a.ld;
        for (long long i = threadIdx.x; i < a.n; i += kPcgNT) se[i] = s[i];
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      st.outcome = 3;
      st.phase = kDone;
      atomicOr(a.status, kStatusBreakdown);
    }
    return;
  }
  const T btT = first ? T(0) : (T)((ez_new - ez_old) / ax.ez);
  for (long long i = threadIdx.x; i < a.n; i += kPcgNT) {
    const T xi = x[i];
    d[i] = first ? xi : fma(btT, d[i], xi);
    z[i] = xi;
  }
  __syncthreads();
  if (threadIdx.x == 0) ax.ez = ez_new;
}

// One outer iteration with K d given: alpha, the updates of s and e, the ULISSE tail terms,
// and the early-stop / convergence / max_iter decisions (those of cg_finish_body).
template <typename T>
__global__ void __launch_bounds__(kPcgNT) pcg_step_kernel(const PcgArgs<T> a) {
  __shared__ double red[kPcgNT / 32];
  const int c = a.live[blockIdx.x];
  ColState& st = a.st[c];
  const PcgAux& ax = a.aux[c];
  T* s = a.S + c * a.ld;
  T* e = a.E + c * a.ld;
  const T* d = a.D + c * a.ld;
  const T* kd = a.KD + c * a.ld;
  T* se0 = a.SE + (long long)st.est_off * a.ld;
  const int phase = st.phase, l = st.l, m = st.m, n_est = st.n_est;
  const int J0 = st.J[0], J1 = st.J[1];
  double pd = 0.0;
  for (long long i = threadIdx.x; i < a.n; i += kPcgNT) pd += (double)d[i] * (double)kd[i];
  const double dKd = block_sum<kPcgNT>(pd, red);
  if (!(dKd > 0.0) || !isfinite(dKd)) {
    if (phase == kPre)
      for (int t = 0; t < n_est; ++t)
        for (long long i = threadIdx.x; i < a.n; i += kPcgNT) se0[t * a.ld + i] = s[i];
    __syncthreads();
    if (threadIdx.x == 0) {
      st.outcome = 3;
      st.phase = kDone;
      atomicOr(a.status, kStatusBreakdown);
    }
    return;
  }
  const double al = ax.ez / dKd;
  const T alT = (T)al;
  T w0 = T(0), w1 = T(0);
  if (phase == kTail) {
    const int j = m + 1 - l;
    const double Wa = weight_product(j, a.beta) * al;
    if (J0 >= j) w0 = (T)Wa;
    if (n_est > 1 && J1 >= j) w1 = (T)Wa;
  }
  T* se1 = se0 + a.ld;
  double p2 = 0.0;
  for (long long i = threadIdx.x; i < a.n; i += kPcgNT) {
    const T di = d[i];
    s[i] = fma(alT, di, s[i]);
    const T ei = fma(-alT, kd[i], e[i]);
    e[i] = ei;
    p2 += (double)ei * (double)ei;
    if (w0 != T(0)) se0[i] = fma(w0, di, se0[i]);
    if (w1 != T(0)) se1[i] = fma(w1, di, se1[i]);
  }
  const double ee1 = block_sum<kPcgNT>(p2, red);
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
      for (long long i = threadIdx.x; i < a.n; i += kPcgNT) se0[t * a.ld + i] = s[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    st.ee = ee1;
    st.m = m1;
    st.l = l1;
    st.outcome = outcome;
    st.phase = done ? kDone : ph;
    if (outcome == 4) atomicOr(a.status, kStatusMaxIter);
  }
}

}  // namespace ulisse
