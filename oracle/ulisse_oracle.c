/*
 * FP64 CPU oracle for SGLD + ULISSE on GP covariance parameters
 * (Filippone & Engler, "Enabling scalable stochastic gradient-based inference for
 * Gaussian processes by employing the Unbiased LInear System SolvEr (ULISSE)", ICML 2015).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the CUDA path is
 * checked against.  Only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg may load it.  It shares no code, header, table or constant generator with the CUDA
 * library: every routine here is written from the paper's text.
 *
 * Conventions (readings of the paper, each one also listed in the design notes):
 *   - Parameters are psi = log(theta), ordered (log l_1..log l_d, log sigma^2, log lambda),
 *     p = d + 2 (the paper samples theta = (sigma, tau, lambda), Sec. 2; the ARD form with
 *     one lengthscale per input dimension is the paper's stated extension, Sec. 6).
 *   - Covariance (Eq. covariance:rbf, read as the decaying ARD squared exponential):
 *       k(x_i, x_j) = sigma^2 exp(-1/2 sum_d (x_id - x_jd)^2 / l_d^2) + lambda delta_ij.
 *   - Derivatives with respect to psi (chain rule dK/dpsi = theta dK/dtheta):
 *       dK/dlog l_d    = k_s(x_i,x_j) (x_id - x_jd)^2 / l_d^2
 *       dK/dlog sigma2 = k_s(x_i,x_j)
 *       dK/dlog lambda = lambda delta_ij
 *     where k_s is the signal part (without the lambda term).
 *   - Matrices of vectors are column-major: column c of an n x R block starts at c*n.
 *   - Random numbers: Philox4x64-10 (Salmon et al., SC'11) keyed by (seed, 0); the counter
 *     names the draw: (index, column, step-or-epoch, purpose | estimator << 8).
 *
 * Everything is double precision.  Loops are the plain definitions; the only parallelism is
 * an OpenMP loop over output rows of the O(n^2) products.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_D 16
#define ORC_PURPOSE_PROBE 1u
#define ORC_PURPOSE_ULISSE 2u
#define ORC_PURPOSE_SGLD 3u

/* Column outcome codes reported by orc_ulisse_solve. */
#define ORC_OK 0
#define ORC_BREAKDOWN 3
#define ORC_MAXITER 4

/* ------------------------------------------------------------------------------------ */
/* Philox4x64-10, from the published description (Salmon, Moraes, Dror, Shaw, SC'11):    */
/* each round multiplies counter words 0 and 2 by fixed odd constants, keeps the 128-bit  */
/* products' high and low halves, mixes the high halves with the other two counter words  */
/* and the key, and permutes; the key is bumped by the Weyl constants between rounds.     */
/* ------------------------------------------------------------------------------------ */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        unsigned __int128 p0 = (unsigned __int128)M0 * c0;
        unsigned __int128 p1 = (unsigned __int128)M1 * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        uint64_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform on [0,1) from the top 53 bits of a 64-bit word. */
double orc_u01(uint64_t w) { return (double)(w >> 11) * 0x1.0p-53; }

static void draw(uint64_t seed, uint64_t i, uint64_t col, uint64_t step, uint64_t tag, uint64_t out[4])
{
    uint64_t ctr[4] = {i, col, step, tag};
    uint64_t key[2] = {seed, 0};
    orc_philox4x64_10(ctr, key, out);
}

/* Standard normal by the Box-Muller transform (one of the pair). */
static double box_muller(uint64_t w0, uint64_t w1)
{
    double u1 = orc_u01(w0), u2 = orc_u01(w1);
    return sqrt(-2.0 * log(1.0 - u1)) * cos(2.0 * M_PI * u2);
}

/* ------------------------------------------------------------------------------------ */
/* Covariance function and its derivatives (Eq. covariance:rbf, ARD reading).            */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    int d;
    double inv_l2[ORC_MAX_D]; /* 1 / l_d^2 */
    double sigma2;
    double lambda;
} orc_theta;

static orc_theta unpack(const double *psi, int d)
{
    orc_theta t;
    if (d < 1 || d > ORC_MAX_D) {
        fprintf(stderr, "oracle: input width %d outside 1..%d\n", d, ORC_MAX_D);
        abort();
    }
    t.d = d;
    for (int k = 0; k < d; ++k) {
        double l = exp(psi[k]);
        t.inv_l2[k] = 1.0 / (l * l);
    }
    t.sigma2 = exp(psi[d]);
    t.lambda = exp(psi[d + 1]);
    return t;
}

static double k_signal(const double *xi, const double *xj, const orc_theta *t)
{
    double sq = 0.0;
    for (int k = 0; k < t->d; ++k) {
        double diff = xi[k] - xj[k];
        sq += diff * diff * t->inv_l2[k];
    }
    return t->sigma2 * exp(-0.5 * sq);
}

/* Entry (i,j) of K (which = -1) or of dK/dpsi_which (0 <= which < d+2). */
static double entry(const double *X, long i, long j, const orc_theta *t, int which)
{
    const int d = t->d;
    const double *xi = X + i * d, *xj = X + j * d;
    if (which == d + 1) return (i == j) ? t->lambda : 0.0;
    double ks = k_signal(xi, xj, t);
    if (which == -1) return ks + ((i == j) ? t->lambda : 0.0);
    if (which == d) return ks;
    double diff = xi[which] - xj[which];
    return ks * diff * diff * t->inv_l2[which];
}

/* Dense K or dK/dpsi_which, n x n row-major (small n only). */
void orc_cov_matrix(const double *X, long n, int d, const double *psi, int which, double *K)
{
    orc_theta t = unpack(psi, d);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i)
        for (long j = 0; j < n; ++j) K[i * n + j] = entry(X, i, j, &t, which);
}

/* ------------------------------------------------------------------------------------ */
/* Covariance matrix-vector products without storing K (Sec. 3: O(n^2) time, O(n) space). */
/* U[:, r] = A V[:, r] with A = K (which = -1) or dK/dpsi_which.                          */
/* ------------------------------------------------------------------------------------ */
void orc_kmv(const double *X, long n, int d, const double *psi, int which,
             const double *V, int R, double *U)
{
    orc_theta t = unpack(psi, d);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
        /* every column, in blocks of 512 accumulators */
        double acc[512];
        for (int r0 = 0; r0 < R; r0 += 512) {
            const int Rc = R - r0 < 512 ? R - r0 : 512;
            for (int r = 0; r < Rc; ++r) acc[r] = 0.0;
            for (long j = 0; j < n; ++j) {
                double a = entry(X, i, j, &t, which);
                for (int r = 0; r < Rc; ++r) acc[r] += a * V[(long)(r0 + r) * n + j];
            }
            for (int r = 0; r < Rc; ++r) U[(long)(r0 + r) * n + i] = acc[r];
        }
    }
}

/* The same product restricted to the output rows listed in rows[0..nrows-1]:
 * U[k + r*nrows] = sum_j A[rows[k], j] V[j, r]  (for checks of large problems). */
void orc_kmv_rows(const double *X, long n, int d, const double *psi, int which,
                  const double *V, int R, const long *rows, long nrows, double *U)
{
    orc_theta t = unpack(psi, d);
#pragma omp parallel for schedule(dynamic, 4)
    for (long k = 0; k < nrows; ++k) {
        const long i = rows[k];
        for (int r = 0; r < R; ++r) {
            double acc = 0.0;
            for (long j = 0; j < n; ++j) acc += entry(X, i, j, &t, which) * V[(long)r * n + j];
            U[(long)r * nrows + k] = acc;
        }
    }
}

/* Sum over j of |A[i,j]| |V[j,r]| for the listed rows: the scale of each output entry's
 * rounding error (a dot product's condition). */
void orc_kmv_rows_abs(const double *X, long n, int d, const double *psi, int which,
                      const double *V, int R, const long *rows, long nrows, double *U)
{
    orc_theta t = unpack(psi, d);
#pragma omp parallel for schedule(dynamic, 4)
    for (long k = 0; k < nrows; ++k) {
        const long i = rows[k];
        for (int r = 0; r < R; ++r) {
            double acc = 0.0;
            for (long j = 0; j < n; ++j)
                acc += fabs(entry(X, i, j, &t, which)) * fabs(V[(long)r * n + j]);
            U[(long)r * nrows + k] = acc;
        }
    }
}

/* All p derivative products restricted to the listed output rows:
 * U_all[(q*R + r)*nrows + k] = sum_j dK/dpsi_q[rows[k], j] V[j, r]. */
void orc_dkmv_all_rows(const double *X, long n, int d, const double *psi, const double *V,
                       int R, const long *rows, long nrows, double *U_all)
{
    orc_theta t = unpack(psi, d);
    const int p = d + 2;
#pragma omp parallel for schedule(dynamic, 4)
    for (long k = 0; k < nrows; ++k) {
        const long i = rows[k];
        const double *xi = X + i * d;
        for (int q = 0; q < p; ++q)
            for (int r = 0; r < R; ++r) U_all[((long)q * R + r) * nrows + k] = 0.0;
        for (long j = 0; j < n; ++j) {
            const double *xj = X + j * d;
            double ks = k_signal(xi, xj, &t);
            for (int q = 0; q < d; ++q) {
                double diff = xi[q] - xj[q];
                double a = ks * diff * diff * t.inv_l2[q];
                for (int r = 0; r < R; ++r) U_all[((long)q * R + r) * nrows + k] += a * V[(long)r * n + j];
            }
            for (int r = 0; r < R; ++r) U_all[((long)d * R + r) * nrows + k] += ks * V[(long)r * n + j];
            if (i == j)
                for (int r = 0; r < R; ++r) U_all[((long)(d + 1) * R + r) * nrows + k] += t.lambda * V[(long)r * n + j];
        }
    }
}

/* Signal covariance between two point sets: C[a*n2 + b] = k_s(x1_a, x2_b) (n1 x n2,
 * row-major; no noise term: the points are distinct inputs of the model). */
void orc_cross_signal(const double *X1, long n1, const double *X2, long n2, int d,
                      const double *psi, double *C)
{
    orc_theta t = unpack(psi, d);
#pragma omp parallel for schedule(static)
    for (long a = 0; a < n1; ++a)
        for (long b = 0; b < n2; ++b) C[a * n2 + b] = k_signal(X1 + a * d, X2 + b * d, &t);
}

/* All p derivative products in one sweep over the entries:
 * U_all[q] (n x R, col-major, q = 0..p-1) = dK/dpsi_q V. */
void orc_dkmv_all(const double *X, long n, int d, const double *psi,
                  const double *V, int R, double *U_all)
{
    orc_theta t = unpack(psi, d);
    const int p = d + 2;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
        const double *xi = X + i * d;
        for (int q = 0; q < p; ++q)
            for (int r = 0; r < R; ++r) U_all[((long)q * R + r) * n + i] = 0.0;
        for (long j = 0; j < n; ++j) {
            const double *xj = X + j * d;
            double ks = k_signal(xi, xj, &t);
            for (int q = 0; q < d; ++q) {
                double diff = xi[q] - xj[q];
                double a = ks * diff * diff * t.inv_l2[q];
                for (int r = 0; r < R; ++r) U_all[((long)q * R + r) * n + i] += a * V[(long)r * n + j];
            }
            for (int r = 0; r < R; ++r) U_all[((long)d * R + r) * n + i] += ks * V[(long)r * n + j];
            if (i == j)
                for (int r = 0; r < R; ++r) U_all[((long)(d + 1) * R + r) * n + i] += t.lambda * V[(long)r * n + j];
        }
    }
}

/* ------------------------------------------------------------------------------------ */
/* Hutchinson probes (Sec. 2.1): entries +-1 with probability 1/2 (kind 0) or standard   */
/* normal (kind 1).  Column j (1-based probe index) of the solve's right-hand sides.     */
/* ------------------------------------------------------------------------------------ */
void orc_probes(long n, int nr, int kind, uint64_t seed, uint64_t epoch, double *Rm)
{
    for (int j = 0; j < nr; ++j)
        for (long i = 0; i < n; ++i) {
            uint64_t w[4];
            draw(seed, (uint64_t)i, (uint64_t)(j + 1), epoch, ORC_PURPOSE_PROBE, w);
            double v = (kind == 0) ? ((w[0] >> 63) ? -1.0 : 1.0) : box_muller(w[0], w[1]);
            Rm[(long)j * n + i] = v;
        }
}

/* ------------------------------------------------------------------------------------ */
/* ULISSE truncation (Sec. 4): after the early-stop threshold is reached at iteration l,  */
/* step j = 1, 2, ... is accepted while u_j < 1/w_j with w_r = exp(beta r); w_0 = 1 so   */
/* step 0 always is.  Drawing the u_j up front gives the number J of accepted steps       */
/* j >= 1 (the acceptance can be simulated beforehand since it does not depend on CG).    */
/* ------------------------------------------------------------------------------------ */
int orc_draw_J(uint64_t seed, uint64_t step, uint64_t colid, int est, double beta, int jcap)
{
    int J = 0;
    for (int j = 1; j <= jcap; ++j) {
        uint64_t w[4];
        draw(seed, (uint64_t)j, colid, step, ORC_PURPOSE_ULISSE | ((uint64_t)est << 8), w);
        double u = orc_u01(w[0]);
        double inv_w = exp(-beta * (double)j);
        if (u < inv_w) J = j; else break;
    }
    return J;
}

/* prod_{r=0}^{j} w_r with w_r = exp(beta r), as a literal product. */
static double weight_product(int j, double beta)
{
    double W = 1.0;
    for (int r = 0; r <= j; ++r) W *= exp(beta * (double)r);
    return W;
}

static double dot(const double *a, const double *b, long n)
{
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* ------------------------------------------------------------------------------------ */
/* Algorithm 1 (CG), one column, with every iterate recorded (small n, for the tests).   */
/* S, E, D: n x (max_iter+1) col-major; alpha, beta: max_iter.  Returns the number T of   */
/* iterations done; S[:, T] is the returned solution.                                     */
/* ------------------------------------------------------------------------------------ */
int orc_cg_record(const double *X, long n, int d, const double *psi, const double *b,
                  const double *s0, double eps, int max_iter,
                  double *S, double *E, double *D, double *alpha_out, double *beta_out)
{
    double *Kv = (double *)malloc(sizeof(double) * n);
    for (long i = 0; i < n; ++i) S[i] = s0 ? s0[i] : 0.0;
    if (s0) {
        orc_kmv(X, n, d, psi, -1, S, 1, Kv);
        for (long i = 0; i < n; ++i) E[i] = b[i] - Kv[i];
    } else {
        for (long i = 0; i < n; ++i) E[i] = b[i];
    }
    for (long i = 0; i < n; ++i) D[i] = E[i];
    int T = 0;
    for (int it = 0; it < max_iter; ++it) {
        double *s = S + (long)it * n, *e = E + (long)it * n, *dv = D + (long)it * n;
        double *s1 = s + n, *e1 = e + n, *d1 = dv + n;
        orc_kmv(X, n, d, psi, -1, dv, 1, Kv);
        double ee = dot(e, e, n);
        double a = ee / dot(dv, Kv, n);
        for (long i = 0; i < n; ++i) s1[i] = s[i] + a * dv[i];
        for (long i = 0; i < n; ++i) e1[i] = e[i] - a * Kv[i];
        alpha_out[it] = a;
        T = it + 1;
        double ee1 = dot(e1, e1, n);
        if (sqrt(ee1) < eps) { beta_out[it] = 0.0; break; }
        double bt = ee1 / ee;
        beta_out[it] = bt;
        for (long i = 0; i < n; ++i) d1[i] = e1[i] + bt * dv[i];
    }
    free(Kv);
    return T;
}

/* ------------------------------------------------------------------------------------ */
/* ULISSE (Sec. 4) on R columns.  Each column runs Algorithm 1 on its own right-hand side */
/* (the columns only share the O(n^2) sweep that forms K d for all live columns).        */
/* Column c carries n_est[c] independent estimators (two for y, Sec. 4.1), each with its  */
/* own uniforms.  The estimate is                                                         */
/*   s~ = s_0 + sum_{i<l} delta_i + sum_{j=0}^{J} (prod_{r<=j} w_r) delta_{l+j}           */
/* where l is the first iteration i >= 1 with ||e_i|| < alpha, alpha = q sqrt(n).          */
/* Outputs: S_est has sum(n_est) columns (estimators of column 0 first, then column 1...). */
/* stats per column: [l, iterations, outcome, J_0, J_1] (l = 0 if never reached).         */
/* ------------------------------------------------------------------------------------ */
void orc_ulisse_solve(const double *X, long n, int d, const double *psi,
                      const double *B, int R, const double *S0, const int *n_est,
                      const int64_t *colid, double q, double beta, double eps, int max_iter,
                      uint64_t seed, uint64_t step, double *S_est, int64_t *stats)
{
    const double alpha_thr = q * sqrt((double)n);
    double *s = (double *)calloc((size_t)n * R, sizeof(double));
    double *e = (double *)calloc((size_t)n * R, sizeof(double));
    double *dv = (double *)calloc((size_t)n * R, sizeof(double));
    double *Kd = (double *)calloc((size_t)n * R, sizeof(double));
    double *Dlive = (double *)calloc((size_t)n * R, sizeof(double));
    double *ee = (double *)calloc((size_t)R, sizeof(double));
    int *phase = (int *)calloc((size_t)R, sizeof(int)); /* 0 pre, 1 tail, 2 done */
    int *l = (int *)calloc((size_t)R, sizeof(int));
    int *m = (int *)calloc((size_t)R, sizeof(int));
    int *J = (int *)calloc((size_t)R * 2, sizeof(int));
    int *outcome = (int *)calloc((size_t)R, sizeof(int));
    int *est_off = (int *)calloc((size_t)R, sizeof(int));
    int *live = (int *)calloc((size_t)R, sizeof(int));

    int off = 0;
    for (int c = 0; c < R; ++c) { est_off[c] = off; off += n_est[c]; }

    /* e_0 = b - K s_0, d_0 = e_0 (Algorithm 1).  A given s_0 is kept for a column only   */
    /* when ||b - K s_0|| < ||b||; otherwise the column starts from s_0 = 0.  The choice   */
    /* uses no random draw, so the estimators stay unbiased whichever start is taken.      */
    for (int c = 0; c < R; ++c)
        for (long i = 0; i < n; ++i) s[(long)c * n + i] = S0 ? S0[(long)c * n + i] : 0.0;
    if (S0) orc_kmv(X, n, d, psi, -1, s, R, Kd);
    for (int c = 0; c < R; ++c) {
        const double *bc = B + (long)c * n;
        int keep = 0;
        if (S0) {
            double rr = 0.0;
            for (long i = 0; i < n; ++i) {
                const double r = bc[i] - Kd[(long)c * n + i];
                rr += r * r;
            }
            keep = rr < dot(bc, bc, n);
        }
        for (long i = 0; i < n; ++i) {
            long k = (long)c * n + i;
            if (!keep) s[k] = 0.0;
            e[k] = B[k] - (keep ? Kd[k] : 0.0);
            dv[k] = e[k];
        }
        ee[c] = dot(e + (long)c * n, e + (long)c * n, n);
        for (int t = 0; t < n_est[c]; ++t)
            J[2 * c + t] = orc_draw_J(seed, step, (uint64_t)colid[c], t, beta, max_iter);
        if (sqrt(ee[c]) < eps) {
            /* Already converged at s_0: every estimator returns s_0. */
            for (int t = 0; t < n_est[c]; ++t)
                memcpy(S_est + (long)(est_off[c] + t) * n, s + (long)c * n, sizeof(double) * n);
            phase[c] = 2;
        }
    }

    for (;;) {
        int nlive = 0;
        for (int c = 0; c < R; ++c)
            if (phase[c] != 2) live[nlive++] = c;
        if (nlive == 0) break;
        /* K d for every live column. */
        for (int a = 0; a < nlive; ++a)
            memcpy(Dlive + (long)a * n, dv + (long)live[a] * n, sizeof(double) * n);
        orc_kmv(X, n, d, psi, -1, Dlive, nlive, Kd);
        for (int a = 0; a < nlive; ++a) {
            const int c = live[a];
            double *sc = s + (long)c * n, *ec = e + (long)c * n, *dc = dv + (long)c * n;
            const double *kd = Kd + (long)a * n;
            double dKd = dot(dc, kd, n);
            if (!(dKd > 0.0) || !isfinite(dKd)) {
                /* Breakdown: K not positive definite along d (or a non-finite value). */
                outcome[c] = ORC_BREAKDOWN;
                for (int t = 0; t < n_est[c]; ++t)
                    if (phase[c] == 0)
                        memcpy(S_est + (long)(est_off[c] + t) * n, sc, sizeof(double) * n);
                phase[c] = 2;
                continue;
            }
            double al = ee[c] / dKd;
            /* delta_{m+1} = al d_m; s_{m+1} = s_m + delta; e_{m+1} = e_m - al K d_m. */
            for (long i = 0; i < n; ++i) sc[i] += al * dc[i];
            for (long i = 0; i < n; ++i) ec[i] -= al * kd[i];
            double ee1 = dot(ec, ec, n);
            m[c] += 1;
            if (phase[c] == 1) {
                int j = m[c] - l[c];
                double Wj = weight_product(j, beta);
                for (int t = 0; t < n_est[c]; ++t)
                    if (J[2 * c + t] >= j) {
                        double *st = S_est + (long)(est_off[c] + t) * n;
                        for (long i = 0; i < n; ++i) st[i] += Wj * (al * dc[i]);
                    }
            }
            int jmax = 0;
            for (int t = 0; t < n_est[c]; ++t) if (J[2 * c + t] > jmax) jmax = J[2 * c + t];
            if (phase[c] == 0 && sqrt(ee1) < alpha_thr) {
                l[c] = m[c];
                phase[c] = 1;
                for (int t = 0; t < n_est[c]; ++t)
                    memcpy(S_est + (long)(est_off[c] + t) * n, sc, sizeof(double) * n);
            }
            int converged = sqrt(ee1) < eps;
            if (phase[c] == 0 && converged) {
                for (int t = 0; t < n_est[c]; ++t)
                    memcpy(S_est + (long)(est_off[c] + t) * n, sc, sizeof(double) * n);
                phase[c] = 2;
            } else if (phase[c] == 1 && (m[c] - l[c] >= jmax || converged)) {
                phase[c] = 2;
            } else if (m[c] >= max_iter) {
                if (phase[c] == 0)
                    for (int t = 0; t < n_est[c]; ++t)
                        memcpy(S_est + (long)(est_off[c] + t) * n, sc, sizeof(double) * n);
                outcome[c] = ORC_MAXITER;
                phase[c] = 2;
            }
            if (phase[c] != 2) {
                double bt = ee1 / ee[c];
                for (long i = 0; i < n; ++i) dc[i] = ec[i] + bt * dc[i];
            }
            ee[c] = ee1;
        }
    }
    for (int c = 0; c < R; ++c) {
        stats[5 * c + 0] = l[c];
        stats[5 * c + 1] = m[c];
        stats[5 * c + 2] = outcome[c];
        stats[5 * c + 3] = J[2 * c];
        stats[5 * c + 4] = n_est[c] > 1 ? J[2 * c + 1] : -1;
    }
    free(s); free(e); free(dv); free(Kd); free(Dlive); free(ee); free(phase); free(l);
    free(m); free(J); free(outcome); free(est_off); free(live);
}

/* ------------------------------------------------------------------------------------ */
/* Unbiased gradient (Eq. gradient:unbiased), with psi coordinates:                       */
/*   g~_i = 1/2 a1^T dK_i a2 - 1/(2 Nr) sum_j z_j^T dK_i r_j                               */
/* where a1, a2 are two independent ULISSE estimates of K^{-1} y from one CG run and      */
/* z_j the ULISSE estimate of K^{-1} r_j (Sec. 4.1).  The probes are redrawn every         */
/* probe_refresh steps (epoch = step / probe_refresh).                                    */
/* stats: per column [l, iterations, outcome, J_0, J_1] for the 1+Nr columns.              */
/* ------------------------------------------------------------------------------------ */
void orc_grad_estimate(const double *X, const double *y, long n, int d, const double *psi,
                       int nr, int probe_kind, int probe_refresh, double q, double beta,
                       double eps, int max_iter, uint64_t seed, uint64_t step,
                       double *g, int64_t *stats)
{
    const int R = 1 + nr, p = d + 2;
    double *B = (double *)malloc(sizeof(double) * n * R);
    double *S_est = (double *)malloc(sizeof(double) * n * (R + 1));
    int *n_est = (int *)malloc(sizeof(int) * R);
    int64_t *colid = (int64_t *)malloc(sizeof(int64_t) * R);
    memcpy(B, y, sizeof(double) * n);
    uint64_t epoch = step / (uint64_t)(probe_refresh > 0 ? probe_refresh : 1);
    orc_probes(n, nr, probe_kind, seed, epoch, B + n);
    for (int c = 0; c < R; ++c) { n_est[c] = (c == 0) ? 2 : 1; colid[c] = c; }
    orc_ulisse_solve(X, n, d, psi, B, R, NULL, n_est, colid, q, beta, eps, max_iter, seed,
                     step, S_est, stats);
    /* S_est columns: a1, a2, z_1..z_Nr.  Right factors: a2, r_1..r_Nr. */
    double *Rt = (double *)malloc(sizeof(double) * n * R);
    memcpy(Rt, S_est + n, sizeof(double) * n);            /* a2 */
    memcpy(Rt + n, B + n, sizeof(double) * n * nr);       /* r_j */
    double *U = (double *)malloc(sizeof(double) * n * R * p);
    orc_dkmv_all(X, n, d, psi, Rt, R, U);
    for (int i = 0; i < p; ++i) {
        const double *Ui = U + (long)i * R * n;
        double quad = dot(S_est, Ui, n);                  /* a1^T dK_i a2 */
        double tr = 0.0;
        for (int j = 0; j < nr; ++j)
            tr += dot(S_est + (long)(2 + j) * n, Ui + (long)(1 + j) * n, n); /* z_j^T dK_i r_j */
        g[i] = 0.5 * quad - tr / (2.0 * nr);
    }
    free(B); free(S_est); free(n_est); free(colid); free(Rt); free(U);
}

/* Cholesky factor L (lower, row-major) of a symmetric positive definite p x p matrix.
 * Returns 0 on success, -1 if a pivot is not positive. */
int orc_chol(int p, const double *M, double *L)
{
    for (int i = 0; i < p * p; ++i) L[i] = 0.0;
    for (int j = 0; j < p; ++j) {
        double s = M[j * p + j];
        for (int k = 0; k < j; ++k) s -= L[j * p + k] * L[j * p + k];
        if (!(s > 0.0)) return -1;
        L[j * p + j] = sqrt(s);
        for (int i = j + 1; i < p; ++i) {
            double t = M[i * p + j];
            for (int k = 0; k < j; ++k) t -= L[i * p + k] * L[j * p + k];
            L[i * p + j] = t / L[j * p + j];
        }
    }
    return 0;
}

/* Standard normal vector xi (p entries) for the SGLD noise of a step. */
void orc_sgld_noise(uint64_t seed, uint64_t step, int p, double *xi)
{
    for (int k = 0; k < p; ++k) {
        uint64_t w[4];
        draw(seed, (uint64_t)k, 0, step, ORC_PURPOSE_SGLD, w);
        xi[k] = box_muller(w[0], w[1]);
    }
}

/* SGLD proposal (Sec. 2.1): psi' = psi + eps/2 M (g~ + grad log p) + eta, eta ~ N(0, eps M),
 * eta = sqrt(eps) L xi with L L^T = M.  M = NULL means the identity; prior_grad = NULL
 * means a flat prior.  Returns 0, or -1 if M is not positive definite. */
int orc_sgld_update(int p, const double *psi, const double *g, const double *M,
                    const double *prior_grad, double eps_t, uint64_t seed, uint64_t step,
                    double *psi_out)
{
    double L[ORC_MAX_D + 2][ORC_MAX_D + 2], Mm[(ORC_MAX_D + 2) * (ORC_MAX_D + 2)];
    double xi[ORC_MAX_D + 2], v[ORC_MAX_D + 2];
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j) Mm[i * p + j] = M ? M[i * p + j] : (i == j ? 1.0 : 0.0);
    double Lf[(ORC_MAX_D + 2) * (ORC_MAX_D + 2)];
    if (orc_chol(p, Mm, Lf) != 0) return -1;
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j) L[i][j] = Lf[i * p + j];
    orc_sgld_noise(seed, step, p, xi);
    for (int i = 0; i < p; ++i) v[i] = g[i] + (prior_grad ? prior_grad[i] : 0.0);
    for (int i = 0; i < p; ++i) {
        double drift = 0.0, noise = 0.0;
        for (int j = 0; j < p; ++j) drift += Mm[i * p + j] * v[j];
        for (int j = 0; j <= i; ++j) noise += L[i][j] * xi[j];
        psi_out[i] = psi[i] + 0.5 * eps_t * drift + sqrt(eps_t) * noise;
    }
    return 0;
}

/* One SGLD step with the ULISSE gradient: the whole path of the method for one step. */
int orc_sgld_step(const double *X, const double *y, long n, int d, const double *psi,
                  int nr, int probe_kind, int probe_refresh, double q, double beta, double eps,
                  int max_iter, uint64_t seed, uint64_t step, double eps_t, const double *M,
                  const double *prior_grad, double *psi_out, double *g, int64_t *stats)
{
    orc_grad_estimate(X, y, n, d, psi, nr, probe_kind, probe_refresh, q, beta, eps, max_iter,
                      seed, step, g, stats);
    return orc_sgld_update(d + 2, psi, g, M, prior_grad, eps_t, seed, step, psi_out);
}
