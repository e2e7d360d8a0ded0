/*
 * ulisse.h -- C ABI of libulisse, a GB300 (sm_103a) implementation of the hot path of
 * "Enabling scalable stochastic gradient-based inference for Gaussian processes by
 * employing the Unbiased LInear System SolvEr (ULISSE)" (Filippone & Engler, ICML 2015).
 *
 * The library samples GP covariance parameters with stochastic gradient Langevin dynamics
 * (SGLD, Sec. 2.1).  Each gradient is the unbiased estimate of Eq. gradient:unbiased, built
 * from ULISSE solves (Sec. 4) of K s = y and K s = r_j for Hutchinson probes r_j; every
 * solve iterates matrix-free covariance products K V (Sec. 3), generated tile by tile on the
 * GPU and never stored.
 *
 * Model (Eq. covariance:rbf, read as the decaying ARD squared exponential; Sec. 6 names the
 * ARD extension):
 *     k(x_i, x_j) = sigma^2 exp(-1/2 sum_d (x_id - x_jd)^2 / l_d^2) + lambda delta_ij
 * Parameters are psi = log theta = (log l_1 .. log l_d, log sigma^2, log lambda), p = d + 2;
 * derivatives are taken with respect to psi (dK/dpsi_i = theta_i dK/dtheta_i).
 *
 * Conventions for every call:
 *   - Pointers marked "device" are CUDA device pointers on the context's device; "host"
 *     pointers are ordinary host memory (pinned or pageable).  The caller owns every buffer
 *     it passes; the context owns its own scratch.
 *   - Blocks of vectors are column-major: column c of an n x R block starts at c * n
 *     (leading dimension n).  float unless stated otherwise.
 *   - All GPU work is ordered on the stream given to ulisse_create (a cudaStream_t passed
 *     as void*; NULL = the legacy default stream).  Calls that return host results
 *     synchronise that stream before returning.
 *   - Every call returns a ulisse_status and never aborts.  ulisse_last_error gives a
 *     message for the last failing call.  Kernels report breakdowns through a device status
 *     word that the next synchronising call reads; no kernel traps.
 *   - Results are deterministic for a given (seed, step): random draws come from a
 *     counter-based generator (Philox4x64-10) and reductions use a fixed order.
 *   - Not thread-safe per context: calls on one context must not overlap.
 */
#ifndef ULISSE_H
#define ULISSE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ulisse_ctx ulisse_ctx;

typedef enum {
    ULISSE_OK = 0,
    ULISSE_ERR_ARG = 1,       /* invalid argument (null pointer, size out of range, ...) */
    ULISSE_ERR_CUDA = 2,      /* a CUDA runtime call failed */
    ULISSE_ERR_BREAKDOWN = 3, /* CG breakdown: d^T K d <= 0 or a non-finite value (K not
                                 positive definite along d, or NaN in the inputs) */
    ULISSE_ERR_MAXITER = 4,   /* a solve hit max_iter before its stopping rule: the
                                 estimate is returned but is not unbiased */
    ULISSE_ERR_NOMEM = 5,     /* device allocation failed */
    ULISSE_ERR_TIMEOUT = 6    /* a bounded device wait ran out (the kernel returned early) */
} ulisse_status;

typedef enum {
    ULISSE_PREC_FP32 = 0,     /* FP32 vectors and SIMT products, FP64 scalar recurrences */
    ULISSE_PREC_MIXED = 1,    /* tensor-core (tcgen05) products, FP32 vectors: K V with the
                                 exponent's dot product by three TF32 products and the
                                 contraction by three BF16 products, the gradient's bilinear
                                 forms by three BF16 products (its exponent's dot product by
                                 three TF32 products for d <= 8); each result's error is
                                 stated at the call (about 1e-4 of its dot-product scale at
                                 most) */
    ULISSE_PREC_FP64 = 2      /* FP64 everywhere (the paper's double-precision CMVPs) */
} ulisse_precision;

typedef enum {
    ULISSE_PROBE_RADEMACHER = 0, /* entries +-1 with probability 1/2 (Sec. 2.1) */
    ULISSE_PROBE_GAUSSIAN = 1    /* entries N(0,1); also E[r r^T] = I */
} ulisse_probe_kind;

typedef struct {
    int precision;           /* ulisse_precision */
    int n_probes;            /* N_r >= 1, Hutchinson probes per gradient (Eq. gradient:unbiased) */
    int probe_kind;          /* ulisse_probe_kind */
    int probe_refresh;       /* redraw the probes every probe_refresh steps (>= 1; the paper's
                                Concrete run used 20, Sec. 5.1); epoch = step / probe_refresh */
    int warm_start_probes;   /* nonzero: start each solve from the previous step's final CG
                                iterate of its column while the right-hand side is unchanged
                                -- y always, the probes within a refresh epoch (Sec. 5.1's
                                reuse of probes and solutions); one extra K V round forms the
                                initial residuals, and an iterate is kept only when it lowers
                                the residual (no random draw: the estimates stay unbiased). */
    double q;                /* early-stop threshold alpha = q sqrt(n) (Sec. 4; the paper uses q=1) */
    double beta;             /* ULISSE weights w_r = exp(beta r) (Sec. 4; the paper uses beta=1) */
    double eps;              /* CG convergence threshold on ||e|| (Algorithm 1; paper: 1e-8) */
    int max_iter;            /* cap on CG iterations per solve (>= 1) */
    unsigned long long seed; /* key of the counter-based generator */
    int kmv_rows_per_thread; /* K V tile shape: output rows per thread, 2 or 4; 0 = the
                                tuned default.  Changes the summation order of the split
                                j range, hence the last bits of the results. */
    int tc_cross_term;       /* mixed precision: where the cross term x^_i . x^_j of the
                                K V products' kernel values is formed (the gradient pass
                                forms it on the tensor cores for d <= 8, on the CUDA cores
                                for d > 8, whatever this says) -- 1 = FP32 FMAs on the CUDA
                                cores, 2 = three TF32 products on the tensor cores (x^ split
                                into a TF32 high part and the remainder), 0 = the default (2)
                                or the autotuner's choice.  The two differ in the last bits of each
                                kernel value (relative 1e-6 to 1e-5). */
    double pcg_delta;        /* 0: the solves run CG (Algorithm 1).  > 0: preconditioned CG
                                with J = K + pcg_delta I (Sec. 3, "Preconditioned CG"), every
                                iteration solving J z = e by an inner CG on the same K V
                                products (same precision); ULISSE truncates the outer
                                iteration (Sec. 4).  Solves then start from zero
                                (warm_start_probes = 0, no S0, no learned warm start) and a
                                step runs from the host loop. */
    double pcg_inner_tol;    /* inner CG stops at ||r|| <= pcg_inner_tol ||e||, 0 < tol < 1 */
    int pcg_inner_max;       /* ... or after this many inner iterations (>= 1) */
} ulisse_config;

/* Fill *cfg with the paper's settings: FP32, 4 Rademacher probes redrawn every step,
 * q = 1, beta = 1, eps = 1e-8, max_iter = 1000, seed 0, tuned K V tile shape, plain CG
 * (pcg_delta = 0; pcg_inner_tol = 1e-2, pcg_inner_max = 100 when enabled). */
void ulisse_config_default(ulisse_config *cfg);

/*
 * Create a context for one GP regression problem (Sec. 2: labels y for inputs X).
 *   X      device, n x d float, ROW-major (point i at X + i*d); copied into the context.
 *   y      device, n floats; copied into the context.
 *   n      number of inputs, 1 <= n <= 2^31 - 1.
 *   d      input dimension, 1 <= d <= 16.
 *   cfg    host; copied.  stream: cudaStream_t (as void*) for all later work.
 * The context selects the current CUDA device at creation and uses it for its lifetime.
 * Errors: ULISSE_ERR_ARG (null pointers, n or d out of range, bad cfg), ULISSE_ERR_NOMEM.
 */
ulisse_status ulisse_create(ulisse_ctx **out, const float *X, const float *y, long long n,
                            int d, const ulisse_config *cfg, void *stream);

/* As ulisse_create, but X and y are HOST arrays (row-major n x d, and n). */
ulisse_status ulisse_create_host(ulisse_ctx **out, const float *X, const float *y,
                                 long long n, int d, const ulisse_config *cfg, void *stream);

/*
 * Covariance matrix-vector products without storing K (Sec. 3; Algorithm 1's CMVP):
 *     U = A V,  A = K(psi) if which == -1, else A = dK/dpsi_which (0 <= which < d+2).
 *   psi  host, p = d+2 doubles.
 *   V    device, n x R column-major (leading dimension n), R >= 1.
 *   U    device, n x R column-major; must not overlap V.
 * In FP64 precision V and U are read and written as float and converted; use
 * ulisse_kmv_f64 for double data.  In mixed precision K V (which == -1) runs on the tensor
 * cores (each entry of U within 1e-4 of sum_j |K_ij| |V_jr|) and the derivative products in
 * FP32.  Asynchronous on the context's stream.
 * Errors: ULISSE_ERR_ARG (which out of range, R < 1, null, non-finite psi).
 */
ulisse_status ulisse_kmv(ulisse_ctx *ctx, const double *psi, int which, const float *V, int R,
                         float *U);

/* As ulisse_kmv with double V and U (computed in FP64 on the GPU). */
ulisse_status ulisse_kmv_f64(ulisse_ctx *ctx, const double *psi, int which, const double *V,
                             int R, double *U);

/*
 * K V for callers that cannot allocate device memory.  The paper has no counterpart: this
 * is a deployment variant of ulisse_kmv.  Some callers must not call cudaMalloc -- for
 * example code running inside a host application that owns the device memory budget and
 * forbids allocations by the libraries it loads, or a latency-critical loop where an
 * allocation (with the device synchronisation it may imply) is not acceptable.  They can
 * still compute U = A V, A = K(psi) (which == -1) or dK/dpsi_which, with this call: it
 * creates no context and calls no cudaMalloc, cudaFree or allocating library routine.
 *   X      device, n x d float, row-major (as for ulisse_create); read only.
 *   n, d   1 <= d <= 16; see the size limit below.
 *   psi    host, d + 2 doubles.   which: -1 or 0 <= which < d + 2.
 *   V      device, n x R column-major (leading dimension n), 1 <= R <= 32.
 *   U      device, n x R column-major output; must not overlap V.
 *   stream cudaStream_t (as void*) the work is ordered on; the call is asynchronous.
 * Scratch: one static device array of 64 MiB (reserved on every GPU that loads the
 * library, until the process exits) holds the prescaled inputs, a zero-padded copy of V,
 * the split partial sums and the counters.  Size limit: (n rounded up to a multiple of
 * 64) x (d rounded up to 2, 4, 8 or 16, plus R) floats must fit in 16 MiB (for d = 8 and
 * R = 17, n <= 167,000); larger requests return ULISSE_ERR_ARG without touching the GPU.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current); make that first call before any stream capture.  Do not
 * capture this call in a CUDA graph at all: psi is copied from (possibly pageable) host
 * memory when the call is made, and a captured copy would read the host buffer again at each
 * replay.
 * All calls share the array: each call clears the parts that must start at zero, but two
 * calls whose GPU work overlaps (different streams, or different host threads) race on it
 * and may return wrong results.  Serialise them.
 * The split of the j range is planned for the SMs whose partial sums fit the array (about
 * 48 MiB / 2 MiB per SM, so ~23 SMs' worth of splits), fewer than ulisse_kmv would use: for
 * small and medium n the call runs below ulisse_kmv's throughput.
 * Errors: ULISSE_ERR_ARG (null pointer, sizes out of range or too large, non-finite psi),
 * ULISSE_ERR_CUDA (no device, or a launch or copy failed).  The call returns before the GPU
 * work ends, so a bounded device wait that runs out (after about a second, i.e. when the GPU
 * is stalled) is not in its return value: the kernel records it in the array's status word
 * and U is then undefined.  ulisse_kmv_noalloc_status reads that word back.
 */
ulisse_status ulisse_kmv_noalloc(const float *X, long long n, int d, const double *psi,
                                 int which, const float *V, int R, float *U, void *stream);

/*
 * Outcome of the device work of the last ulisse_kmv_noalloc call on the current device.
 * Each ulisse_kmv_noalloc call clears the status word (on its stream) before its kernels;
 * this call copies the word to host memory on `stream` and synchronises that stream, so
 * pass the stream of the call being checked (or synchronise the device first).  It
 * allocates nothing.
 *   stream  cudaStream_t (as void*).
 *   status  host int: 0 = every wait ended, else the timeout flags the kernels set.
 * Returns ULISSE_OK (status 0), ULISSE_ERR_TIMEOUT (a bounded wait ran out: U of that call is
 * undefined), ULISSE_ERR_ARG (status is null), ULISSE_ERR_CUDA (no device, or the copy
 * failed).
 */
ulisse_status ulisse_kmv_noalloc_status(void *stream, int *status);

/* Per-column outcome of a solve, written to host memory when requested. */
typedef struct {
    int l;          /* early-stop iteration (first i >= 1 with ||e_i|| < q sqrt(n)); 0 = never */
    int iterations; /* CG iterations run for the column */
    int outcome;    /* ULISSE_OK, ULISSE_ERR_BREAKDOWN or ULISSE_ERR_MAXITER */
    int J0, J1;     /* accepted steps after the early stop, estimator 0 and 1 (-1 if absent) */
} ulisse_col_stats;

/*
 * ULISSE solve (Sec. 4): unbiased estimates of K(psi)^{-1} B[:, c] for every column c.
 * Each column runs Algorithm 1; after the early-stop threshold is reached at iteration l,
 * step j is kept with probability 1/w_j and reweighted by prod_{r<=j} w_r.
 *   psi       host, p doubles.
 *   B         device, n x R column-major right-hand sides, 1 <= R <= 1024.
 *   n_est     host, R ints in {1, 2}: independent estimators per column (NULL = all 1).  Two
 *             estimators share one CG run and differ only in their uniforms (Sec. 4.1).
 *   S0        device, n x R initial iterates, or NULL for zero.  A column keeps its iterate
 *             only when ||b - K s_0|| < ||b|| (decided without random draws, so the
 *             estimates stay unbiased); otherwise it starts from zero.
 *   S_est     device, n x sum(n_est) column-major: the estimators of column 0, then of
 *             column 1, ...
 *   step      counter for the random draws (uniforms for column c, estimator t, step j come
 *             from Philox counter (j, c, step, 2 | t << 8)).
 *   stats     host, R entries, or NULL.
 * Synchronises the stream.  Returns ULISSE_ERR_BREAKDOWN / ULISSE_ERR_MAXITER if any column
 * ended that way (all outputs are still written).
 */
ulisse_status ulisse_solve(ulisse_ctx *ctx, const double *psi, const float *B, int R,
                           const int *n_est, const float *S0, float *S_est,
                           unsigned long long step, ulisse_col_stats *stats);

/*
 * Unbiased gradient estimate g~ of log p(y | theta) with respect to psi
 * (Eq. gradient:unbiased):
 *     g~_i = 1/2 a1^T dK_i a2 - 1/(2 N_r) sum_j z_j^T dK_i r_j
 * with a1, a2 two independent ULISSE estimates of K^{-1} y from one CG run (Sec. 4.1), z_j
 * the ULISSE estimate of K^{-1} r_j, and probes r_j drawn for epoch step / probe_refresh
 * (probe column j >= 1, element i from Philox counter (i, j, epoch, 1)).
 *   psi   host, p doubles.   g  host, p doubles (output).   stats: host, 1 + N_r, or NULL.
 * The sums over covariance entries are the fused pass of ulisse_dk_bilinear (same precision
 * rules).  Synchronises the stream.
 */
ulisse_status ulisse_grad(ulisse_ctx *ctx, const double *psi, unsigned long long step,
                          double *g, ulisse_col_stats *stats);

/*
 * Posterior predictive for new inputs at parameters psi (Sec. 2, Eq. monte:carlo:integration):
 *     p(y*_j | y, psi) = N(mean[j], var[j]),
 *     mean[j] = k*_j^T K^{-1} y,   var[j] = sigma^2 + lambda - k*_j^T K^{-1} k*_j,
 * k*_j = k_s(X, x*_j) the signal covariance between the training inputs and x*_j (var is
 * that of a new noisy label; subtract lambda for the latent function).  K^{-1} y and, when
 * var is requested, K^{-1} k*_j for every j come from one solve of the context's solver
 * (configuration, precision and step as for ulisse_solve): with q > 0 they are ULISSE's
 * unbiased estimates, so mean and the k*^T K^{-1} k* term are unbiased; with q = 0 every
 * column runs to its convergence threshold and the result is the exact predictive up to it.
 * Averaging N(mean, var) over posterior samples psi^(i) is the Monte Carlo estimate of the
 * predictive distribution (paper_1501_05427_gb300.sampler.posterior_predictive).
 *   psi    host, d + 2 doubles.
 *   Xs     device, m x d row-major float test inputs.  m >= 1; m <= 1023 when var != NULL.
 *   step   counter for the solver's random draws.
 *   mean   device, m floats (output).   var  device, m floats (output), or NULL.
 * Synchronises the stream.  Returns ULISSE_ERR_MAXITER / ULISSE_ERR_BREAKDOWN as ulisse_solve
 * does (the outputs are still written).
 */
ulisse_status ulisse_predict(ulisse_ctx *ctx, const double *psi, const float *Xs, long long m,
                             unsigned long long step, float *mean, float *var);

/*
 * The fused gradient pass on its own (Eq. gradient:unbiased, Sec. 4.1): for every parameter
 * i = 0..d+1 (psi order: log l_1..log l_d, log sigma^2, log lambda),
 *     out[i] = sum_{m < M} scale[m] a_m^T (dK/dpsi_i) b_m,
 * dK/dpsi_i the covariance derivatives of ulisse_kmv (which = i).  One sweep over generated
 * covariance tiles gives all d + 2 components: with W_ab = sum_m scale[m] a_m[a] b_m[b],
 *     out[log l_k] = sum_ab k_s(a,b) W_ab (x_ak - x_bk)^2 / l_k^2,
 *     out[log sigma^2] = sum_ab k_s(a,b) W_ab,   out[log lambda] = lambda sum_a W_aa.
 * ulisse_grad evaluates this form with the solver's estimates and the probes as factors.
 *   psi    host, d + 2 doubles.
 *   A, B   device, n x M column-major float (leading dimension n), 1 <= M <= 64; read only.
 *   scale  host, M doubles, or NULL for all ones.
 *   out    host, d + 2 doubles (output).  Synchronises the context's stream.
 * Precision: FP32 contexts sum each tile in FP32 and the tiles in FP64; FP64 contexts convert
 * A and B to double and compute in FP64; mixed contexts run the pass on the tensor cores:
 * W = A B^T and the sums [S | G | H] = P [x, x^2, 1] of P = k_s o W by three BF16 products
 * each (high/low split) with FP32 accumulation, then out[log l_k] = sum_a x_ak^2 S_a -
 * 2 x_ak G_ak + H_ak in FP64 (x = x / l): each component within about 1e-4 of the scale
 * sum_m |scale[m]| |a_m|^T |dK/dpsi_i| |b_m|.
 * Works in the context's right-hand-side and estimate buffers, which every solve and gradient
 * call rewrites; the iterates kept for warm-started solves are not touched.
 * Errors: ULISSE_ERR_ARG (null, M out of range, non-finite psi or scale, batched context),
 * ULISSE_ERR_CUDA, ULISSE_ERR_TIMEOUT.
 */
ulisse_status ulisse_dk_bilinear(ulisse_ctx *ctx, const double *psi, const float *A,
                                 const float *B, int M, const double *scale, double *out);

/*
 * One SGLD step (Sec. 2.1) on psi:
 *     psi <- psi + eps_t/2 M (g~ + grad log p(psi)) + sqrt(eps_t) L xi,   L L^T = M,
 * xi ~ N(0, I_p) from Philox counter (k, 0, step, 3) by the Box-Muller transform; all
 * proposals are accepted (Sec. 2.1).
 *   psi_inout   host, p doubles, updated in place.
 *   M           host, p x p row-major symmetric positive definite, or NULL for I.
 *   prior_grad  host, p doubles of grad_psi log p(psi), or NULL for a flat prior in psi.
 *   g_out       host, p doubles (the g~ used), or NULL.
 * Synchronises the stream.  ULISSE_ERR_ARG if M is not positive definite.
 */
ulisse_status ulisse_sgld_step(ulisse_ctx *ctx, double *psi_inout, double eps_t,
                               const double *M, const double *prior_grad,
                               unsigned long long step, double *g_out);

/*
 * n_steps SGLD steps with psi resident on the device (no host round trip per step):
 *   psi_dev     device, p doubles, updated in place.
 *   eps_dev     device, n_steps doubles: step size of each step.
 *   M           host, p x p or NULL (fixed for the run).  prior_grad: host p or NULL (fixed).
 *   trace_dev   device, n_steps x p doubles (psi after each step), or NULL.
 *   step0       step counter of the first step.
 * Asynchronous with respect to the host except for one status read at the end.
 */
ulisse_status ulisse_sgld_chain(ulisse_ctx *ctx, double *psi_dev, const double *eps_dev,
                                int n_steps, const double *M, const double *prior_grad,
                                unsigned long long step0, double *trace_dev);

/* Work counters since creation (each output pointer may be NULL):
 *   mvp_rounds        K V products issued by the solver (one per batched CG iteration,
 *                     covering every live column at once),
 *   entry_rhs         generated covariance entries times right-hand sides (K V and the
 *                     gradient pass: n^2 R per product),
 *   kernel_launches   CUDA kernels this library launched. */
ulisse_status ulisse_counters(const ulisse_ctx *ctx, long long *mvp_rounds,
                              double *entry_rhs, long long *kernel_launches);

/* Device-time accounting of the two O(n^2) kernels, from CUDA events recorded on the
 * context's stream around every launch while enabled.  Algorithmic FLOPs per launch:
 *   K V:       n^2 (3d + 2 + 2R)   (d differences and d squares-and-adds, the exponent's
 *                                   FMA and exp, R multiply-adds; the exp counted as 1)
 *   gradient:  n^2 (5d + 4 + 2M)   (M = 1 + N_r rank of the bilinear form) */
typedef struct {
    long long kmv_launches;
    double kmv_ms;
    double kmv_flop;
    long long grad_launches;
    double grad_ms;
    double grad_flop;
} ulisse_profile;

/* Enable (1) or disable (0) the event timing above; enabling resets the totals. */
ulisse_status ulisse_profile_enable(ulisse_ctx *ctx, int enable);

/* Totals since enabling (synchronises the stream); reset != 0 clears them afterwards. */
ulisse_status ulisse_profile_read(ulisse_ctx *ctx, ulisse_profile *out, int reset);

/*
 * Learned warm start for the K s = y solve.  Algorithm 1 starts from any iterate s_0, and
 * the ULISSE estimate stays unbiased for K^{-1} y for every s_0 fixed before the step's
 * random draws, so a good guess shortens the y solve without biasing the gradient.  The
 * guess is s_0 = K_s(X, Z) c with Z a seeded subset of the inputs (anchors) and
 * c = MLP(psi): psi standardised, two tanh layers of `hidden` units, a linear output of
 * n_anchors.  The network is trained on the GPU on data the chain records as it runs:
 * at each recorded step's parameters psi_t, n_rows rows I_t drawn uniformly (with
 * replacement, from a counter-based stream), y at those rows and
 * M_t = K(X_{I_t}, X; psi_t) K_s(X, Z; psi_t), so that y_{I_t} - M_t c is the solve's
 * initial residual y - K s_0 on those rows.  Loss
 * 1/T sum_t (||y_{I_t} - M_t c_t||^2 / m + ridge ||c_t||^2), Adam.  Until the first
 * training call c = 0 (s_0 = 0, the method without warm start); a solve keeps s_0 only
 * when it lowers the residual norm below ||y|| (see ulisse_solve).
 * Device memory: max_pairs * n_rows * n_anchors floats for the recorded M_t, plus
 * n * n_anchors floats of scratch.
 */
typedef struct {
    int n_anchors;           /* A <= n (512 in the paper-scale configuration) */
    int hidden;              /* H (256) */
    int n_rows;              /* m rows per recorded pair, 1..8192 */
    int max_pairs;           /* capacity of the pair buffer (a ring: the newest are kept) */
    unsigned long long seed; /* anchors, rows, initial weights and minibatches */
    double ridge;            /* rho >= 0, weight of ||c||^2 in the loss */
} ulisse_ws_config;

/* Weights, sampling and recorded pairs, copied to caller-provided HOST buffers (any
 * pointer may be NULL).  Weights are flattened W1 (p x H), b1, W2 (H x H), b2, W3 (H x A),
 * b3, each matrix row-major with inputs along rows. */
typedef struct {
    float *weights;          /* n_params */
    int *anchors;            /* A row indices of X */
    int *pair_rows;          /* max_pairs x m row indices of X */
    float *mu, *sd;          /* p: input standardisation */
    float *pair_psi;         /* max_pairs x p */
    int n_pairs;             /* out: pairs recorded (<= max_pairs) */
    long long n_params;      /* out */
} ulisse_ws_state;

/* Allocate the warm start (anchors, rows and weights from cfg->seed; W3 = b3 = 0). */
ulisse_status ulisse_ws_init(ulisse_ctx *ctx, const ulisse_ws_config *cfg);
/* record != 0: every gradient / SGLD step appends a pair; use != 0: solves of K s = y
 * start from the warm start (only after the first training call). */
ulisse_status ulisse_ws_set(ulisse_ctx *ctx, int record, int use);
/* Train on the recorded pairs.  First the pooled normal equations of the loss for a
 * constant c, G c = g with G = sum_t M_t^T M_t / (T m) + ridge I, are formed and G = L L^T
 * is factorised on the GPU (FP64); the network restarts from that least-squares constant
 * (W3 = 0, b3 = G^{-1} g) with its output layer whitened, W3 = W~3 L^{-1}, so that the loss
 * is well conditioned in the coordinates Adam updates.  Then `steps` Adam steps (learning
 * rate lr, moments restarted) on minibatches of `batch` (<= max_pairs) pairs.  Once eight
 * or more pairs are recorded, every eighth is held out: minibatches skip it, the held-out
 * loss is evaluated every 25 steps, and the weights with the lowest held-out loss (the
 * pooled start included) are kept.  *loss (may be NULL) receives that held-out loss, or the
 * last minibatch loss without held-out pairs (0 when steps == 0).  batch and lr are not
 * checked when steps == 0.  Refreshes the BF16 inference weights.
 * Errors: ULISSE_ERR_BREAKDOWN if G is not numerically positive definite (raise ridge). */
ulisse_status ulisse_ws_train(ulisse_ctx *ctx, int steps, int batch, double lr, double *loss);
/* Loss over all recorded pairs and its gradient (host, n_params floats) for the current
 * weights: the quantity the training kernels descend, exposed for checking. */
ulisse_status ulisse_ws_loss_grad(ulisse_ctx *ctx, double *loss, float *grad);
ulisse_status ulisse_ws_export(ulisse_ctx *ctx, ulisse_ws_state *out);
/* s_0 = K_s(X, Z) MLP(psi) into x0 (device, n floats); bf16 != 0 uses the inference
 * weights. */
ulisse_status ulisse_ws_x0(ulisse_ctx *ctx, const double *psi, int bf16, float *x0);

/*
 * Batched contexts: many independent GP problems of uneven size (Sec. 2's problem, once per
 * data set), advanced together.  Each problem b keeps its own data, parameters psi_b
 * (p_b = d_b + 2) and solver state, and draws from its own random streams (the generator
 * key is cfg->seed + b, so problem b reproduces a single context created with that seed).
 * The O(n^2) passes of all problems run as one launch each: every CG round's covariance
 * products over all live columns of all problems, and the fused gradient sweep.
 *   ULISSE_PREC_FP32: persistent SIMT launches over (problem, 256-row block) items, longest
 *     rows first;
 *   ULISSE_PREC_MIXED: the tensor-core products (as ulisse_config.tc_cross_term = 2, the
 *     column term added in the epilogue for every d) over (problem, 128-row block, split)
 *     items, and the tensor-core gradient pass, one launch per padded input width (2, 4, 8).
 * Parameters and gradients are packed: problem b's p_b values follow problem b-1's.
 * Batched contexts take n_probes <= 16 (warm_start_probes applies to every problem), and
 * accept only the ulisse_batch_* calls (plus ulisse_set_graph, counters and destroy); the
 * single-problem calls return ULISSE_ERR_ARG on them.
 *
 *   n_problems  1 .. 4096.   n, d: host arrays of n_problems sizes (1 <= d_b <= 8).
 *   X, y        host arrays of n_problems DEVICE pointers (row-major n_b x d_b, and n_b);
 *               copied into the context.
 * Errors: ULISSE_ERR_ARG (bad sizes, null pointers, precision FP64), ULISSE_ERR_NOMEM.
 */
ulisse_status ulisse_create_batched(ulisse_ctx **out, int n_problems, const long long *n,
                                    const int *d, const float *const *X, const float *const *y,
                                    const ulisse_config *cfg, void *stream);

/* Number of problems and total packed parameter count (n_params may be NULL). */
ulisse_status ulisse_batch_size(const ulisse_ctx *ctx, int *n_problems, int *n_params);

/* U_b = K_b(psi_b) V_b for every problem in one persistent launch.
 *   psi  host, packed parameters.  V, U: host arrays of n_problems DEVICE pointers, each
 *   an n_b x R column-major block (leading dimension n_b); 1 <= R <= 32. */
ulisse_status ulisse_batch_kmv(ulisse_ctx *ctx, const double *psi, const float *const *V, int R,
                               float *const *U);

/* Unbiased gradient estimates of every problem (as ulisse_grad, per problem).
 *   psi, g  host, packed.   stats: NULL or n_problems x (1 + n_probes) entries. */
ulisse_status ulisse_batch_grad(ulisse_ctx *ctx, const double *psi, unsigned long long step,
                                double *g, ulisse_col_stats *stats);

/* One SGLD step of every problem (as ulisse_sgld_step with M = I and a flat prior).
 *   psi_inout host, packed; g_out NULL or host, packed. */
ulisse_status ulisse_batch_sgld_step(ulisse_ctx *ctx, double *psi_inout, double eps_t,
                                     unsigned long long step, double *g_out);

/* n_steps SGLD steps of every problem with the packed parameters resident on the device.
 *   psi_dev   device, packed parameters (in place).
 *   eps_dev   device, n_steps step sizes.   step0: step number of the first step.
 *   trace_dev device, NULL or n_steps x n_params (packed parameters after each step).
 * With the graph enabled (ulisse_set_graph, the default) each step is ONE launch of a CUDA
 * graph holding the whole batched step: every problem's prescale, probes and CG start, the
 * round loop as a conditional WHILE node (one batched compaction, the persistent K V over
 * all live columns of all problems with its compiled width chosen by a SWITCH node, three
 * batched CG launches), the persistent gradient sweep and the updates.  The host loop runs
 * the same launches and gives the same results. */
ulisse_status ulisse_batch_sgld_chain(ulisse_ctx *ctx, double *psi_dev, const double *eps_dev,
                                      int n_steps, unsigned long long step0, double *trace_dev);

/* ulisse_sgld_chain runs each step as ONE launch of a CUDA graph (enable != 0, the default)
 * or from the host loop (0).  The graph holds the whole step: prescale, probes, the CG +
 * ULISSE loop as a conditional WHILE node (its body compacts the live columns on the device
 * and a SWITCH node picks the branch compiled for that many live columns), the fused
 * gradient and the update; the step number, step size and trace slot are read from the
 * device.  Both forms launch the same kernels with the same arguments and give the same
 * results.  The chain uses the host loop while the event timing (ulisse_profile_enable) is
 * on or warm-start pairs are recorded.  The graph is captured on first use and again after
 * a call that reallocated the context's buffers. */
ulisse_status ulisse_set_graph(ulisse_ctx *ctx, int enable);

/* Autotuned K V launch configuration for one live column count. */
typedef struct {
    int live_cols;           /* columns of the product */
    int width;               /* compiled column count (SIMT) or MMA N (tensor cores) used */
    int rows_per_thread;     /* SIMT rows per thread (0 on the tensor-core path) */
    int nsplit;              /* j-range split count forced (0: the launch plan's choice) */
    float ms;                /* median time of the chosen configuration */
    float ms_default;        /* median time of the untuned configuration */
    int cross_term;          /* tensor-core path: where the cross term is formed (1 FP32
                                FMAs, 2 tensor cores; see ulisse_config.tc_cross_term);
                                0 on the SIMT path */
} ulisse_tune_entry;

/* Time, for every live column count 1..max_cols (<= 32), the candidate K V configurations
 * on this context's data -- compiled column counts, rows per thread (SIMT), where the cross
 * term is formed (tensor-core path), j-range splits -- with
 * CUDA events on the context's stream (median of `reps` launches each), and use the
 * fastest from then on (the untuned choice is always a candidate).  psi: host, the
 * parameters to tune at (they set the data layout only; any valid psi).  out: NULL or
 * max_cols entries.  The tuning launches are not counted as the method's work.  Results
 * change only in the summation order of the split j range (the last bits).
 * FP32 and mixed contexts. */
ulisse_status ulisse_autotune(ulisse_ctx *ctx, const double *psi, int max_cols, int reps,
                              ulisse_tune_entry *out);

/* Install a K V launch table, e.g. one that ulisse_autotune returned in an earlier run on the
 * same device and problem size, so that a new context skips the tuning (the paper has no
 * counterpart).  table: host, n entries (1 <= n <= 32); entry k is used for products of
 * k + 1 columns.  Per entry (live_cols, ms and ms_default are ignored):
 *   width: k + 1 .. 64; the smallest compiled column count at least this wide is used
 *          (tensor cores: the MMA N 16, 32 or 64; SIMT: up to 32);
 *   rows_per_thread: SIMT 2 or 4 (ignored on the tensor-core path);
 *   nsplit: 0 (the launch plan's choice) or 1 .. 64 (the j range is still split further
 *           where a tensor-core CTA would exceed its accumulation bound);
 *   cross_term: tensor-core path 1 or 2, SIMT path 0.
 * Column counts beyond n keep the untuned choice.  Results differ from another table's only
 * in the summation order of the split j range.  n = 0 (table may be NULL) clears the table.
 * Errors: ULISSE_ERR_ARG (FP64 or batched context, n out of range, an invalid entry; the
 * table in use is then unchanged). */
ulisse_status ulisse_set_tune(ulisse_ctx *ctx, const ulisse_tune_entry *table, int n);

/*
 * Self-test of the failure path (no GPU fault is involved): one CTA waits on an mbarrier
 * that nothing completes.  The wait gives up after about half a second (2^30 SM cycles), the
 * kernel records the timeout in the context's status word as every kernel of the library
 * does when one of its bounded waits runs out, and this call reports it as any call would:
 * ULISSE_ERR_TIMEOUT (after zeroing the context's split counters, as every timeout does).
 * The context stays usable.  Synchronises the stream.
 */
ulisse_status ulisse_selftest_wait_timeout(ulisse_ctx *ctx);

/*
 * Device calibration (the paper has no counterpart; used for roofline reports): the
 * throughput of the base-2 exponential (ex2.approx.ftz.f32), the one operation every
 * generated covariance entry needs on the CUDA cores when the tensor cores form the rest.
 * Runs independent exponentials on every SM of the current device (all resident threads,
 * 16 in flight per thread) on `stream` (NULL: the legacy default stream), `reps` timed
 * launches of about a millisecond each with CUDA events, and reports the best.
 *   reps       1..1000.
 *   ex2_per_s  host, out: exponentials per second of the best launch.
 *   best_ms    host, out (may be NULL): duration of that launch.
 * Needs no context and allocates nothing.  Synchronises the stream.
 * Errors: ULISSE_ERR_ARG (ex2_per_s NULL or reps out of range), ULISSE_ERR_CUDA.
 */
ulisse_status ulisse_measure_ex2_rate(void *stream, int reps, double *ex2_per_s,
                                      double *best_ms);

/* Message for the last failing call on ctx (or on creation if ctx is NULL). */
const char *ulisse_last_error(const ulisse_ctx *ctx);

/* Free the context and all of its device memory.  NULL is allowed. */
void ulisse_destroy(ulisse_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* ULISSE_H */
