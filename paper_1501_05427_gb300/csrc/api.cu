// C ABI of libulisse (include/ulisse.h): context management and the host-side ordering of
// the kernels for one K V product, one ULISSE solve, one gradient and one SGLD step.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ulisse.h"
#include "solver_kernels.cuh"
#include "pcg_kernels.cuh"
#include "predict.cuh"
#include "warm_start.cuh"
#include "batch.cuh"

using namespace ulisse;

struct ulisse_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 1;
  long long n = 0, ldn = 0;
  int d = 0, DP = 0;
  ulisse_config cfg{};
  bool f64 = false;
  bool mixed = false;         // tensor-core K V (tcgen05), FP32 vectors
  size_t esz = 4;
  long long ld128 = 0;        // rows of the tensor-core operand images (multiple of 128)
  float* bneg = nullptr;      // -log2(e)/2 |x^|^2 per input (tensor-core path)
  void *Vt_hi = nullptr, *Vt_lo = nullptr;
  void *Gt_hi = nullptr, *Gt_lo = nullptr;   // packed operands of the tensor-core gradient
  float *Xt_hi = nullptr, *Xt_lo = nullptr;  // TF32 images A | B (tensor-core cross term)

  float* X = nullptr;         // raw inputs, n x d row-major
  void* y = nullptr;          // labels, ldn (element type T)
  void* xhat = nullptr;       // prescaled inputs, ldn x DP
  DevParams* params = nullptr;
  double* psi_dev = nullptr;  // kMaxP

  int cap = 0;                // column capacity of B, S, E, D, KD
  int cap_est = 0;            // column capacity of SE
  void *B = nullptr, *S = nullptr, *E = nullptr, *D = nullptr, *KD = nullptr, *SE = nullptr;
  ColState* st = nullptr;
  ColState* st_next = nullptr;
  double* part1 = nullptr;     // CG partial dot products, cap x kMaxCgChunks each
  double* part2 = nullptr;
  int* live = nullptr;
  int* n_live_dev = nullptr;
  int* iota = nullptr;        // 0, 1, 2, ... (cap entries)
  int* h_n_live = nullptr;    // pinned

  void* partials = nullptr;
  size_t partials_bytes = 0;
  int* counters = nullptr;
  int counters_len = 0;

  double* gpart = nullptr;
  size_t gpart_len = 0;
  int* gcounter = nullptr;
  double* g_dev = nullptr;
  void* sa_dev = nullptr;     // gradient scales (T), kMaxM
  int* amap = nullptr;        // gradient left-factor columns
  int* bmap = nullptr;        // gradient right-factor columns
  int grad_nr = -1;           // probe count the maps were built for
  int* q_map = nullptr;       // ulisse_dk_bilinear: identity column map (kMaxM)
  void* q_sa = nullptr;       // ulisse_dk_bilinear: scales (T), kMaxM

  double* M_dev = nullptr;
  double* prior_dev = nullptr;
  int* status_dev = nullptr;
  int* h_status = nullptr;    // pinned

  long long mvp_rounds = 0;
  double entry_rhs = 0.0;
  long long launches = 0;
  std::string err;

  // learned warm start (ulisse_ws_*)
  bool ws_ready = false, ws_record = false, ws_use = false, ws_trained = false;
  bool ws_standardized = false;
  WsBuffers wsb{};
  int ws_pairs = 0, ws_next = 0, ws_t = 0, ws_loss_blocks = 0;
  unsigned long long ws_seed = 0, ws_batches = 0;
  float* ws_c = nullptr;
  std::vector<void*> ws_allocs;

  int meta_grad_R = -1;       // column count the gradient's column metadata was uploaded for
  int* warm_valid = nullptr;  // device: Sbest holds the iterates of a finished step's solve
  void* Sbest = nullptr;      // cap columns right after S (one allocation), see CgArgs
  int* warm_map = nullptr;    // K s_0 column maps of warm-started solves (2 x cap): S/Sbest

  // autotuned K V launch configuration per live column count (ulisse_autotune); index
  // nl - 1, empty until tuned
  struct KmvTune { int width, tm, nsplit; float ms, ms_default; int cross; };
  std::vector<KmvTune> tune;
  int last_nsplit = 1;        // split count of the last K V launch (or plan)

  // CUDA graph of one SGLD step (ulisse_sgld_chain)
  bool planning = false;      // launch helpers only size their scratch
  bool capturing = false;     // launch helpers are being captured: no host-side counting
  bool graph_enabled = true;
  cudaStream_t cap_stream = nullptr, cap_stream2 = nullptr;
  cudaGraph_t step_graph = nullptr;
  cudaGraphExec_t step_exec = nullptr;
  long long graph_key = -1;   // configuration the graph was captured for
  ChainSlot* chain = nullptr; // device
  long long* gstat = nullptr; // device: rounds, sum of live columns, launches, rounds this step
  long long* h_gstat = nullptr;  // pinned copy
  double* eps_one = nullptr;  // device step size of a single graph step
  bool m_identity = false;    // M_dev holds the identity (the graph's default M)
  bool prior_zero = false;    // prior_dev holds zeros
  long long graph_launches_fixed = 0;  // kernel launches per step outside the CG loop
  double graph_entries_fixed = 0.0;    // entries x right-hand sides per step outside the loop
  long long graph_rounds_fixed = 0;

  // batched context (ulisse_create_batched): one sub-context per problem
  bool batched = false;
  std::vector<ulisse_ctx*> subs;
  std::vector<int> sub_p_off;      // offset of each problem's parameters in the packed vector
  BatchItem* b_items = nullptr;
  int b_n_items = 0;
  BatchKmvDesc* b_kdesc = nullptr;
  BatchKmvDesc* b_kdesc0 = nullptr;    // warm-started solves: the products K s_0 of all problems
  BatchGradDesc* b_gdesc = nullptr;
  int* b_queue = nullptr;
  int* b_nlive = nullptr;          // device, one live count per problem
  int* b_h_nlive = nullptr;        // pinned
  int* b_rcount = nullptr;         // device, column count of ulisse_batch_kmv per problem
  int* b_h_status = nullptr;       // pinned, one status word per problem
  double* b_gpart = nullptr;       // n_items x kMaxP
  double* b_g = nullptr;           // problems x kMaxP
  CgArgs<float>* b_cgargs = nullptr;   // device, one per problem (batched CG launches)
  BatchCgProb* b_cgprob = nullptr;     // device, one per problem (batched compaction)
  int* b_rmax = nullptr;           // device: largest live count of the round
  int* b_h_rmax = nullptr;         // pinned
  double* b_psi = nullptr;         // device: packed parameters of all problems
  int b_np = 0;                    // packed parameter count
  int b_maxch = 1;                 // largest chunk count of the batched CG launches
  // mixed-precision batches: the tensor-core K V over (problem, 128-row block, split) items
  bool tc_no_aug = false;          // sub-context of a mixed batch: rows packed without b_j
  int4* b_tc_items = nullptr;
  int b_tc_n_items = 0;
  void* b_tc_args = nullptr;       // 3 x problems kernel arguments: rounds, K s_0, batch K V
  float* b_tc_part = nullptr;      // split partial sums of all problems
  int* b_tc_cnt = nullptr;         // split counters of all problems (zero between launches)
  std::vector<int> b_tc_nsplit;
  std::vector<size_t> b_tc_part_off, b_tc_cnt_off;
  // ... and the tensor-core gradient pass, one launch per padded input width (group)
  std::vector<std::vector<int>> b_gt_groups;   // problem indices of each width
  std::vector<int> b_gt_dp, b_gt_item_off, b_gt_item_n;
  std::vector<int> b_gt_nsplit;                // per problem
  std::vector<size_t> b_gt_part_off;           // per problem, doubles
  int4* b_gt_items = nullptr;
  void* b_gt_args = nullptr;                   // problems in group order
  double* b_gt_part = nullptr;
  int* b_gt_cnt = nullptr;                     // one counter per problem

  // posterior predictive (ulisse_predict): the prescaled test inputs
  void* pred_xs = nullptr;
  size_t pred_xs_bytes = 0;

  // preconditioned CG (cfg.pcg_delta > 0): Z, X, Rr, P, KP (pcg_cap columns each)
  void* pcg_buf = nullptr;
  int pcg_cap = 0;
  PcgAux* pcg_aux = nullptr;
  int* pcg_live = nullptr;

  // event timing of the O(n^2) kernels (ulisse_profile_enable)
  bool prof = false;
  struct Pending { int kind; cudaEvent_t a, b; double flop; };
  std::vector<Pending> pending;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> free_events;
  ulisse_profile totals{};
};

static thread_local std::string g_create_error;
static constexpr int kMaxCgChunks = 64;

#define CK(call)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);                 \
      return e_ == cudaErrorMemoryAllocation ? ULISSE_ERR_NOMEM : ULISSE_ERR_CUDA;   \
    }                                                                                \
  } while (0)

#define CKS(expr)                          \
  do {                                     \
    ulisse_status s_ = (expr);             \
    if (s_ != ULISSE_OK) return s_;        \
  } while (0)

static ulisse_status fail(ulisse_ctx* ctx, ulisse_status s, const std::string& msg) {
  if (ctx) ctx->err = msg;
  else g_create_error = msg;
  return s;
}

// Events around one O(n^2) kernel launch (kind 0: K V, 1: gradient).
static void prof_begin(ulisse_ctx* ctx, cudaEvent_t* a, cudaEvent_t* b) {
  if (!ctx->prof) return;
  if (ctx->free_events.empty()) {
    cudaEvent_t x, y;
    cudaEventCreate(&x);
    cudaEventCreate(&y);
    ctx->free_events.push_back({x, y});
  }
  *a = ctx->free_events.back().first;
  *b = ctx->free_events.back().second;
  ctx->free_events.pop_back();
  cudaEventRecord(*a, ctx->stream);
}

static void prof_end(ulisse_ctx* ctx, int kind, cudaEvent_t a, cudaEvent_t b, double flop) {
  if (!ctx->prof) return;
  cudaEventRecord(b, ctx->stream);
  ctx->pending.push_back({kind, a, b, flop});
}

// Fold completed event pairs into the totals (call after a stream synchronisation).
static void prof_drain(ulisse_ctx* ctx) {
  for (auto& p : ctx->pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    if (p.kind == 0) {
      ctx->totals.kmv_launches++;
      ctx->totals.kmv_ms += ms;
      ctx->totals.kmv_flop += p.flop;
    } else {
      ctx->totals.grad_launches++;
      ctx->totals.grad_ms += ms;
      ctx->totals.grad_flop += p.flop;
    }
    ctx->free_events.push_back({p.a, p.b});
  }
  ctx->pending.clear();
}

static int dp_for(int d) { return d <= 2 ? 2 : d <= 4 ? 4 : d <= 8 ? 8 : 16; }

static ulisse_status dev_alloc(ulisse_ctx* ctx, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return ULISSE_OK;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(ctx, ULISSE_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  e = cudaMemsetAsync(*p, 0, bytes, ctx->stream);
  if (e != cudaSuccess) return fail(ctx, ULISSE_ERR_CUDA, cudaGetErrorString(e));
  return ULISSE_OK;
}

static void dev_free(void*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

// Column buffers for at least R solver columns and R_est estimate columns.
static ulisse_status ensure_columns(ulisse_ctx* ctx, int R, int R_est) {
  if (R <= ctx->cap && R_est <= ctx->cap_est) return ULISSE_OK;
  ctx->graph_key = -1;   // a captured step graph holds the old buffers
  const int cap = std::max(R, ctx->cap), cap_est = std::max(R_est, ctx->cap_est);
  CK(cudaStreamSynchronize(ctx->stream));
  for (void** p : {&ctx->B, &ctx->S, &ctx->E, &ctx->D, &ctx->KD, &ctx->SE}) dev_free(*p);
  dev_free(reinterpret_cast<void*&>(ctx->st));
  dev_free(reinterpret_cast<void*&>(ctx->st_next));
  dev_free(reinterpret_cast<void*&>(ctx->part1));
  dev_free(reinterpret_cast<void*&>(ctx->part2));
  dev_free(reinterpret_cast<void*&>(ctx->live));
  dev_free(reinterpret_cast<void*&>(ctx->iota));
  dev_free(reinterpret_cast<void*&>(ctx->warm_map));
  const size_t col = (size_t)ctx->ldn * ctx->esz;
  for (void** p : {&ctx->B, &ctx->E, &ctx->D, &ctx->KD})
    CKS(dev_alloc(ctx, p, col * cap));
  CKS(dev_alloc(ctx, &ctx->S, col * cap * 2));   // S, then Sbest
  ctx->Sbest = (char*)ctx->S + col * cap;
  CKS(dev_alloc(ctx, &ctx->SE, col * cap_est));
  CKS(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->st), sizeof(ColState) * cap));
  CKS(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->st_next), sizeof(ColState) * cap));
  CKS(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->part1), sizeof(double) * cap * kMaxCgChunks));
  CKS(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->part2), sizeof(double) * cap * kMaxCgChunks));
  CKS(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->live), sizeof(int) * cap));
  const int ni = std::max(cap, cap_est);
  CKS(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->iota), sizeof(int) * ni));
  std::vector<int> io(ni);
  for (int i = 0; i < ni; ++i) io[i] = i;
  CK(cudaMemcpyAsync(ctx->iota, io.data(), sizeof(int) * ni, cudaMemcpyHostToDevice,
                     ctx->stream));
  // warm-started solves read s_0 from Sbest (column cap + c); with the learned warm start
  // column 0 comes from S
  CKS(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->warm_map), sizeof(int) * 2 * cap));
  std::vector<int> wm(2 * cap);
  for (int c = 0; c < cap; ++c) wm[c] = wm[cap + c] = cap + c;
  wm[cap] = 0;
  CK(cudaMemcpyAsync(ctx->warm_map, wm.data(), sizeof(int) * 2 * cap, cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->cap = cap;
  ctx->cap_est = cap_est;
  return ULISSE_OK;
}

static bool finite_psi(const double* psi, int p) {
  for (int i = 0; i < p; ++i)
    if (!std::isfinite(psi[i])) return false;
  return true;
}

// psi (host) -> device, then the prescale kernel (a1).
static ulisse_status set_psi_host(ulisse_ctx* ctx, const double* psi) {
  const int p = ctx->d + 2;
  if (!psi || !finite_psi(psi, p)) return fail(ctx, ULISSE_ERR_ARG, "psi is null or not finite");
  CK(cudaMemcpyAsync(ctx->psi_dev, psi, sizeof(double) * p, cudaMemcpyHostToDevice,
                     ctx->stream));
  return ULISSE_OK;
}

static ulisse_status prescale(ulisse_ctx* ctx) {
  const int blocks = (int)std::min<long long>((ctx->n + 255) / 256, 4LL * ctx->num_sms);
  if (ctx->f64)
    prescale_kernel<double><<<blocks, 256, 0, ctx->stream>>>(
        ctx->psi_dev, ctx->X, (double*)ctx->xhat, ctx->n, ctx->d, ctx->DP, ctx->params);
  else
    prescale_kernel<float><<<blocks, 256, 0, ctx->stream>>>(
        ctx->psi_dev, ctx->X, (float*)ctx->xhat, ctx->n, ctx->d, ctx->DP, ctx->params);
  CK(cudaGetLastError());
  if (!ctx->capturing) ctx->launches++;
  if (ctx->mixed) {
    CK(launch_prescale_tc((const float*)ctx->xhat, ctx->DP, ctx->d, ctx->n, ctx->ld128,
                          ctx->bneg, ctx->num_sms, ctx->stream));
    CK(launch_pack_x_tf32((const float*)ctx->xhat, ctx->bneg, ctx->params, ctx->DP, ctx->n,
                          ctx->ld128, ctx->Xt_hi, ctx->Xt_lo, ctx->ld128 * 24, ctx->num_sms,
                          ctx->stream, !ctx->tc_no_aug));
    if (!ctx->capturing) ctx->launches += 2;
  }
  return ULISSE_OK;
}

// U[:, umap[r]] = A V[:, vmap[r]] for r < R (chunks of kMaxRChunk columns per launch).
// Grow the split-j scratch of the K V kernels to at least the given sizes.
static ulisse_status grow_kmv_scratch(ulisse_ctx* ctx, size_t need_bytes, int need_counters) {
  if (need_bytes <= ctx->partials_bytes && need_counters <= ctx->counters_len) return ULISSE_OK;
  ctx->graph_key = -1;
  CK(cudaStreamSynchronize(ctx->stream));
  if (need_bytes > ctx->partials_bytes) {
    dev_free(ctx->partials);
    ctx->partials_bytes = 0;
    CKS(dev_alloc(ctx, &ctx->partials, need_bytes));
    ctx->partials_bytes = need_bytes;
  }
  if (need_counters > ctx->counters_len) {
    dev_free(reinterpret_cast<void*&>(ctx->counters));
    ctx->counters_len = 0;
    CKS(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->counters), sizeof(int) * need_counters));
    ctx->counters_len = need_counters;
  }
  return ULISSE_OK;
}

// U[:, umap[r]] = A V[:, vmap[r]] for r < R (chunks of 64 columns per launch).
static ulisse_status run_kmv_tc(ulisse_ctx* ctx, const void* V, const int* vmap, int R, void* U,
                                const int* umap) {
  for (int c0 = 0; c0 < R; c0 += 64) {
    TcLaunch L{};
    L.xhat = (const float*)ctx->xhat;
    L.bneg = ctx->bneg;
    L.V_hi = ctx->Vt_hi;
    L.V_lo = ctx->Vt_lo;
    L.V = V;
    L.ldv = ctx->ldn;
    L.vmap = vmap + c0;
    L.R = std::min(64, R - c0);
    L.U = U;
    L.ldu = ctx->ldn;
    L.umap = umap + c0;
    L.n = ctx->n;
    L.DP = ctx->DP;
    L.params = ctx->params;
    L.status = ctx->status_dev;
    L.num_sms = ctx->num_sms;
    L.X_hi = ctx->Xt_hi;
    L.X_lo = ctx->Xt_lo;
    L.X_off = ctx->ld128 * 24;
    // where the cross term is formed: the tuned choice, else the configured one (default:
    // tensor cores)
    int cross = ctx->cfg.tc_cross_term != 0 ? ctx->cfg.tc_cross_term : kCrossTensor;
    if ((int)ctx->tune.size() >= L.R && ctx->tune[L.R - 1].width > 0) {
      L.n_min = ctx->tune[L.R - 1].width;
      L.nsplit = ctx->tune[L.R - 1].nsplit;
      if (ctx->tune[L.R - 1].cross != 0) cross = ctx->tune[L.R - 1].cross;
    }
    auto launch = [&](TcLaunch& LL) {
      return cross == kCrossTensor ? launch_kmv_tc2(LL, ctx->stream) : launch_kmv_tc(LL, ctx->stream);
    };
    if (ctx->planning) {
      L.plan_only = true;
      cudaError_t e = launch(L);
      ctx->last_nsplit = L.planned_nsplit;
      if (e != cudaSuccess)
        return fail(ctx, ULISSE_ERR_CUDA, std::string("tensor-core K V plan: ") + cudaGetErrorString(e));
      CKS(grow_kmv_scratch(ctx, L.need_partials_bytes, L.need_counters));
      continue;
    }
    for (int attempt = 0; attempt < 2; ++attempt) {
      L.partials = ctx->partials;
      L.partials_bytes = ctx->partials_bytes;
      L.counters = ctx->counters;
      L.counters_len = ctx->counters_len;
      cudaEvent_t ea = nullptr, eb = nullptr;
      prof_begin(ctx, &ea, &eb);
      cudaError_t e = launch(L);
      if (ctx->prof) {
        if (e == cudaSuccess)
          prof_end(ctx, 0, ea, eb, (double)ctx->n * ctx->n * (3.0 * ctx->d + 2.0 + 2.0 * L.R));
        else
          ctx->free_events.push_back({ea, eb});
      }
      if (e == cudaSuccess) {
        if (!ctx->capturing) ctx->launches += 2;
        break;
      }
      if (e != cudaErrorMemoryAllocation || attempt == 1 || ctx->capturing)
        return fail(ctx, ULISSE_ERR_CUDA, std::string("tensor-core K V launch: ") + cudaGetErrorString(e));
      cudaGetLastError();
      CKS(grow_kmv_scratch(ctx, L.need_partials_bytes, L.need_counters));
    }
    if (!ctx->capturing) ctx->entry_rhs += (double)ctx->n * (double)ctx->n * (double)L.R;
  }
  return ULISSE_OK;
}

static ulisse_status run_kmv(ulisse_ctx* ctx, const void* V, const int* vmap, int R, void* U,
                             const int* umap, int mode, int which) {
  if (ctx->mixed && mode == kModeK) return run_kmv_tc(ctx, V, vmap, R, U, umap);
  for (int c0 = 0; c0 < R; c0 += kMaxRChunk) {
    KmvLaunch L{};
    L.xhat = ctx->xhat;
    L.n = ctx->n;
    L.ldn = ctx->ldn;
    L.d = ctx->d;
    L.DP = ctx->DP;
    L.V = V;
    L.ldv = ctx->ldn;
    L.vmap = vmap + c0;
    L.R = std::min(kMaxRChunk, R - c0);
    L.U = U;
    L.ldu = ctx->ldn;
    L.umap = umap + c0;
    L.params = ctx->params;
    L.mode = mode;
    L.which = which;
    L.tm = ctx->cfg.kmv_rows_per_thread;
    L.status = ctx->status_dev;
    L.num_sms = ctx->num_sms;
    if (mode == kModeK && (int)ctx->tune.size() >= L.R && ctx->tune[L.R - 1].width > 0) {
      L.r_min = ctx->tune[L.R - 1].width;
      L.tm = ctx->tune[L.R - 1].tm;
      L.nsplit = ctx->tune[L.R - 1].nsplit;
    }
    if (ctx->planning) {
      L.plan_only = true;
      cudaError_t e = ctx->f64 ? launch_kmv_f64(L, ctx->stream) : launch_kmv_f32(L, ctx->stream);
      ctx->last_nsplit = L.planned_nsplit;
      if (e != cudaSuccess)
        return fail(ctx, ULISSE_ERR_CUDA, std::string("K V plan: ") + cudaGetErrorString(e));
      CKS(grow_kmv_scratch(ctx, L.need_partials_bytes, L.need_counters));
      continue;
    }
    for (int attempt = 0; attempt < 2; ++attempt) {
      L.partials = ctx->partials;
      L.partials_bytes = ctx->partials_bytes;
      L.counters = ctx->counters;
      L.counters_len = ctx->counters_len;
      cudaEvent_t ea = nullptr, eb = nullptr;
      prof_begin(ctx, &ea, &eb);
      cudaError_t e = ctx->f64 ? launch_kmv_f64(L, ctx->stream) : launch_kmv_f32(L, ctx->stream);
      if (ctx->prof) {
        if (e == cudaSuccess)
          prof_end(ctx, 0, ea, eb,
                   (double)ctx->n * ctx->n * (3.0 * ctx->d + 2.0 + 2.0 * L.R));
        else
          ctx->free_events.push_back({ea, eb});
      }
      if (e == cudaSuccess) {
        if (!ctx->capturing) ctx->launches++;
        break;
      }
      if (e != cudaErrorMemoryAllocation || attempt == 1 || ctx->capturing)
        return fail(ctx, ULISSE_ERR_CUDA, std::string("K V launch: ") + cudaGetErrorString(e));
      cudaGetLastError();
      // Grow the split-j scratch to what this launch needs, then retry.
      CKS(grow_kmv_scratch(ctx, L.need_partials_bytes, L.need_counters));
    }
    if (!ctx->capturing) ctx->entry_rhs += (double)ctx->n * (double)ctx->n * (double)L.R;
  }
  return ULISSE_OK;
}

static ulisse_status read_status(ulisse_ctx* ctx, int* status) {
  CK(cudaMemcpyAsync(ctx->h_status, ctx->status_dev, sizeof(int), cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  prof_drain(ctx);
  *status = *ctx->h_status;
  return ULISSE_OK;
}

// A CTA whose bounded wait ran out returns before it counts itself in its row block's split
// counter or the gradient's last-CTA counter (both reset themselves only when every CTA
// arrives): zero them, so that the context's next launches pick their last CTA correctly.
static void reset_counters_after_timeout(ulisse_ctx* ctx) {
  if (ctx->counters && ctx->counters_len > 0)
    cudaMemsetAsync(ctx->counters, 0, sizeof(int) * ctx->counters_len, ctx->stream);
  if (ctx->gcounter) cudaMemsetAsync(ctx->gcounter, 0, sizeof(int), ctx->stream);
  cudaStreamSynchronize(ctx->stream);
}

static ulisse_status status_to_result(ulisse_ctx* ctx, int s) {
  if (s & kStatusTimeout) {
    reset_counters_after_timeout(ctx);
    return fail(ctx, ULISSE_ERR_TIMEOUT, "a bounded device wait ran out");
  }
  if (s & kStatusBadM) return fail(ctx, ULISSE_ERR_ARG, "M is not positive definite");
  if (s & kStatusBreakdown)
    return fail(ctx, ULISSE_ERR_BREAKDOWN, "CG breakdown (d^T K d <= 0 or non-finite)");
  if (s & kStatusMaxIter) return fail(ctx, ULISSE_ERR_MAXITER, "a solve reached max_iter");
  return ULISSE_OK;
}

template <typename T>
static CgArgs<T> cg_args(ulisse_ctx* ctx, int has_s0, unsigned long long step) {
  CgArgs<T> a;
  a.S = (T*)ctx->S;
  a.E = (T*)ctx->E;
  a.D = (T*)ctx->D;
  a.KD = (const T*)ctx->KD;
  a.B = (const T*)ctx->B;
  a.SE = (T*)ctx->SE;
  a.n = ctx->n;
  a.ld = ctx->ldn;
  a.st = ctx->st;
  a.st_next = ctx->st_next;
  a.part1 = ctx->part1;
  a.part2 = ctx->part2;
  a.nchunk = 1;
  a.chunk = ctx->n;
  a.live = ctx->live;
  a.alpha_thr = ctx->cfg.q * std::sqrt((double)ctx->n);
  a.eps = ctx->cfg.eps;
  a.beta = ctx->cfg.beta;
  a.max_iter = ctx->cfg.max_iter;
  a.has_s0 = has_s0;
  a.seed = ctx->cfg.seed;
  a.step = step;
  a.cs = nullptr;
  a.n_live = nullptr;
  a.warm_refresh = 0;
  a.warm_valid = ctx->warm_valid;
  a.y_learned = 0;
  a.Sbest = (T*)ctx->Sbest;
  a.status = ctx->status_dev;
  return a;
}

// Rows per CTA of the CG start over all R columns: about two waves of CTAs, at least 2048
// rows each (one CTA per column for small problems).  Returns the chunk count.
static int cg_init_split(long long n, int R, int num_sms, long long* chunk) {
  const long long target = std::max(1, (2 * num_sms + R - 1) / R);
  long long ch = std::max<long long>((n + target - 1) / target, 2048);
  ch = std::max<long long>(ch, (n + kMaxCgChunks - 1) / kMaxCgChunks);
  ch = (ch + 255) / 256 * 256;
  *chunk = ch;
  return (int)((n + ch - 1) / ch);
}

// Kernel launches of the CG start: the partial sums first when a column spans several chunks.
static int cg_init_launch_count(long long n, int R, int num_sms) {
  long long ch;
  return cg_init_split(n, R, num_sms, &ch) > 1 ? 2 : 1;
}

// The CG start of columns 0..R-1 (cg_init_kernel, after cg_init_dot_kernel when a column
// spans several chunks).
template <typename T>
static cudaError_t launch_cg_init(CgArgs<T> a, int R, int num_sms, cudaStream_t s) {
  a.nchunk = cg_init_split(a.n, R, num_sms, &a.chunk);
  const dim3 grid((unsigned)a.nchunk, (unsigned)R);
  if (a.nchunk > 1) cg_init_dot_kernel<T><<<grid, kCgChunkNT, 0, s>>>(a);
  cg_init_kernel<T><<<grid, kCgChunkNT, 0, s>>>(a);
  return cudaGetLastError();
}

// Column metadata (estimator count, estimator offset, random-stream column) for R columns.
static ulisse_status upload_meta(ulisse_ctx* ctx, int R, const int* n_est, int* total_est) {
  std::vector<ColState> h(R);
  int off = 0;
  for (int c = 0; c < R; ++c) {
    std::memset(&h[c], 0, sizeof(ColState));
    h[c].n_est = n_est ? n_est[c] : 1;
    h[c].est_off = off;
    h[c].colid = c;
    off += h[c].n_est;
  }
  CK(cudaMemcpyAsync(ctx->st, h.data(), sizeof(ColState) * R, cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  *total_est = off;
  return ULISSE_OK;
}

// Batched CG + ULISSE on columns 0..R-1 of B (S holds s_0 when has_s0).  The host learns
// the live count after every iteration and launches K V on the live columns only.
// s0_cols > 0: columns 0..s0_cols-1 of S hold initial iterates (the rest are zero).
// warm: every column's previous final iterate is in S (cg_init decides per column which to
// keep, see CgArgs); y_learned: column 0 holds the learned warm start instead.
template <typename T>
static ulisse_status solve_core(ulisse_ctx* ctx, int R, int s0_cols, unsigned long long step,
                                bool warm = false, bool y_learned = false) {
  CgArgs<T> a = cg_args<T>(ctx, s0_cols > 0, step);
  if (warm) {
    a.warm_refresh = ctx->cfg.probe_refresh;
    a.y_learned = y_learned ? 1 : 0;
    CKS(run_kmv(ctx, ctx->S, ctx->warm_map + (y_learned ? ctx->cap : 0), R, ctx->KD, ctx->iota,
                kModeK, -1));
    ctx->mvp_rounds += 1;
  } else if (s0_cols > 0) {
    if (s0_cols < R)
      CK(cudaMemsetAsync((char*)ctx->KD + (size_t)s0_cols * ctx->ldn * ctx->esz, 0,
                         (size_t)(R - s0_cols) * ctx->ldn * ctx->esz, ctx->stream));
    CKS(run_kmv(ctx, ctx->S, ctx->iota, s0_cols, ctx->KD, ctx->iota, kModeK, -1));
    ctx->mvp_rounds += 1;
  }
  CK(launch_cg_init(a, R, ctx->num_sms, ctx->stream));
  ctx->launches += cg_init_launch_count(ctx->n, R, ctx->num_sms);
  int n_prev = 0;
  for (int it = 0; it <= ctx->cfg.max_iter; ++it) {
    compact_kernel<<<1, 32, 0, ctx->stream>>>(ctx->st, ctx->st_next, R, n_prev, ctx->live,
                                              ctx->n_live_dev);
    CK(cudaGetLastError());
    ctx->launches++;
    CK(cudaMemcpyAsync(ctx->h_n_live, ctx->n_live_dev, sizeof(int), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    prof_drain(ctx);
    const int nl = *ctx->h_n_live;
    if (nl == 0) break;
    CKS(run_kmv(ctx, ctx->D, ctx->live, nl, ctx->KD, ctx->live, kModeK, -1));
    ctx->mvp_rounds += 1;
    // Spread the live columns over about two waves of CTAs (at least 2048 rows each).
    const long long target = std::max(1, (2 * ctx->num_sms + nl - 1) / nl);
    long long ch = std::max<long long>((ctx->n + target - 1) / target, 2048);
    ch = std::max<long long>(ch, (ctx->n + kMaxCgChunks - 1) / kMaxCgChunks);
    ch = (ch + 255) / 256 * 256;
    a.chunk = ch;
    a.nchunk = (int)((ctx->n + ch - 1) / ch);
    const dim3 grid(a.nchunk, nl);
    cg_dot_kernel<T><<<grid, kCgChunkNT, 0, ctx->stream>>>(a);
    cg_update_kernel<T><<<grid, kCgChunkNT, 0, ctx->stream>>>(a);
    cg_finish_kernel<T><<<grid, kCgChunkNT, 0, ctx->stream>>>(a);
    CK(cudaGetLastError());
    ctx->launches += 3;
    n_prev = nl;
  }
  return ULISSE_OK;
}

// Preconditioned CG (cfg.pcg_delta > 0) with ULISSE on the outer iteration, columns 0..R-1
// of B, zero start; see pcg_kernels.cuh.  The host learns which columns are live after every
// outer iteration and every inner one (one small read each, as solve_core does) and launches
// K V on those columns only; every K V product, outer or inner, counts as a round.
template <typename T>
static ulisse_status pcg_core(ulisse_ctx* ctx, int R, unsigned long long step) {
  if (ctx->pcg_cap < ctx->cap) {
    CK(cudaStreamSynchronize(ctx->stream));
    dev_free(ctx->pcg_buf);
    dev_free(reinterpret_cast<void*&>(ctx->pcg_aux));
    dev_free(reinterpret_cast<void*&>(ctx->pcg_live));
    CKS(dev_alloc(ctx, &ctx->pcg_buf, (size_t)ctx->ldn * ctx->esz * ctx->cap * 5));
    CKS(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->pcg_aux), sizeof(PcgAux) * ctx->cap));
    CKS(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->pcg_live), sizeof(int) * ctx->cap));
    // the padding rows of every vector stay zero (the K V kernels read whole tiles)
    CK(cudaMemsetAsync(ctx->pcg_buf, 0, (size_t)ctx->ldn * ctx->esz * ctx->cap * 5, ctx->stream));
    ctx->pcg_cap = ctx->cap;
  }
  const size_t blk = (size_t)ctx->ldn * ctx->cap;   // elements per buffer
  T* base = (T*)ctx->pcg_buf;
  PcgArgs<T> a;
  a.S = (T*)ctx->S;
  a.E = (T*)ctx->E;
  a.D = (T*)ctx->D;
  a.KD = (const T*)ctx->KD;
  a.Z = base;
  a.X = base + blk;
  a.Rr = base + 2 * blk;
  a.P = base + 3 * blk;
  a.KP = base + 4 * blk;
  a.B = (const T*)ctx->B;
  a.SE = (T*)ctx->SE;
  a.n = ctx->n;
  a.ld = ctx->ldn;
  a.st = ctx->st;
  a.aux = ctx->pcg_aux;
  a.live = ctx->pcg_live;
  a.alpha_thr = ctx->cfg.q * std::sqrt((double)ctx->n);
  a.eps = ctx->cfg.eps;
  a.beta = ctx->cfg.beta;
  a.delta = ctx->cfg.pcg_delta;
  a.tau = ctx->cfg.pcg_inner_tol;
  a.max_iter = ctx->cfg.max_iter;
  a.inner_max = ctx->cfg.pcg_inner_max;
  a.seed = ctx->cfg.seed;
  a.step = step;
  a.status = ctx->status_dev;

  std::vector<int> cols;
  auto upload = [&](const std::vector<int>& v) -> ulisse_status {
    CK(cudaMemcpyAsync(ctx->pcg_live, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice,
                       ctx->stream));
    return ULISSE_OK;
  };
  // columns whose outer iteration is still running
  std::vector<ColState> hst(R);
  auto outer_live = [&](std::vector<int>& out) -> ulisse_status {
    CK(cudaMemcpyAsync(hst.data(), ctx->st, sizeof(ColState) * R, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    prof_drain(ctx);
    out.clear();
    for (int c = 0; c < R; ++c)
      if (hst[c].phase != kDone) out.push_back(c);
    return ULISSE_OK;
  };
  std::vector<PcgAux> hax(R);
  // z = J^{-1} e for the listed columns (inner CG), then the new directions
  auto precondition = [&](const std::vector<int>& L) -> ulisse_status {
    CKS(upload(L));
    pcg_inner_init_kernel<T><<<(unsigned)L.size(), kPcgNT, 0, ctx->stream>>>(a);
    CK(cudaGetLastError());
    ctx->launches++;
    std::vector<int> in = L;
    for (int k = 0; k < ctx->cfg.pcg_inner_max && !in.empty(); ++k) {
      CKS(upload(in));
      CKS(run_kmv(ctx, a.P, ctx->pcg_live, (int)in.size(), (void*)a.KP, ctx->pcg_live, kModeK,
                  -1));
      ctx->mvp_rounds += 1;
      pcg_inner_step_kernel<T><<<(unsigned)in.size(), kPcgNT, 0, ctx->stream>>>(a);
      CK(cudaGetLastError());
      ctx->launches++;
      CK(cudaMemcpyAsync(hax.data(), ctx->pcg_aux, sizeof(PcgAux) * R, cudaMemcpyDeviceToHost,
                         ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      prof_drain(ctx);
      std::vector<int> next;
      for (int c : in)
        if (!hax[c].inner_done) next.push_back(c);
      in.swap(next);
    }
    CKS(upload(L));
    pcg_dir_kernel<T><<<(unsigned)L.size(), kPcgNT, 0, ctx->stream>>>(a);
    CK(cudaGetLastError());
    ctx->launches++;
    return ULISSE_OK;
  };

  for (int c = 0; c < R; ++c) cols.push_back(c);
  CKS(upload(cols));
  pcg_init_kernel<T><<<R, kPcgNT, 0, ctx->stream>>>(a);
  CK(cudaGetLastError());
  ctx->launches++;
  CKS(outer_live(cols));
  if (!cols.empty()) CKS(precondition(cols));
  for (int it = 0; it < ctx->cfg.max_iter; ++it) {
    CKS(outer_live(cols));
    if (cols.empty()) break;
    CKS(upload(cols));
    CKS(run_kmv(ctx, ctx->D, ctx->pcg_live, (int)cols.size(), ctx->KD, ctx->pcg_live, kModeK,
                -1));
    ctx->mvp_rounds += 1;
    pcg_step_kernel<T><<<(unsigned)cols.size(), kPcgNT, 0, ctx->stream>>>(a);
    CK(cudaGetLastError());
    ctx->launches++;
    CKS(outer_live(cols));
    if (cols.empty()) break;
    CKS(precondition(cols));
  }
  return ULISSE_OK;
}

static ulisse_status solve_dispatch(ulisse_ctx* ctx, int R, int s0_cols,
                                    unsigned long long step, bool warm = false,
                                    bool y_learned = false) {
  if (ctx->cfg.pcg_delta > 0.0) {
    if (s0_cols > 0 || warm || y_learned)
      return fail(ctx, ULISSE_ERR_ARG, "preconditioned CG solves start from zero (no S0, "
                                       "no warm-started solves, no learned warm start)");
    return ctx->f64 ? pcg_core<double>(ctx, R, step) : pcg_core<float>(ctx, R, step);
  }
  return ctx->f64 ? solve_core<double>(ctx, R, s0_cols, step, warm, y_learned)
                  : solve_core<float>(ctx, R, s0_cols, step, warm, y_learned);
}

// Gradient column maps: left factors SE[0] (a1) and SE[2..1+nr] (z_j) with scales 1/2 and
// -1/(2 nr); right factors B[0] (a2, copied there after the solve) and B[1..nr] (r_j).
static ulisse_status ensure_grad_maps(ulisse_ctx* ctx, int nr) {
  if (ctx->grad_nr == nr) return ULISSE_OK;
  const int M = 1 + nr;
  std::vector<int> am(M), bm(M);
  std::vector<float> sf(M);
  std::vector<double> sd(M);
  for (int m = 0; m < M; ++m) {
    am[m] = (m == 0) ? 0 : m + 1;
    bm[m] = m;
    const double s = (m == 0) ? 0.5 : -1.0 / (2.0 * nr);
    sf[m] = (float)s;
    sd[m] = s;
  }
  CK(cudaMemcpyAsync(ctx->amap, am.data(), sizeof(int) * M, cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaMemcpyAsync(ctx->bmap, bm.data(), sizeof(int) * M, cudaMemcpyHostToDevice,
                     ctx->stream));
  if (ctx->f64)
    CK(cudaMemcpyAsync(ctx->sa_dev, sd.data(), sizeof(double) * M, cudaMemcpyHostToDevice,
                       ctx->stream));
  else
    CK(cudaMemcpyAsync(ctx->sa_dev, sf.data(), sizeof(float) * M, cudaMemcpyHostToDevice,
                       ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->grad_nr = nr;
  return ULISSE_OK;
}

// The tensor-core gradient pass reads the TF32 row images of the K V pass (padded d <= 8);
// the single-context images carry b_j in their augmented column when d pads to less than 8.
static void set_grad_images(GradLaunch& L, const ulisse_ctx* c) {
  L.X_hi = c->Xt_hi;
  L.X_lo = c->Xt_lo;
  L.X_off = c->ld128 * 24;
  L.c_has_bj = c->DP < 8 && !c->tc_no_aug;
}

// The fused gradient pass over the columns of SE (left factors, scaled) and B (right factors);
// the maps and scales default to the gradient's own.
static ulisse_status run_grad(ulisse_ctx* ctx, int M, const int* amap = nullptr,
                              const void* sa = nullptr, const int* bmap = nullptr) {
  GradLaunch L{};
  L.xhat = ctx->xhat;
  L.n = ctx->n;
  L.ldn = ctx->ldn;
  L.d = ctx->d;
  L.DP = ctx->DP;
  L.A = ctx->SE;
  L.amap = amap ? amap : ctx->amap;
  L.sa = sa ? sa : ctx->sa_dev;
  L.B = ctx->B;
  L.bmap = bmap ? bmap : ctx->bmap;
  L.ld = ctx->ldn;
  L.M = M;
  L.params = ctx->params;
  L.counter = ctx->gcounter;
  L.g_out = ctx->g_dev;
  L.status = ctx->status_dev;
  L.num_sms = ctx->num_sms;
  L.bneg = ctx->bneg;
  L.tc_hi = ctx->Gt_hi;
  L.tc_lo = ctx->Gt_lo;
  L.tc_ld = ctx->ld128;
  set_grad_images(L, ctx);
  for (int attempt = 0; attempt < 2; ++attempt) {
    L.partials = ctx->gpart;
    L.partials_len = ctx->gpart_len;
    L.plan_only = ctx->planning;
    cudaEvent_t ea = nullptr, eb = nullptr;
    prof_begin(ctx, &ea, &eb);
    cudaError_t e = ctx->f64     ? launch_grad_f64(L, ctx->stream)
                    : ctx->mixed ? launch_grad_tc(L, ctx->stream)
                                 : launch_grad_f32(L, ctx->stream);
    if (ctx->prof) {
      if (e == cudaSuccess && !ctx->planning) {
        // the tensor-core pass visits each unordered pair once with 2M factor products; the
        // SIMT passes visit every ordered pair with M
        const double nn = (double)ctx->n;
        const double flop = ctx->mixed ? nn * (nn + 1.0) / 2.0 * (5.0 * ctx->d + 4.0 + 4.0 * M)
                                       : nn * nn * (5.0 * ctx->d + 4.0 + 2.0 * M);
        prof_end(ctx, 1, ea, eb, flop);
      }
      else
        ctx->free_events.push_back({ea, eb});
    }
    if (e == cudaSuccess && !ctx->planning) {
      if (!ctx->capturing) ctx->launches += ctx->mixed ? 3 : 1;   // tensor cores: 2 packings
      break;
    }
    if (e != cudaSuccess && (e != cudaErrorMemoryAllocation || attempt == 1 || ctx->capturing))
      return fail(ctx, ULISSE_ERR_CUDA, std::string("gradient launch: ") + cudaGetErrorString(e));
    cudaGetLastError();
    if (L.need_partials_len > ctx->gpart_len) {
      ctx->graph_key = -1;
      CK(cudaStreamSynchronize(ctx->stream));
      dev_free(reinterpret_cast<void*&>(ctx->gpart));
      ctx->gpart_len = 0;
      CKS(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->gpart), sizeof(double) * L.need_partials_len));
      ctx->gpart_len = L.need_partials_len;
    }
    if (ctx->planning) return ULISSE_OK;
  }
  if (!ctx->capturing) ctx->entry_rhs += (double)ctx->n * (double)ctx->n * (double)M;
  return ULISSE_OK;
}

// Whole gradient path for one step (a1..a6): psi must already be in psi_dev.  With
// prologue_only the call stops after the probes and the column metadata (a batch runs the
// solves and the gradient pass of all its problems together).
static ulisse_status grad_core(ulisse_ctx* ctx, unsigned long long step,
                               bool prologue_only = false) {
  const int nr = ctx->cfg.n_probes, R = 1 + nr;
  CKS(ensure_columns(ctx, R, R + 1));
  CKS(ensure_grad_maps(ctx, nr));
  CKS(prescale(ctx));
  // B[0] = y, B[1..nr] = probes for this epoch
  CK(cudaMemcpyAsync(ctx->B, ctx->y, ctx->ldn * ctx->esz, cudaMemcpyDeviceToDevice,
                     ctx->stream));
  const unsigned long long epoch = step / (unsigned long long)ctx->cfg.probe_refresh;
  dim3 pg((unsigned)std::min<long long>((ctx->n + 255) / 256, 2LL * ctx->num_sms), nr);
  if (ctx->f64)
    probes_kernel<double><<<pg, 256, 0, ctx->stream>>>((double*)ctx->B, ctx->ldn, ctx->n, nr,
                                                        ctx->cfg.probe_kind, ctx->cfg.seed, epoch);
  else
    probes_kernel<float><<<pg, 256, 0, ctx->stream>>>((float*)ctx->B, ctx->ldn, ctx->n, nr,
                                                       ctx->cfg.probe_kind, ctx->cfg.seed, epoch);
  CK(cudaGetLastError());
  ctx->launches++;
  if (ctx->meta_grad_R != R) {
    // column metadata (estimator counts, offsets, stream ids) survives the solves
    std::vector<int> n_est(R, 1);
    n_est[0] = 2;
    int tot = 0;
    CKS(upload_meta(ctx, R, n_est.data(), &tot));
    ctx->meta_grad_R = R;
  }
  if (prologue_only) return ULISSE_OK;
  int s0_cols = 0;
  const bool warm = ctx->cfg.warm_start_probes != 0;
  const bool learned = ctx->ws_use && ctx->ws_trained;
  if (learned) {
    // learned warm start for the y column; the probe columns start from zero (or, with
    // warm-started solves, from their previous iterates)
    ws_x0(ctx->wsb, ctx->psi_dev, true, (const float*)ctx->xhat, ctx->DP, ctx->n, ctx->params,
          ctx->ws_c, (float*)ctx->S, ctx->num_sms, ctx->stream);
    CK(cudaGetLastError());
    ctx->launches += 2;
    if (!warm)
      CK(cudaMemsetAsync((char*)ctx->S + ctx->ldn * ctx->esz, 0,
                         (size_t)(R - 1) * ctx->ldn * ctx->esz, ctx->stream));
    s0_cols = 1;
  }
  CKS(solve_dispatch(ctx, R, warm ? 0 : s0_cols, step, warm, learned));
  if (warm) CK(cudaMemsetAsync(ctx->warm_valid, 0x01, sizeof(int), ctx->stream));
  if (ctx->ws_record) {
    ws_record(ctx->wsb, ctx->psi_dev, (const float*)ctx->y, (const float*)ctx->xhat, ctx->DP,
              ctx->params, ctx->ws_next % ctx->wsb.max_pairs, (unsigned long long)ctx->ws_next,
              ctx->stream);
    CK(cudaGetLastError());
    ctx->launches += 4;
    ctx->ws_next++;
    ctx->ws_pairs = std::min(ctx->ws_pairs + 1, ctx->wsb.max_pairs);
  }
  // a2 (second estimate of K^{-1} y) becomes the right factor of the quadratic term.
  CK(cudaMemcpyAsync(ctx->B, (char*)ctx->SE + ctx->ldn * ctx->esz, ctx->ldn * ctx->esz,
                     cudaMemcpyDeviceToDevice, ctx->stream));
  CKS(run_grad(ctx, R));
  return ULISSE_OK;
}

static ulisse_status check_cfg(const ulisse_config* c) {
  if (!c) return ULISSE_ERR_ARG;
  if (c->precision < 0 || c->precision > 2) return ULISSE_ERR_ARG;
  if (c->n_probes < 1 || c->n_probes > kMaxM - 1) return ULISSE_ERR_ARG;
  if (c->probe_kind < 0 || c->probe_kind > 1) return ULISSE_ERR_ARG;
  if (c->probe_refresh < 1 || c->max_iter < 1) return ULISSE_ERR_ARG;
  if (!(c->q >= 0.0) || !(c->beta > 0.0) || !(c->eps >= 0.0)) return ULISSE_ERR_ARG;
  if (!std::isfinite(c->q) || !std::isfinite(c->beta) || !std::isfinite(c->eps))
    return ULISSE_ERR_ARG;
  if (c->kmv_rows_per_thread != 0 && c->kmv_rows_per_thread != 2 && c->kmv_rows_per_thread != 4)
    return ULISSE_ERR_ARG;
  if (c->tc_cross_term < 0 || c->tc_cross_term > 2) return ULISSE_ERR_ARG;
  if (!(c->pcg_delta >= 0.0) || !std::isfinite(c->pcg_delta)) return ULISSE_ERR_ARG;
  if (c->pcg_delta > 0.0) {
    if (!(c->pcg_inner_tol > 0.0 && c->pcg_inner_tol < 1.0) || c->pcg_inner_max < 1)
      return ULISSE_ERR_ARG;
    if (c->warm_start_probes != 0) return ULISSE_ERR_ARG;   // PCG solves start from zero
  }
  return ULISSE_OK;
}

static ulisse_status create_impl(ulisse_ctx** out, const float* X, const float* y, long long n,
                                 int d, const ulisse_config* cfg, void* stream,
                                 cudaMemcpyKind kind) {
  if (!out) return fail(nullptr, ULISSE_ERR_ARG, "out is null");
  *out = nullptr;
  if (!X || !y) return fail(nullptr, ULISSE_ERR_ARG, "X or y is null");
  if (n < 1 || n > 2147483647LL) return fail(nullptr, ULISSE_ERR_ARG, "n out of range");
  if (d < 1 || d > kMaxD) return fail(nullptr, ULISSE_ERR_ARG, "d must be in 1..16");
  if (check_cfg(cfg) != ULISSE_OK) return fail(nullptr, ULISSE_ERR_ARG, "invalid config");
  ulisse_ctx* ctx = new ulisse_ctx();
  ctx->stream = (cudaStream_t)stream;
  ctx->cfg = *cfg;
  ctx->n = n;
  ctx->d = d;
  ctx->DP = dp_for(d);
  ctx->ldn = (n + kBN - 1) / kBN * kBN;
  ctx->f64 = cfg->precision == ULISSE_PREC_FP64;
  ctx->mixed = cfg->precision == ULISSE_PREC_MIXED;
  ctx->esz = ctx->f64 ? 8 : 4;
  ctx->ld128 = (n + 127) / 128 * 128;
  auto bail = [&](ulisse_status s) {
    g_create_error = ctx->err;
    ulisse_destroy(ctx);
    return s;
  };
  if (cudaGetDevice(&ctx->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device) !=
          cudaSuccess) {
    ctx->err = "no CUDA device";
    return bail(ULISSE_ERR_CUDA);
  }
  ulisse_status s;
  if ((s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->X), sizeof(float) * n * d)) ||
      (s = dev_alloc(ctx, &ctx->y, ctx->ldn * ctx->esz)) ||
      (s = dev_alloc(ctx, &ctx->xhat, ctx->ldn * ctx->DP * ctx->esz)) ||
      (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->params), sizeof(DevParams))) ||
      (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->psi_dev), sizeof(double) * kMaxP)) ||
      (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->n_live_dev), sizeof(int))) ||
      (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->gcounter), sizeof(int))) ||
      (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->g_dev), sizeof(double) * kMaxP)) ||
      (s = dev_alloc(ctx, &ctx->sa_dev, sizeof(double) * kMaxM)) ||
      (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->amap), sizeof(int) * kMaxM)) ||
      (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->bmap), sizeof(int) * kMaxM)) ||
      (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->M_dev), sizeof(double) * kMaxP * kMaxP)) ||
      (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->prior_dev), sizeof(double) * kMaxP)) ||
      (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->status_dev), sizeof(int))) ||
      (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->warm_valid), sizeof(int))))
    return bail(s);
  if (ctx->mixed) {
    if ((s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->bneg), sizeof(float) * ctx->ld128)) ||
        (s = dev_alloc(ctx, &ctx->Vt_hi, 2 * ctx->ld128 * 64)) ||
        (s = dev_alloc(ctx, &ctx->Vt_lo, 2 * ctx->ld128 * 64)) ||
        (s = dev_alloc(ctx, &ctx->Gt_hi, 2 * ctx->ld128 * kGtScratchRows)) ||
        (s = dev_alloc(ctx, &ctx->Gt_lo, 2 * ctx->ld128 * kGtScratchRows)) ||
        (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->Xt_hi), 4 * ctx->ld128 * 48)) ||
        (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->Xt_lo), 4 * ctx->ld128 * 48)))
      return bail(s);
  }
  if (cudaMallocHost(&ctx->h_n_live, sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&ctx->h_status, sizeof(int)) != cudaSuccess) {
    ctx->err = "cudaMallocHost failed";
    return bail(ULISSE_ERR_NOMEM);
  }
  // Inputs: X as given (row-major float); y into the context's element type.
  if (cudaMemcpyAsync(ctx->X, X, sizeof(float) * n * d, kind, ctx->stream) != cudaSuccess) {
    ctx->err = "copy of X failed";
    return bail(ULISSE_ERR_CUDA);
  }
  if (!ctx->f64) {
    if (cudaMemcpyAsync(ctx->y, y, sizeof(float) * n, kind, ctx->stream) != cudaSuccess) {
      ctx->err = "copy of y failed";
      return bail(ULISSE_ERR_CUDA);
    }
  } else {
    float* tmp = nullptr;
    if (cudaMalloc(&tmp, sizeof(float) * n) != cudaSuccess) {
      ctx->err = "cudaMalloc failed";
      return bail(ULISSE_ERR_NOMEM);
    }
    cudaMemcpyAsync(tmp, y, sizeof(float) * n, kind, ctx->stream);
    convert_cols_kernel<float, double><<<dim3(64, 1), 256, 0, ctx->stream>>>(
        tmp, n, (double*)ctx->y, ctx->ldn, n);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(tmp);
  }
  if ((s = ensure_columns(ctx, 1 + cfg->n_probes, 2 + cfg->n_probes))) return bail(s);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    ctx->err = "stream synchronisation failed";
    return bail(ULISSE_ERR_CUDA);
  }
  *out = ctx;
  return ULISSE_OK;
}

extern "C" {

// the step graph (defined with ulisse_sgld_chain)
static bool graph_usable(const ulisse_ctx* ctx);
static ulisse_status graph_alloc(ulisse_ctx* ctx);
static ulisse_status graph_prepare(ulisse_ctx* ctx, const double* M, const double* prior,
                                   unsigned long long step0, const double* eps_dev,
                                   double* trace_dev);
static void graph_fold_counters(ulisse_ctx* ctx, int n_steps);

void ulisse_config_default(ulisse_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->precision = ULISSE_PREC_FP32;
  cfg->n_probes = 4;
  cfg->probe_kind = ULISSE_PROBE_RADEMACHER;
  cfg->probe_refresh = 1;
  cfg->warm_start_probes = 0;
  cfg->q = 1.0;
  cfg->beta = 1.0;
  cfg->eps = 1e-8;
  cfg->max_iter = 1000;
  cfg->seed = 0;
  cfg->kmv_rows_per_thread = 0;
  cfg->tc_cross_term = 0;
  cfg->pcg_delta = 0.0;
  cfg->pcg_inner_tol = 1e-2;
  cfg->pcg_inner_max = 100;
}

ulisse_status ulisse_create(ulisse_ctx** out, const float* X, const float* y, long long n, int d,
                            const ulisse_config* cfg, void* stream) {
  return create_impl(out, X, y, n, d, cfg, stream, cudaMemcpyDeviceToDevice);
}

ulisse_status ulisse_create_host(ulisse_ctx** out, const float* X, const float* y, long long n,
                                 int d, const ulisse_config* cfg, void* stream) {
  return create_impl(out, X, y, n, d, cfg, stream, cudaMemcpyHostToDevice);
}

static ulisse_status copy_stats(ulisse_ctx* ctx, ulisse_col_stats* stats, int R) {
  if (!stats) return ULISSE_OK;
  std::vector<ColState> h(R);
  CK(cudaMemcpyAsync(h.data(), ctx->st, sizeof(ColState) * R, cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int c = 0; c < R; ++c) {
    stats[c].l = h[c].l;
    stats[c].iterations = h[c].m;
    stats[c].outcome = h[c].outcome;
    stats[c].J0 = h[c].J[0];
    stats[c].J1 = h[c].n_est > 1 ? h[c].J[1] : -1;
  }
  return ULISSE_OK;
}

static ulisse_status kmv_common(ulisse_ctx* ctx, const double* psi, int which, const void* V,
                                int R, void* U, bool f64_data) {
  if (!ctx) return ULISSE_ERR_ARG;
  if (ctx->batched) return fail(ctx, ULISSE_ERR_ARG, "batched context: use the ulisse_batch_* calls");
  if (!V || !U || R < 1 || R > 4096) return fail(ctx, ULISSE_ERR_ARG, "V/U null or R out of range");
  if (which < -1 || which > ctx->d + 1) return fail(ctx, ULISSE_ERR_ARG, "which out of range");
  if (f64_data && !ctx->f64)
    return fail(ctx, ULISSE_ERR_ARG, "double data needs a context created with FP64 precision");
  CKS(set_psi_host(ctx, psi));
  CKS(prescale(ctx));
  CKS(ensure_columns(ctx, R, R));
  const long long n = ctx->n;
  const size_t ue = f64_data ? 8 : 4;
  // caller's V (leading dimension n) -> context buffer D (leading dimension ldn)
  if (ctx->esz == ue) {
    CK(cudaMemcpy2DAsync(ctx->D, ctx->ldn * ctx->esz, V, n * ue, n * ue, R,
                         cudaMemcpyDeviceToDevice, ctx->stream));
  } else {
    convert_cols_kernel<float, double><<<dim3(64, R), 256, 0, ctx->stream>>>(
        (const float*)V, n, (double*)ctx->D, ctx->ldn, n);
    CK(cudaGetLastError());
  }
  int mode = kModeK, w = -1;
  if (which >= 0 && which < ctx->d) { mode = kModeDLen; w = which; }
  else if (which == ctx->d) mode = kModeDSig;
  else if (which == ctx->d + 1) mode = kModeDLam;
  CKS(run_kmv(ctx, ctx->D, ctx->iota, R, ctx->KD, ctx->iota, mode, w));
  if (ctx->esz == ue) {
    CK(cudaMemcpy2DAsync(U, n * ue, ctx->KD, ctx->ldn * ctx->esz, n * ue, R,
                         cudaMemcpyDeviceToDevice, ctx->stream));
  } else {
    convert_cols_kernel<double, float><<<dim3(64, R), 256, 0, ctx->stream>>>(
        (const double*)ctx->KD, ctx->ldn, (float*)U, n, n);
    CK(cudaGetLastError());
  }
  return ULISSE_OK;
}

ulisse_status ulisse_kmv(ulisse_ctx* ctx, const double* psi, int which, const float* V, int R,
                         float* U) {
  return kmv_common(ctx, psi, which, V, R, U, false);
}

ulisse_status ulisse_kmv_f64(ulisse_ctx* ctx, const double* psi, int which, const double* V,
                             int R, double* U) {
  return kmv_common(ctx, psi, which, V, R, U, true);
}

ulisse_status ulisse_solve(ulisse_ctx* ctx, const double* psi, const float* B, int R,
                           const int* n_est, const float* S0, float* S_est,
                           unsigned long long step, ulisse_col_stats* stats) {
  if (!ctx) return ULISSE_ERR_ARG;
  if (ctx->batched) return fail(ctx, ULISSE_ERR_ARG, "batched context: use the ulisse_batch_* calls");
  if (!B || !S_est || R < 1 || R > 1024) return fail(ctx, ULISSE_ERR_ARG, "B/S_est null or R out of range");
  int tot = 0;
  if (n_est)
    for (int c = 0; c < R; ++c) {
      if (n_est[c] < 1 || n_est[c] > 2) return fail(ctx, ULISSE_ERR_ARG, "n_est must be 1 or 2");
      tot += n_est[c];
    }
  else tot = R;
  CKS(set_psi_host(ctx, psi));
  CKS(prescale(ctx));
  CKS(ensure_columns(ctx, R, tot));
  CK(cudaMemsetAsync(ctx->status_dev, 0, sizeof(int), ctx->stream));
  CK(cudaMemsetAsync(ctx->warm_valid, 0, sizeof(int), ctx->stream));   // S is overwritten
  const long long n = ctx->n;
  auto in_cols = [&](const float* src, void* dst) -> ulisse_status {
    if (!ctx->f64) {
      CK(cudaMemcpy2DAsync(dst, ctx->ldn * 4, src, n * 4, n * 4, R, cudaMemcpyDeviceToDevice,
                           ctx->stream));
    } else {
      convert_cols_kernel<float, double><<<dim3(64, R), 256, 0, ctx->stream>>>(
          src, n, (double*)dst, ctx->ldn, n);
      CK(cudaGetLastError());
    }
    return ULISSE_OK;
  };
  CKS(in_cols(B, ctx->B));
  if (S0) CKS(in_cols(S0, ctx->S));
  CKS(upload_meta(ctx, R, n_est, &tot));
  ctx->meta_grad_R = -1;
  CKS(solve_dispatch(ctx, R, S0 ? R : 0, step));
  if (!ctx->f64) {
    CK(cudaMemcpy2DAsync(S_est, n * 4, ctx->SE, ctx->ldn * 4, n * 4, tot,
                         cudaMemcpyDeviceToDevice, ctx->stream));
  } else {
    convert_cols_kernel<double, float><<<dim3(64, tot), 256, 0, ctx->stream>>>(
        (const double*)ctx->SE, ctx->ldn, S_est, n, n);
    CK(cudaGetLastError());
  }
  CKS(copy_stats(ctx, stats, R));
  int st = 0;
  CKS(read_status(ctx, &st));
  return status_to_result(ctx, st);
}

ulisse_status ulisse_grad(ulisse_ctx* ctx, const double* psi, unsigned long long step, double* g,
                          ulisse_col_stats* stats) {
  if (!ctx) return ULISSE_ERR_ARG;
  if (ctx->batched) return fail(ctx, ULISSE_ERR_ARG, "batched context: use the ulisse_batch_* calls");
  if (!g) return fail(ctx, ULISSE_ERR_ARG, "g is null");
  CKS(set_psi_host(ctx, psi));
  CK(cudaMemsetAsync(ctx->status_dev, 0, sizeof(int), ctx->stream));
  CKS(grad_core(ctx, step));
  CK(cudaMemcpyAsync(g, ctx->g_dev, sizeof(double) * (ctx->d + 2), cudaMemcpyDeviceToHost,
                     ctx->stream));
  CKS(copy_stats(ctx, stats, 1 + ctx->cfg.n_probes));
  int st = 0;
  CKS(read_status(ctx, &st));
  return status_to_result(ctx, st);
}

extern "C++" {
template <typename T>
static ulisse_status predict_core(ulisse_ctx* ctx, const float* Xs, long long m,
                                  unsigned long long step, float* mean, float* var) {
  const int R = var ? 1 + (int)m : 1;
  CKS(ensure_columns(ctx, R, R));
  CK(cudaMemsetAsync(ctx->status_dev, 0, sizeof(int), ctx->stream));
  CK(cudaMemsetAsync(ctx->warm_valid, 0, sizeof(int), ctx->stream));   // S is overwritten
  const size_t xs_bytes = (size_t)m * ctx->DP * sizeof(T);
  if (xs_bytes > ctx->pred_xs_bytes) {
    CK(cudaStreamSynchronize(ctx->stream));
    dev_free(ctx->pred_xs);
    ctx->pred_xs_bytes = 0;
    CKS(dev_alloc(ctx, &ctx->pred_xs, xs_bytes));
    ctx->pred_xs_bytes = xs_bytes;
  }
  CK(launch_predict_prescale<T>(Xs, m, ctx->d, ctx->DP, ctx->params, ctx->pred_xs,
                                ctx->num_sms, ctx->stream));
  // B[:, 0] = y and, for the variance, B[:, 1 + j] = k*_j = k_s(X, x*_j)
  CK(cudaMemcpyAsync(ctx->B, ctx->y, ctx->ldn * ctx->esz, cudaMemcpyDeviceToDevice,
                     ctx->stream));
  if (var)
    CK(launch_predict_cross_cols<T>(ctx->xhat, ctx->n, ctx->ldn, ctx->DP, ctx->pred_xs, m,
                                    ctx->params, ctx->B, 1, ctx->stream));
  int tot = 0;
  CKS(upload_meta(ctx, R, nullptr, &tot));
  ctx->meta_grad_R = -1;
  CKS(solve_dispatch(ctx, R, 0, step));
  CK(launch_predict_mean<T>(ctx->xhat, ctx->n, ctx->DP, ctx->pred_xs, m, ctx->params, ctx->SE,
                            mean, ctx->stream));
  if (var)
    CK(launch_predict_var<T>(ctx->B, ctx->SE, ctx->n, ctx->ldn, 1, 1, m, ctx->params, var,
                             ctx->stream));
  ctx->launches += var ? 4 : 2;
  return ULISSE_OK;
}
}  // extern "C++"

ulisse_status ulisse_predict(ulisse_ctx* ctx, const double* psi, const float* Xs, long long m,
                             unsigned long long step, float* mean, float* var) {
  if (!ctx) return ULISSE_ERR_ARG;
  if (ctx->batched) return fail(ctx, ULISSE_ERR_ARG, "batched context: not supported");
  if (!Xs || !mean || m < 1) return fail(ctx, ULISSE_ERR_ARG, "Xs/mean null or m < 1");
  if (var && m > 1023)
    return fail(ctx, ULISSE_ERR_ARG, "with the variance, at most 1023 test inputs per call");
  if (m > (1LL << 26)) return fail(ctx, ULISSE_ERR_ARG, "m too large");
  CKS(set_psi_host(ctx, psi));
  CKS(prescale(ctx));
  CKS(ctx->f64 ? predict_core<double>(ctx, Xs, m, step, mean, var)
               : predict_core<float>(ctx, Xs, m, step, mean, var));
  int st = 0;
  CKS(read_status(ctx, &st));
  return status_to_result(ctx, st);
}

ulisse_status ulisse_dk_bilinear(ulisse_ctx* ctx, const double* psi, const float* A,
                                 const float* B, int M, const double* scale, double* out) {
  if (!ctx) return ULISSE_ERR_ARG;
  if (ctx->batched) return fail(ctx, ULISSE_ERR_ARG, "batched context: not supported");
  if (!A || !B || !out || M < 1 || M > kMaxM)
    return fail(ctx, ULISSE_ERR_ARG, "A/B/out null or M out of range");
  if (scale)
    for (int m = 0; m < M; ++m)
      if (!std::isfinite(scale[m])) return fail(ctx, ULISSE_ERR_ARG, "scale not finite");
  CKS(set_psi_host(ctx, psi));
  CKS(prescale(ctx));
  CKS(ensure_columns(ctx, M, M));
  if (!ctx->q_map) {
    std::vector<int> id(kMaxM);
    for (int m = 0; m < kMaxM; ++m) id[m] = m;
    CKS(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->q_map), sizeof(int) * kMaxM));
    CKS(dev_alloc(ctx, &ctx->q_sa, sizeof(double) * kMaxM));
    CK(cudaMemcpy(ctx->q_map, id.data(), sizeof(int) * kMaxM, cudaMemcpyHostToDevice));
  }
  CK(cudaStreamSynchronize(ctx->stream));   // the scale upload below reuses a host buffer
  std::vector<double> sd(M, 1.0);
  std::vector<float> sf(M, 1.f);
  for (int m = 0; m < M; ++m) {
    if (scale) sd[m] = scale[m];
    sf[m] = (float)sd[m];
  }
  if (ctx->f64)
    CK(cudaMemcpy(ctx->q_sa, sd.data(), sizeof(double) * M, cudaMemcpyHostToDevice));
  else
    CK(cudaMemcpy(ctx->q_sa, sf.data(), sizeof(float) * M, cudaMemcpyHostToDevice));
  CK(cudaMemsetAsync(ctx->status_dev, 0, sizeof(int), ctx->stream));
  const long long n = ctx->n;
  auto in_cols = [&](const float* src, void* dst) -> ulisse_status {
    if (!ctx->f64) {
      CK(cudaMemcpy2DAsync(dst, ctx->ldn * 4, src, n * 4, n * 4, M, cudaMemcpyDeviceToDevice,
                           ctx->stream));
    } else {
      convert_cols_kernel<float, double><<<dim3(64, M), 256, 0, ctx->stream>>>(
          src, n, (double*)dst, ctx->ldn, n);
      CK(cudaGetLastError());
    }
    return ULISSE_OK;
  };
  CKS(in_cols(A, ctx->SE));
  CKS(in_cols(B, ctx->B));
  CKS(run_grad(ctx, M, ctx->q_map, ctx->q_sa, ctx->q_map));
  CK(cudaMemcpyAsync(out, ctx->g_dev, sizeof(double) * (ctx->d + 2), cudaMemcpyDeviceToHost,
                     ctx->stream));
  int st = 0;
  CKS(read_status(ctx, &st));
  return status_to_result(ctx, st);
}

static ulisse_status upload_M_prior(ulisse_ctx* ctx, const double* M, const double* prior,
                                    const double** Md, const double** pd) {
  const int p = ctx->d + 2;
  *Md = nullptr;
  *pd = nullptr;
  if (M) {
    for (int i = 0; i < p * p; ++i)
      if (!std::isfinite(M[i])) return fail(ctx, ULISSE_ERR_ARG, "M not finite");
    CK(cudaMemcpyAsync(ctx->M_dev, M, sizeof(double) * p * p, cudaMemcpyHostToDevice,
                       ctx->stream));
    ctx->m_identity = false;
    *Md = ctx->M_dev;
  }
  if (prior) {
    if (!finite_psi(prior, p)) return fail(ctx, ULISSE_ERR_ARG, "prior_grad not finite");
    CK(cudaMemcpyAsync(ctx->prior_dev, prior, sizeof(double) * p, cudaMemcpyHostToDevice,
                       ctx->stream));
    ctx->prior_zero = false;
    *pd = ctx->prior_dev;
  }
  return ULISSE_OK;
}

ulisse_status ulisse_sgld_step(ulisse_ctx* ctx, double* psi_inout, double eps_t, const double* M,
                               const double* prior_grad, unsigned long long step, double* g_out) {
  if (!ctx) return ULISSE_ERR_ARG;
  if (ctx->batched) return fail(ctx, ULISSE_ERR_ARG, "batched context: use the ulisse_batch_* calls");
  if (!(eps_t >= 0.0) || !std::isfinite(eps_t)) return fail(ctx, ULISSE_ERR_ARG, "eps_t invalid");
  CKS(set_psi_host(ctx, psi_inout));
  const double *Md, *pd;
  CKS(upload_M_prior(ctx, M, prior_grad, &Md, &pd));
  CK(cudaMemsetAsync(ctx->status_dev, 0, sizeof(int), ctx->stream));
  if (graph_usable(ctx)) {
    // one launch of the step graph; the step size travels through the device
    CKS(graph_alloc(ctx));
    CK(cudaMemcpyAsync(ctx->eps_one, &eps_t, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CKS(graph_prepare(ctx, M, prior_grad, step, ctx->eps_one, nullptr));
    CK(cudaGraphLaunch(ctx->step_exec, ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_gstat, ctx->gstat, sizeof(long long) * 4, cudaMemcpyDeviceToHost,
                       ctx->stream));
    int st = 0;
    CKS(read_status(ctx, &st));
    graph_fold_counters(ctx, 1);
    ulisse_status r = status_to_result(ctx, st);
    if (r == ULISSE_ERR_ARG) return r;
    CK(cudaMemcpyAsync(psi_inout, ctx->psi_dev, sizeof(double) * (ctx->d + 2),
                       cudaMemcpyDeviceToHost, ctx->stream));
    if (g_out)
      CK(cudaMemcpyAsync(g_out, ctx->g_dev, sizeof(double) * (ctx->d + 2),
                         cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return r;
  }
  CKS(grad_core(ctx, step));
  sgld_kernel<<<1, 32, 0, ctx->stream>>>(ctx->psi_dev, ctx->g_dev, Md, pd, nullptr, eps_t,
                                         ctx->d + 2, ctx->cfg.seed, step, nullptr,
                                         ctx->status_dev);
  CK(cudaGetLastError());
  ctx->launches++;
  int st = 0;
  CKS(read_status(ctx, &st));
  ulisse_status r = status_to_result(ctx, st);
  if (r == ULISSE_ERR_ARG) return r;
  CK(cudaMemcpyAsync(psi_inout, ctx->psi_dev, sizeof(double) * (ctx->d + 2),
                     cudaMemcpyDeviceToHost, ctx->stream));
  if (g_out)
    CK(cudaMemcpyAsync(g_out, ctx->g_dev, sizeof(double) * (ctx->d + 2), cudaMemcpyDeviceToHost,
                       ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return r;
}

// ---------------------------------------------------------------------------------------
// One SGLD step as a CUDA graph (ulisse_sgld_chain).  The data-dependent CG loop becomes a
// WHILE node whose body is the compaction kernel and a SWITCH node with one branch per live
// column count: branch k holds exactly the launches the host loop makes for k + 1 live
// columns (same instantiations, same splits), so a graph step and a host-loop step give the
// same results.  The step number, step size and trace slot come from a device chain slot.
// ---------------------------------------------------------------------------------------
static void graph_release(ulisse_ctx* ctx) {
  if (ctx->step_exec) cudaGraphExecDestroy(ctx->step_exec);
  if (ctx->step_graph) cudaGraphDestroy(ctx->step_graph);
  ctx->step_exec = nullptr;
  ctx->step_graph = nullptr;
  ctx->graph_key = -1;
}

extern "C++" {
template <typename T>
static void cg_round_launches(ulisse_ctx* ctx, CgArgs<T>& a, int nl) {
  const long long target = std::max(1, (2 * ctx->num_sms + nl - 1) / nl);
  long long ch = std::max<long long>((ctx->n + target - 1) / target, 2048);
  ch = std::max<long long>(ch, (ctx->n + kMaxCgChunks - 1) / kMaxCgChunks);
  ch = (ch + 255) / 256 * 256;
  a.chunk = ch;
  a.nchunk = (int)((ctx->n + ch - 1) / ch);
  const dim3 grid(a.nchunk, nl);
  cg_dot_kernel<T><<<grid, kCgChunkNT, 0, ctx->stream>>>(a);
  cg_update_kernel<T><<<grid, kCgChunkNT, 0, ctx->stream>>>(a);
  cg_finish_kernel<T><<<grid, kCgChunkNT, 0, ctx->stream>>>(a);
}

template <typename T>
static ulisse_status graph_capture_body(ulisse_ctx* ctx, int s0_cols) {
  const int nr = ctx->cfg.n_probes, R = 1 + nr, p = ctx->d + 2;
  CKS(prescale(ctx));
  CK(cudaMemcpyAsync(ctx->B, ctx->y, ctx->ldn * ctx->esz, cudaMemcpyDeviceToDevice,
                     ctx->stream));
  dim3 pg((unsigned)std::min<long long>((ctx->n + 255) / 256, 2LL * ctx->num_sms), nr);
  probes_kernel<T><<<pg, 256, 0, ctx->stream>>>((T*)ctx->B, ctx->ldn, ctx->n, nr,
                                                ctx->cfg.probe_kind, ctx->cfg.seed, 0,
                                                ctx->chain, ctx->cfg.probe_refresh);
  CK(cudaGetLastError());
  const bool warm = ctx->cfg.warm_start_probes != 0;
  if (s0_cols > 0) {
    ws_x0(ctx->wsb, ctx->psi_dev, true, (const float*)ctx->xhat, ctx->DP, ctx->n, ctx->params,
          ctx->ws_c, (float*)ctx->S, ctx->num_sms, ctx->stream);
    CK(cudaGetLastError());
    if (!warm) {
      CK(cudaMemsetAsync((char*)ctx->S + ctx->ldn * ctx->esz, 0,
                         (size_t)(R - 1) * ctx->ldn * ctx->esz, ctx->stream));
      CK(cudaMemsetAsync((char*)ctx->KD + (size_t)s0_cols * ctx->ldn * ctx->esz, 0,
                         (size_t)(R - s0_cols) * ctx->ldn * ctx->esz, ctx->stream));
      CKS(run_kmv(ctx, ctx->S, ctx->iota, s0_cols, ctx->KD, ctx->iota, kModeK, -1));
    }
  }
  if (warm)
    CKS(run_kmv(ctx, ctx->S, ctx->warm_map + (s0_cols > 0 ? ctx->cap : 0), R, ctx->KD,
                ctx->iota, kModeK, -1));
  CgArgs<T> a = cg_args<T>(ctx, s0_cols > 0 && !warm, 0);
  a.cs = ctx->chain;
  if (warm) {
    a.warm_refresh = ctx->cfg.probe_refresh;
    a.y_learned = s0_cols > 0 ? 1 : 0;
  }
  CK(launch_cg_init(a, R, ctx->num_sms, ctx->stream));
  CK(cudaMemsetAsync(ctx->n_live_dev, 0, sizeof(int), ctx->stream));
  CK(cudaMemsetAsync(ctx->gstat + 3, 0, sizeof(long long), ctx->stream));

  // WHILE node on the outer graph
  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  CK(cudaStreamGetCaptureInfo(ctx->stream, &cst, nullptr, &g, &deps, nullptr, &ndeps));
  cudaGraphConditionalHandle h_loop, h_branch;
  CK(cudaGraphConditionalHandleCreate(&h_loop, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams wp = {};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = h_loop;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wnode;
  CK(cudaGraphAddNode(&wnode, g, deps, nullptr, ndeps, &wp));
  CK(cudaStreamUpdateCaptureDependencies(ctx->stream, &wnode, nullptr, 1,
                                         cudaStreamSetCaptureDependencies));
  cudaGraph_t body = wp.conditional.phGraph_out[0];

  // loop body: compaction, then the SWITCH over the live column count
  CK(cudaGraphConditionalHandleCreate(&h_branch, body, (unsigned)R, cudaGraphCondAssignDefault));
  cudaStream_t outer = ctx->stream;
  CK(cudaStreamBeginCaptureToGraph(ctx->cap_stream2, body, nullptr, nullptr, 0,
                                   cudaStreamCaptureModeThreadLocal));
  const int chunk_cols = ctx->mixed ? 64 : kMaxRChunk;
  const int per_chunk = ctx->mixed ? 2 : 1;
  compact_graph_kernel<<<1, 32, 0, ctx->cap_stream2>>>(
      ctx->st, ctx->st_next, R, ctx->live, ctx->n_live_dev, h_loop, h_branch, chunk_cols,
      per_chunk, 3, ctx->cfg.max_iter + 2, ctx->gstat, ctx->status_dev);
  cudaError_t e = cudaGetLastError();
  const cudaGraphNode_t* bdeps = nullptr;
  size_t nbdeps = 0;
  cudaGraph_t bg = nullptr;
  if (e == cudaSuccess)
    e = cudaStreamGetCaptureInfo(ctx->cap_stream2, &cst, nullptr, &bg, &bdeps, nullptr, &nbdeps);
  cudaGraphNodeParams sp = {};
  sp.type = cudaGraphNodeTypeConditional;
  sp.conditional.handle = h_branch;
  sp.conditional.type = cudaGraphCondTypeSwitch;
  sp.conditional.size = (unsigned)R;
  cudaGraphNode_t snode;
  if (e == cudaSuccess) e = cudaGraphAddNode(&snode, bg, bdeps, nullptr, nbdeps, &sp);
  if (e == cudaSuccess)
    e = cudaStreamUpdateCaptureDependencies(ctx->cap_stream2, &snode, nullptr, 1,
                                            cudaStreamSetCaptureDependencies);
  cudaGraph_t tmp = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(ctx->cap_stream2, &tmp);
  CK(e);
  CK(e2);
  // branch k: one CG round with k + 1 live columns
  for (int k = 0; k < R; ++k) {
    CK(cudaStreamBeginCaptureToGraph(ctx->cap_stream2, sp.conditional.phGraph_out[k], nullptr,
                                     nullptr, 0, cudaStreamCaptureModeThreadLocal));
    ctx->stream = ctx->cap_stream2;
    ulisse_status r = run_kmv(ctx, ctx->D, ctx->live, k + 1, ctx->KD, ctx->live, kModeK, -1);
    if (r == ULISSE_OK) cg_round_launches<T>(ctx, a, k + 1);
    ctx->stream = outer;
    const cudaError_t e3 = cudaGetLastError();
    const cudaError_t e4 = cudaStreamEndCapture(ctx->cap_stream2, &tmp);
    CKS(r);
    CK(e3);
    CK(e4);
  }
  // after the loop: the second estimate of K^{-1} y as the right factor, gradient, update
  if (warm) CK(cudaMemsetAsync(ctx->warm_valid, 0x01, sizeof(int), ctx->stream));
  CK(cudaMemcpyAsync(ctx->B, (char*)ctx->SE + ctx->ldn * ctx->esz, ctx->ldn * ctx->esz,
                     cudaMemcpyDeviceToDevice, ctx->stream));
  CKS(run_grad(ctx, R));
  sgld_chain_kernel<<<1, 32, 0, ctx->stream>>>(ctx->psi_dev, ctx->g_dev, ctx->M_dev,
                                               ctx->prior_dev, p, ctx->cfg.seed, ctx->chain,
                                               ctx->status_dev);
  CK(cudaGetLastError());
  return ULISSE_OK;
}

}  // extern "C++"

static ulisse_status graph_build(ulisse_ctx* ctx, int s0_cols) {
  graph_release(ctx);
  const int nr = ctx->cfg.n_probes, R = 1 + nr;
  CKS(ensure_columns(ctx, R, R + 1));
  CKS(ensure_grad_maps(ctx, nr));
  if (ctx->meta_grad_R != R) {
    std::vector<int> n_est(R, 1);
    n_est[0] = 2;
    int tot = 0;
    CKS(upload_meta(ctx, R, n_est.data(), &tot));
    ctx->meta_grad_R = R;
  }
  if (!ctx->cap_stream) {
    CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&ctx->cap_stream2, cudaStreamNonBlocking));
  }
  // size every launch's scratch first: nothing may allocate inside the capture
  const bool prof = ctx->prof;
  ctx->prof = false;
  ctx->planning = true;
  ulisse_status r = ULISSE_OK;
  for (int k = 1; k <= R && r == ULISSE_OK; ++k)
    r = run_kmv(ctx, ctx->D, ctx->live, k, ctx->KD, ctx->live, kModeK, -1);
  if (r == ULISSE_OK && s0_cols > 0)
    r = run_kmv(ctx, ctx->S, ctx->iota, s0_cols, ctx->KD, ctx->iota, kModeK, -1);
  const bool warm = ctx->cfg.warm_start_probes != 0;
  if (r == ULISSE_OK && warm)
    r = run_kmv(ctx, ctx->S, ctx->warm_map + (s0_cols > 0 ? ctx->cap : 0), R, ctx->KD, ctx->iota,
                kModeK, -1);
  if (r == ULISSE_OK) r = run_grad(ctx, R);
  ctx->planning = false;
  if (r != ULISSE_OK) {
    ctx->prof = prof;
    return r;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  cudaStream_t saved = ctx->stream;
  ctx->stream = ctx->cap_stream;
  ctx->capturing = true;
  cudaError_t e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) r = ctx->f64 ? graph_capture_body<double>(ctx, s0_cols)
                                     : graph_capture_body<float>(ctx, s0_cols);
  cudaGraph_t graph = nullptr;
  const cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(ctx->cap_stream, &graph) : e;
  ctx->stream = saved;
  ctx->capturing = false;
  ctx->prof = prof;
  if (r != ULISSE_OK) {
    if (graph) cudaGraphDestroy(graph);
    return r;
  }
  if (e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(ctx, ULISSE_ERR_CUDA, std::string("step graph capture: ") + cudaGetErrorString(e2));
  }
  ctx->step_graph = graph;
  CK(cudaGraphInstantiate(&ctx->step_exec, graph, 0));
  // what one launch does outside the CG loop (the loop's share is counted on the device)
  const long long kmv_per = ctx->mixed ? 2 : 1, kmv_cols = ctx->mixed ? 64 : kMaxRChunk;
  const int init_cols = warm ? R : s0_cols;   // columns of the product K s_0
  // prescale (+ the tensor-core images), probes, the CG start, the gradient pass (+ its
  // operand images), the update, the learned start's two kernels, the product K s_0
  ctx->graph_launches_fixed = (ctx->mixed ? 3 : 1) + 1 + cg_init_launch_count(ctx->n, R, ctx->num_sms) +
      (ctx->mixed ? 3 : 1) + 1 + (s0_cols > 0 ? 2 : 0) +
      (init_cols > 0 ? kmv_per * ((init_cols + kmv_cols - 1) / kmv_cols) : 0);
  ctx->graph_entries_fixed = (double)ctx->n * (double)ctx->n * (double)(R + init_cols);
  ctx->graph_rounds_fixed = init_cols > 0 ? 1 : 0;
  ctx->graph_key = s0_cols;
  return ULISSE_OK;
}

static bool graph_usable(const ulisse_ctx* ctx) {
  return ctx->graph_enabled && !ctx->prof && !ctx->ws_record && !(ctx->cfg.pcg_delta > 0.0);
}

static ulisse_status graph_alloc(ulisse_ctx* ctx) {
  if (ctx->chain) return ULISSE_OK;
  CKS(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->chain), sizeof(ChainSlot)));
  CKS(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->gstat), sizeof(long long) * 4));
  CKS(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->eps_one), sizeof(double)));
  if (cudaMallocHost(&ctx->h_gstat, sizeof(long long) * 4) != cudaSuccess)
    return fail(ctx, ULISSE_ERR_NOMEM, "cudaMallocHost failed");
  return ULISSE_OK;
}

// Identity M / zero prior in the context's buffers when not given (the graph always reads
// them), the chain slot for the coming launches, and the graph itself if it is stale.
static ulisse_status graph_prepare(ulisse_ctx* ctx, const double* M, const double* prior,
                                   unsigned long long step0, const double* eps_dev,
                                   double* trace_dev) {
  const int p = ctx->d + 2;
  if (!M && !ctx->m_identity) {
    std::vector<double> I((size_t)p * p, 0.0);
    for (int i = 0; i < p; ++i) I[(size_t)i * p + i] = 1.0;
    CK(cudaMemcpyAsync(ctx->M_dev, I.data(), sizeof(double) * p * p, cudaMemcpyHostToDevice,
                       ctx->stream));
    ctx->m_identity = true;
  }
  if (!prior && !ctx->prior_zero) {
    CK(cudaMemsetAsync(ctx->prior_dev, 0, sizeof(double) * p, ctx->stream));
    ctx->prior_zero = true;
  }
  CKS(graph_alloc(ctx));
  const ChainSlot cs{0, step0, eps_dev, trace_dev};
  CK(cudaMemcpyAsync(ctx->chain, &cs, sizeof(ChainSlot), cudaMemcpyHostToDevice, ctx->stream));
  const int s0 = (ctx->ws_use && ctx->ws_trained) ? 1 : 0;
  if (ctx->graph_key != s0) CKS(graph_build(ctx, s0));
  return ULISSE_OK;
}

// Host counters after n_steps graph launches (h_gstat already copied back and synchronised).
static void graph_fold_counters(ulisse_ctx* ctx, int n_steps) {
  const long long* gs = ctx->h_gstat;
  ctx->mvp_rounds += n_steps * ctx->graph_rounds_fixed + gs[0];
  ctx->entry_rhs += n_steps * ctx->graph_entries_fixed + (double)ctx->n * (double)ctx->n * gs[1];
  ctx->launches += n_steps * ctx->graph_launches_fixed + gs[2];
  cudaMemsetAsync(ctx->gstat, 0, sizeof(long long) * 3, ctx->stream);
}

ulisse_status ulisse_set_graph(ulisse_ctx* ctx, int enable) {
  if (!ctx) return ULISSE_ERR_ARG;
  ctx->graph_enabled = enable != 0;
  return ULISSE_OK;
}

ulisse_status ulisse_sgld_chain(ulisse_ctx* ctx, double* psi_dev, const double* eps_dev,
                                int n_steps, const double* M, const double* prior_grad,
                                unsigned long long step0, double* trace_dev) {
  if (!ctx) return ULISSE_ERR_ARG;
  if (ctx->batched) return fail(ctx, ULISSE_ERR_ARG, "batched context: use the ulisse_batch_* calls");
  if (!psi_dev || !eps_dev || n_steps < 0) return fail(ctx, ULISSE_ERR_ARG, "bad chain arguments");
  const int p = ctx->d + 2;
  const double *Md, *pd;
  CKS(upload_M_prior(ctx, M, prior_grad, &Md, &pd));
  CK(cudaMemsetAsync(ctx->status_dev, 0, sizeof(int), ctx->stream));
  CK(cudaMemcpyAsync(ctx->psi_dev, psi_dev, sizeof(double) * p, cudaMemcpyDeviceToDevice,
                     ctx->stream));
  // Each step as one launch of the step graph, unless the event timing is on (it times
  // single launches) or warm-start pairs are being recorded (host-side bookkeeping).
  if (graph_usable(ctx) && n_steps > 0) {
    CKS(graph_prepare(ctx, M, prior_grad, step0, eps_dev, trace_dev));
    for (int k = 0; k < n_steps; ++k) CK(cudaGraphLaunch(ctx->step_exec, ctx->stream));
    CK(cudaMemcpyAsync(psi_dev, ctx->psi_dev, sizeof(double) * p, cudaMemcpyDeviceToDevice,
                       ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_gstat, ctx->gstat, sizeof(long long) * 4, cudaMemcpyDeviceToHost,
                       ctx->stream));
    int st = 0;
    CKS(read_status(ctx, &st));
    graph_fold_counters(ctx, n_steps);
    return status_to_result(ctx, st);
  }
  for (int k = 0; k < n_steps; ++k) {
    const unsigned long long step = step0 + (unsigned long long)k;
    CKS(grad_core(ctx, step));
    sgld_kernel<<<1, 32, 0, ctx->stream>>>(ctx->psi_dev, ctx->g_dev, Md, pd, eps_dev + k, 0.0, p,
                                           ctx->cfg.seed, step,
                                           trace_dev ? trace_dev + (long long)k * p : nullptr,
                                           ctx->status_dev);
    CK(cudaGetLastError());
    ctx->launches++;
  }
  CK(cudaMemcpyAsync(psi_dev, ctx->psi_dev, sizeof(double) * p, cudaMemcpyDeviceToDevice,
                     ctx->stream));
  int st = 0;
  CKS(read_status(ctx, &st));
  return status_to_result(ctx, st);
}

// ---------------------------------------------------------------------------------------
// Learned warm start
// ---------------------------------------------------------------------------------------
static uint64_t splitmix64(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// k distinct indices of [0, n) (Floyd's sampling), sorted.
static std::vector<int> sample_distinct(long long n, int k, uint64_t& state) {
  std::vector<int> out;
  std::vector<char> used;
  if (n <= 50000000) used.assign((size_t)n, 0);
  for (long long j = n - k; j < n; ++j) {
    const long long t = (long long)(splitmix64(state) % (uint64_t)(j + 1));
    bool taken = false;
    if (!used.empty()) taken = used[(size_t)t];
    else taken = std::find(out.begin(), out.end(), (int)t) != out.end();
    const long long pick = taken ? j : t;
    out.push_back((int)pick);
    if (!used.empty()) used[(size_t)pick] = 1;
  }
  std::sort(out.begin(), out.end());
  return out;
}

static ulisse_status ws_alloc(ulisse_ctx* ctx, void** p, size_t bytes) {
  CKS(dev_alloc(ctx, p, bytes));
  ctx->ws_allocs.push_back(*p);
  return ULISSE_OK;
}

ulisse_status ulisse_ws_init(ulisse_ctx* ctx, const ulisse_ws_config* cfg) {
  if (!ctx) return ULISSE_ERR_ARG;
  if (!cfg) return fail(ctx, ULISSE_ERR_ARG, "cfg is null");
  if (ctx->batched) return fail(ctx, ULISSE_ERR_ARG, "batched context: use the ulisse_batch_* calls");
  if (ctx->f64) return fail(ctx, ULISSE_ERR_ARG, "the warm start needs an FP32 or mixed context");
  if (ctx->ws_ready) return fail(ctx, ULISSE_ERR_ARG, "warm start already initialised");
  const int A = cfg->n_anchors, H = cfg->hidden, m = cfg->n_rows, P = cfg->max_pairs;
  const int d = ctx->d, p = d + 2;
  if (A < 1 || A > ctx->n || H < 1 || H > 4096 || m < 1 || m > 8192 || P < 1 ||
      (long long)A * (ctx->DP + 1) > 12288 || !(cfg->ridge >= 0.0) || !std::isfinite(cfg->ridge))
    return fail(ctx, ULISSE_ERR_ARG, "warm start sizes out of range");
  WsBuffers& b = ctx->wsb;
  b.p = p; b.H = H; b.A = A; b.m = m; b.max_pairs = P; b.d = d; b.n = ctx->n;
  b.ridge = (float)cfg->ridge;
  b.seed = cfg->seed;
  ctx->ws_seed = cfg->seed;
  uint64_t st = cfg->seed ^ 0x5A17A11CE0FF5E75ull;
  const std::vector<int> anch = sample_distinct(ctx->n, A, st);
  {
    // split the j range of the recording product so that about two CTAs run per SM
    const long long tiles = (long long)((A + 63) / 64) * ((m + 63) / 64);
    long long ns = std::max<long long>(1, (2LL * ctx->num_sms + tiles - 1) / tiles);
    ns = std::min<long long>(ns, std::max<long long>(1, ctx->n / 256));
    b.n_split = (int)std::min<long long>(ns, 32);
  }
  const long long np = ws_param_count(p, H, A);
  std::vector<float> w((size_t)np, 0.f);
  auto normal = [&]() {
    const double u1 = ((splitmix64(st) >> 11) + 1.0) * (1.0 / 9007199254740993.0);
    const double u2 = (splitmix64(st) >> 11) * (1.0 / 9007199254740992.0);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  };
  for (long long k = 0; k < (long long)p * H; ++k) w[k] = (float)(normal() / std::sqrt((double)p));
  const long long oW2 = (long long)p * H + H;
  for (long long k = 0; k < (long long)H * H; ++k) w[oW2 + k] = (float)(normal() / std::sqrt((double)H));
  const int nlb = ws_loss_blocks(m);
  ctx->ws_loss_blocks = nlb;
  void* q = nullptr;
#define WSA(field, bytes) do { CKS(ws_alloc(ctx, &q, (bytes))); b.field = reinterpret_cast<decltype(b.field)>(q); } while (0)
  WSA(anch, sizeof(int) * A);
  WSA(w, sizeof(float) * np);
  WSA(g, sizeof(float) * np);
  WSA(adam_m, sizeof(float) * np);
  WSA(adam_v, sizeof(float) * np);
  WSA(wb, sizeof(__nv_bfloat16) * np);
  WSA(pair_psi, sizeof(float) * (size_t)P * p);
  WSA(pair_rows, sizeof(int) * (size_t)P * m);
  WSA(pair_y, sizeof(float) * (size_t)P * m);
  WSA(pair_M, sizeof(float) * (size_t)P * m * A);
  WSA(cross, sizeof(float) * (size_t)ctx->n * A);
  WSA(Mpart, sizeof(float) * (size_t)b.n_split * m * A);
  WSA(mu, sizeof(float) * p);
  WSA(sd, sizeof(float) * p);
  WSA(idx, sizeof(int) * P);
  WSA(Z, sizeof(float) * (size_t)P * p);
  WSA(H1, sizeof(float) * (size_t)P * H);
  WSA(H2, sizeof(float) * (size_t)P * H);
  WSA(dH, sizeof(float) * (size_t)P * H);
  WSA(dA, sizeof(float) * (size_t)P * H);
  WSA(C, sizeof(float) * (size_t)P * A);
  WSA(dC, sizeof(float) * (size_t)P * A);
  WSA(R, sizeof(float) * (size_t)P * m);
  WSA(loss_part, sizeof(double) * (size_t)P * nlb);
  WSA(G, sizeof(double) * (size_t)A * A);
  WSA(Ginv, sizeof(double) * (size_t)A * A);
  WSA(gb, sizeof(double) * (size_t)A);
  WSA(P, sizeof(float) * (size_t)A * A);
  WSA(gbf, sizeof(float) * (size_t)A);
  WSA(wt, sizeof(float) * (size_t)(H + 1) * A);
  WSA(gt, sizeof(float) * (size_t)(H + 1) * A);
  WSA(flag, sizeof(int));
  WSA(w_best, sizeof(float) * np);
  WSA(wt_best, sizeof(float) * (size_t)(H + 1) * A);
#undef WSA
  CKS(ws_alloc(ctx, &q, sizeof(float) * A));
  ctx->ws_c = static_cast<float*>(q);
  CK(cudaMemcpyAsync(b.anch, anch.data(), sizeof(int) * A, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(b.w, w.data(), sizeof(float) * np, cudaMemcpyHostToDevice, ctx->stream));
  std::vector<float> ones(p, 1.f);
  CK(cudaMemcpyAsync(b.sd, ones.data(), sizeof(float) * p, cudaMemcpyHostToDevice, ctx->stream));
  ws_to_bf16(b, ctx->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->ws_ready = true;
  return ULISSE_OK;
}

ulisse_status ulisse_ws_set(ulisse_ctx* ctx, int record, int use) {
  if (!ctx) return ULISSE_ERR_ARG;
  if (!ctx->ws_ready) return fail(ctx, ULISSE_ERR_ARG, "warm start not initialised");
  ctx->ws_record = record != 0;
  ctx->ws_use = use != 0;
  return ULISSE_OK;
}

static ulisse_status ws_sum_loss(ulisse_ctx* ctx, int B, double* loss) {
  std::vector<double> parts((size_t)B * ctx->ws_loss_blocks);
  CK(cudaMemcpyAsync(parts.data(), ctx->wsb.loss_part, sizeof(double) * parts.size(),
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  double t = 0.0;
  for (double v : parts) t += v;
  if (loss) *loss = t / ((double)B * ctx->wsb.m);
  return ULISSE_OK;
}

ulisse_status ulisse_ws_train(ulisse_ctx* ctx, int steps, int batch, double lr, double* loss) {
  if (!ctx) return ULISSE_ERR_ARG;
  if (!ctx->ws_ready || ctx->ws_pairs < 1)
    return fail(ctx, ULISSE_ERR_ARG, "no recorded pairs to train on");
  if (steps < 0 || (steps > 0 && (batch < 1 || batch > ctx->wsb.max_pairs || !(lr > 0.0) ||
                                  !std::isfinite(lr))))
    return fail(ctx, ULISSE_ERR_ARG, "bad training arguments");
  WsBuffers& b = ctx->wsb;
  const int T = ctx->ws_pairs;
  ws_standardize(b, T, ctx->stream);
  ctx->ws_standardized = true;
  // Start from the pooled least-squares constant with the output layer whitened, then take
  // Adam steps in the whitened coordinates (moments restart with each call).
  if (!ws_whiten(b, T, ctx->stream)) {
    CK(cudaGetLastError());
    return fail(ctx, ULISSE_ERR_BREAKDOWN,
                "warm start: pooled normal matrix is not positive definite (raise ridge)");
  }
  CK(cudaGetLastError());
  ctx->launches += 6;
  const long long np = ws_param_count(b.p, b.H, b.A);
  const long long nl = (long long)(b.H + 1) * b.A;
  CK(cudaMemsetAsync(b.adam_m, 0, sizeof(float) * np, ctx->stream));
  CK(cudaMemsetAsync(b.adam_v, 0, sizeof(float) * np, ctx->stream));
  ctx->ws_t = 0;
  // Every eighth pair is held out once there are at least eight: minibatches come from the
  // rest, and the weights with the lowest held-out loss (the pooled start included) are kept.
  std::vector<int> train, val;
  for (int t = 0; t < T; ++t) ((T >= 8 && t % 8 == 7) ? val : train).push_back(t);
  const bool validate = !val.empty() && steps > 0;
  auto val_loss = [&](double* out) -> ulisse_status {
    CK(cudaMemcpyAsync(b.idx, val.data(), sizeof(int) * val.size(), cudaMemcpyHostToDevice,
                       ctx->stream));
    ws_loss_grad(b, (int)val.size(), ctx->ws_loss_blocks, ctx->stream);
    CK(cudaGetLastError());
    ctx->launches += 16;
    return ws_sum_loss(ctx, (int)val.size(), out);
  };
  auto save_best = [&]() -> ulisse_status {
    CK(cudaMemcpyAsync(b.w_best, b.w, sizeof(float) * np, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(b.wt_best, b.wt, sizeof(float) * nl, cudaMemcpyDeviceToDevice,
                       ctx->stream));
    return ULISSE_OK;
  };
  double best = 0.0, cur = 0.0, last = 0.0;
  if (validate) {
    CKS(val_loss(&best));
    CKS(save_best());
  }
  constexpr int kEvalEvery = 25;
  std::vector<int> idx(std::max(batch, 1));
  for (int it = 0; it < steps; ++it) {
    uint64_t st = ctx->ws_seed ^ (0xB5AD4ECEDA1CE2A9ull * (++ctx->ws_batches));
    for (int k = 0; k < batch; ++k)
      idx[k] = train[(size_t)(splitmix64(st) % (uint64_t)train.size())];
    CK(cudaMemcpyAsync(b.idx, idx.data(), sizeof(int) * batch, cudaMemcpyHostToDevice,
                       ctx->stream));
    ws_loss_grad(b, batch, ctx->ws_loss_blocks, ctx->stream);
    ws_adam_whitened(b, (float)lr, ++ctx->ws_t, ctx->stream);
    CK(cudaGetLastError());
    ctx->launches += 20;
    if (!validate && it == steps - 1) CKS(ws_sum_loss(ctx, batch, &last));
    if (validate && ((it + 1) % kEvalEvery == 0 || it == steps - 1)) {
      CKS(val_loss(&cur));
      if (cur < best) {
        best = cur;
        CKS(save_best());
      }
    }
  }
  if (validate) {
    CK(cudaMemcpyAsync(b.w, b.w_best, sizeof(float) * np, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(b.wt, b.wt_best, sizeof(float) * nl, cudaMemcpyDeviceToDevice,
                       ctx->stream));
  }
  if (loss) *loss = validate ? best : last;
  ws_to_bf16(b, ctx->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->ws_trained = true;
  return ULISSE_OK;
}

ulisse_status ulisse_ws_loss_grad(ulisse_ctx* ctx, double* loss, float* grad) {
  if (!ctx) return ULISSE_ERR_ARG;
  if (!ctx->ws_ready || ctx->ws_pairs < 1)
    return fail(ctx, ULISSE_ERR_ARG, "no recorded pairs");
  WsBuffers& b = ctx->wsb;
  if (!ctx->ws_standardized) {
    ws_standardize(b, ctx->ws_pairs, ctx->stream);
    ctx->ws_standardized = true;
  }
  const int T = ctx->ws_pairs;
  std::vector<int> idx(T);
  for (int k = 0; k < T; ++k) idx[k] = k;
  CK(cudaMemcpyAsync(b.idx, idx.data(), sizeof(int) * T, cudaMemcpyHostToDevice, ctx->stream));
  ws_loss_grad(b, T, ctx->ws_loss_blocks, ctx->stream);
  CK(cudaGetLastError());
  CKS(ws_sum_loss(ctx, T, loss));
  if (grad)
    CK(cudaMemcpyAsync(grad, b.g, sizeof(float) * ws_param_count(b.p, b.H, b.A),
                       cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return ULISSE_OK;
}

ulisse_status ulisse_ws_export(ulisse_ctx* ctx, ulisse_ws_state* out) {
  if (!ctx || !out) return ULISSE_ERR_ARG;
  if (!ctx->ws_ready) return fail(ctx, ULISSE_ERR_ARG, "warm start not initialised");
  const WsBuffers& b = ctx->wsb;
  const long long np = ws_param_count(b.p, b.H, b.A);
  auto cp = [&](void* dst, const void* src, size_t bytes) -> ulisse_status {
    if (dst) CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    return ULISSE_OK;
  };
  CKS(cp(out->weights, b.w, sizeof(float) * np));
  CKS(cp(out->anchors, b.anch, sizeof(int) * b.A));

  CKS(cp(out->mu, b.mu, sizeof(float) * b.p));
  CKS(cp(out->sd, b.sd, sizeof(float) * b.p));
  CKS(cp(out->pair_psi, b.pair_psi, sizeof(float) * (size_t)b.max_pairs * b.p));
  CKS(cp(out->pair_rows, b.pair_rows, sizeof(int) * (size_t)b.max_pairs * b.m));
  CK(cudaStreamSynchronize(ctx->stream));
  out->n_pairs = ctx->ws_pairs;
  out->n_params = np;
  return ULISSE_OK;
}

ulisse_status ulisse_ws_x0(ulisse_ctx* ctx, const double* psi, int bf16, float* x0) {
  if (!ctx) return ULISSE_ERR_ARG;
  if (!ctx->ws_ready || !x0) return fail(ctx, ULISSE_ERR_ARG, "warm start not initialised or x0 null");
  CKS(set_psi_host(ctx, psi));
  CKS(prescale(ctx));
  ws_x0(ctx->wsb, ctx->psi_dev, bf16 != 0, (const float*)ctx->xhat, ctx->DP, ctx->n, ctx->params,
        ctx->ws_c, x0, ctx->num_sms, ctx->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->stream));
  return ULISSE_OK;
}

// ---------------------------------------------------------------------------------------
// Batched contexts: many independent problems, O(n^2) passes in one persistent launch
// ---------------------------------------------------------------------------------------
#define BATCHED_ONLY(ctx)                                                                 \
  do {                                                                                    \
    if (!(ctx)) return ULISSE_ERR_ARG;                                                    \
    if (!(ctx)->batched) return fail((ctx), ULISSE_ERR_ARG, "not a batched context");     \
  } while (0)

ulisse_status ulisse_create_batched(ulisse_ctx** out, int n_problems, const long long* n,
                                    const int* d, const float* const* X, const float* const* y,
                                    const ulisse_config* cfg, void* stream) {
  if (!out) return fail(nullptr, ULISSE_ERR_ARG, "out is null");
  *out = nullptr;
  if (n_problems < 1 || n_problems > 4096 || !n || !d || !X || !y || !cfg)
    return fail(nullptr, ULISSE_ERR_ARG, "bad batch description");
  if (check_cfg(cfg) != ULISSE_OK) return fail(nullptr, ULISSE_ERR_ARG, "invalid config");
  if (cfg->precision != ULISSE_PREC_FP32 && cfg->precision != ULISSE_PREC_MIXED)
    return fail(nullptr, ULISSE_ERR_ARG, "batched contexts run the FP32 or the mixed path");
  if (cfg->n_probes > 16) return fail(nullptr, ULISSE_ERR_ARG, "batched contexts take n_probes <= 16");
  for (int b = 0; b < n_problems; ++b)
    if (d[b] < 1 || d[b] > kBatchMaxDP) return fail(nullptr, ULISSE_ERR_ARG, "batched contexts take d <= 8");
  ulisse_ctx* ctx = new ulisse_ctx();
  ctx->stream = (cudaStream_t)stream;
  ctx->cfg = *cfg;
  ctx->batched = true;
  auto bail = [&](ulisse_status s) {
    g_create_error = ctx->err;
    ulisse_destroy(ctx);
    return s;
  };
  if (cudaGetDevice(&ctx->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device) !=
          cudaSuccess) {
    ctx->err = "no CUDA device";
    return bail(ULISSE_ERR_CUDA);
  }
  int poff = 0;
  for (int b = 0; b < n_problems; ++b) {
    ulisse_config sc = *cfg;
    sc.seed = cfg->seed + (unsigned long long)b;   // problem b draws from its own streams
    ulisse_ctx* sub = nullptr;
    const ulisse_status s = create_impl(&sub, X[b], y[b], n[b], d[b], &sc, stream,
                                        cudaMemcpyDeviceToDevice);
    if (s != ULISSE_OK) {
      ctx->err = "problem " + std::to_string(b) + ": " + g_create_error;
      return bail(s);
    }
    sub->tc_no_aug = true;   // the batched tensor-core K V adds b_j in its epilogue
    ctx->subs.push_back(sub);
    ctx->sub_p_off.push_back(poff);
    poff += d[b] + 2;
    ctx->n += n[b];
  }
  // Work list: one item per (problem, 256-row block), longest rows first.
  std::vector<BatchItem> items;
  int slot = 0;
  for (int b = 0; b < n_problems; ++b) {
    const int nrb = (int)((n[b] + kBatchBM - 1) / kBatchBM);
    for (int rb = 0; rb < nrb; ++rb) items.push_back(BatchItem{b, rb, slot + rb, 0});
    slot += nrb;
  }
  std::stable_sort(items.begin(), items.end(), [&](const BatchItem& a, const BatchItem& c) {
    return n[a.prob] > n[c.prob];
  });
  ctx->b_n_items = (int)items.size();
  ulisse_status s;
  if ((s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->b_items), sizeof(BatchItem) * items.size())) ||
      (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->b_kdesc), sizeof(BatchKmvDesc) * n_problems)) ||
      (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->b_gdesc), sizeof(BatchGradDesc) * n_problems)) ||
      (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->b_queue), sizeof(int))) ||
      (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->b_nlive), sizeof(int) * n_problems)) ||
      (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->b_rcount), sizeof(int) * n_problems)) ||
      (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->b_gpart), sizeof(double) * kMaxP * items.size())) ||
      (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->b_g), sizeof(double) * kMaxP * n_problems)) ||
      (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->status_dev), sizeof(int))))
    return bail(s);
  if (cfg->precision == ULISSE_PREC_MIXED) {
    // tensor-core K V work list: per problem its 128-row blocks times a split of the j range
    // into ranges of about kTcBatchTiles 32-point tiles; the longest ranges first
    constexpr long long kTcBatchTiles = 256;
    std::vector<int4> tci;
    std::vector<std::pair<long long, int>> order;
    size_t part = 0, cnt = 0;
    for (int b = 0; b < n_problems; ++b) {
      const long long nt = (n[b] + 31) / 32, nrb = (n[b] + 127) / 128;
      int ns = (int)std::min<long long>(64, (nt + kTcBatchTiles - 1) / kTcBatchTiles);
      const long long tps = (nt + ns - 1) / ns;
      ns = (int)((nt + tps - 1) / tps);
      ctx->b_tc_nsplit.push_back(ns);
      ctx->b_tc_part_off.push_back(part);
      ctx->b_tc_cnt_off.push_back(cnt);
      if (ns > 1) part += (size_t)nrb * ns * 32 * 128;
      cnt += (size_t)nrb;
      order.push_back({tps, b});
    }
    std::stable_sort(order.begin(), order.end(),
                     [](const std::pair<long long, int>& a, const std::pair<long long, int>& c) {
                       return a.first > c.first;
                     });
    for (const auto& o : order) {
      const int b = o.second;
      const int nrb = (int)((n[b] + 127) / 128);
      for (int rb = 0; rb < nrb; ++rb)
        for (int sp = 0; sp < ctx->b_tc_nsplit[b]; ++sp) tci.push_back(make_int4(b, rb, sp, 0));
    }
    ctx->b_tc_n_items = (int)tci.size();
    // gradient pass: per width group the (problem, row block, split) items, most tiles first
    // (row block rb visits the tiles [4 rb, ntiles): the symmetric pass)
    std::vector<int4> gti;
    size_t gpart = 0;
    ctx->b_gt_nsplit.assign(n_problems, 1);
    ctx->b_gt_part_off.assign(n_problems, 0);
    for (int dp : {2, 4, 8}) {
      std::vector<int> grp;
      for (int b = 0; b < n_problems; ++b)
        if ((d[b] <= 2 ? 2 : d[b] <= 4 ? 4 : 8) == dp) grp.push_back(b);
      if (grp.empty()) continue;
      std::vector<std::pair<long long, int4>> its;
      for (int li = 0; li < (int)grp.size(); ++li) {
        const int b = grp[li];
        const long long nt = (n[b] + 31) / 32, nrb = (n[b] + 127) / 128;
        const int ns = (int)std::min<long long>(64, (nt + 255) / 256);
        ctx->b_gt_nsplit[b] = ns;
        ctx->b_gt_part_off[b] = gpart;
        gpart += (size_t)nrb * ns * kMaxP;
        for (int rb = 0; rb < nrb; ++rb) {
          const long long span = nt - 4LL * rb, per = (span + ns - 1) / ns;
          for (int sp = 0; sp < ns; ++sp) {
            const long long tiles = std::max<long long>(0, std::min(per, span - sp * per));
            its.push_back({tiles, make_int4(li, rb, sp, 0)});
          }
        }
      }
      std::stable_sort(its.begin(), its.end(),
                       [](const std::pair<long long, int4>& a, const std::pair<long long, int4>& c) {
                         return a.first > c.first;
                       });
      ctx->b_gt_groups.push_back(grp);
      ctx->b_gt_dp.push_back(dp);
      ctx->b_gt_item_off.push_back((int)gti.size());
      ctx->b_gt_item_n.push_back((int)its.size());
      for (const auto& e : its) gti.push_back(e.second);
    }
    if ((s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->b_tc_items), sizeof(int4) * tci.size())) ||
        (s = dev_alloc(ctx, &ctx->b_tc_args, 3 * tc2_batch_args_bytes(n_problems))) ||
        (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->b_tc_part), sizeof(float) * std::max<size_t>(part, 1))) ||
        (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->b_tc_cnt), sizeof(int) * cnt)) ||
        (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->b_gt_items), sizeof(int4) * gti.size())) ||
        (s = dev_alloc(ctx, &ctx->b_gt_args, gt_batch_args_bytes(n_problems))) ||
        (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->b_gt_part), sizeof(double) * gpart)) ||
        (s = dev_alloc(ctx, reinterpret_cast<void**>(&ctx->b_gt_cnt), sizeof(int) * n_problems)))
      return bail(s);
    if (cudaMemsetAsync(ctx->b_tc_cnt, 0, sizeof(int) * cnt, ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->b_gt_cnt, 0, sizeof(int) * n_problems, ctx->stream) != cudaSuccess ||
        cudaMemcpyAsync(ctx->b_gt_items, gti.data(), sizeof(int4) * gti.size(),
                        cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
        cudaMemcpyAsync(ctx->b_tc_items, tci.data(), sizeof(int4) * tci.size(),
                        cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
      ctx->err = "upload of the tensor-core work list failed";
      return bail(ULISSE_ERR_CUDA);
    }
  }
  if (cudaMallocHost(&ctx->b_h_nlive, sizeof(int) * n_problems) != cudaSuccess ||
      cudaMallocHost(&ctx->b_h_status, sizeof(int) * (n_problems + 1)) != cudaSuccess ||
      cudaMallocHost(&ctx->h_status, sizeof(int)) != cudaSuccess) {
    ctx->err = "cudaMallocHost failed";
    return bail(ULISSE_ERR_NOMEM);
  }
  if (cudaMemcpyAsync(ctx->b_items, items.data(), sizeof(BatchItem) * items.size(),
                      cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
      cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    ctx->err = "upload of the work list failed";
    return bail(ULISSE_ERR_CUDA);
  }
  *out = ctx;
  return ULISSE_OK;
}

ulisse_status ulisse_batch_size(const ulisse_ctx* ctx, int* n_problems, int* n_params) {
  if (!ctx || !ctx->batched || !n_problems) return ULISSE_ERR_ARG;
  *n_problems = (int)ctx->subs.size();
  if (n_params) {
    int t = 0;
    for (const ulisse_ctx* sub : ctx->subs) t += sub->d + 2;
    *n_params = t;
  }
  return ULISSE_OK;
}

static ulisse_status batch_set_psi(ulisse_ctx* ctx, const double* psi) {
  if (!psi) return fail(ctx, ULISSE_ERR_ARG, "psi is null");
  for (size_t b = 0; b < ctx->subs.size(); ++b) {
    ulisse_ctx* sub = ctx->subs[b];
    if (!finite_psi(psi + ctx->sub_p_off[b], sub->d + 2))
      return fail(ctx, ULISSE_ERR_ARG, "psi of problem " + std::to_string(b) + " not finite");
    if (set_psi_host(sub, psi + ctx->sub_p_off[b]) != ULISSE_OK) {
      ctx->err = sub->err;
      return ULISSE_ERR_CUDA;
    }
  }
  return ULISSE_OK;
}

// Status words of the batch and of every problem, OR-ed (synchronises the stream).
static ulisse_status batch_read_status(ulisse_ctx* ctx, int* status) {
  const int B = (int)ctx->subs.size();
  CK(cudaMemcpyAsync(ctx->b_h_status + B, ctx->status_dev, sizeof(int), cudaMemcpyDeviceToHost,
                     ctx->stream));
  for (int b = 0; b < B; ++b)
    CK(cudaMemcpyAsync(ctx->b_h_status + b, ctx->subs[b]->status_dev, sizeof(int),
                       cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  int st = 0;
  for (int b = 0; b <= B; ++b) st |= ctx->b_h_status[b];
  *status = st;
  return ULISSE_OK;
}

static ulisse_status batch_clear_status(ulisse_ctx* ctx) {
  CK(cudaMemsetAsync(ctx->status_dev, 0, sizeof(int), ctx->stream));
  for (ulisse_ctx* sub : ctx->subs)
    CK(cudaMemsetAsync(sub->status_dev, 0, sizeof(int), ctx->stream));
  return ULISSE_OK;
}

// A sub-context's failure (its message) reported on the batch.
#define SUBS(ctx, sub, expr)                  \
  do {                                        \
    ulisse_status s_ = (expr);                \
    if (s_ != ULISSE_OK) {                    \
      (ctx)->err = (sub)->err;                \
      return s_;                              \
    }                                         \
  } while (0)

extern "C++" {
// Kernel arguments of the batched tensor-core K V into slot k of b_tc_args (0: the CG
// rounds, 1: K s_0 of warm-started solves, 2: ulisse_batch_kmv): cols(b, sub, L) sets each
// problem's V, vmap, R or R_dev, U and umap; the rest is the problem's own operand buffers.
template <typename Fn>
static ulisse_status batch_tc_upload(ulisse_ctx* ctx, int k, Fn cols) {
  const int B = (int)ctx->subs.size();
  std::vector<TcLaunch> L((size_t)B);
  for (int b = 0; b < B; ++b) {
    ulisse_ctx* sub = ctx->subs[b];
    TcLaunch l{};
    cols(b, sub, l);
    l.ldv = sub->ldn;
    l.ldu = sub->ldn;
    l.xhat = (const float*)sub->xhat;
    l.bneg = sub->bneg;
    l.V_hi = sub->Vt_hi;
    l.V_lo = sub->Vt_lo;
    l.n = sub->n;
    l.DP = sub->DP;
    l.params = sub->params;
    l.nsplit = ctx->b_tc_nsplit[b];
    l.partials = ctx->b_tc_part + ctx->b_tc_part_off[b];
    l.counters = ctx->b_tc_cnt + ctx->b_tc_cnt_off[b];
    l.status = ctx->status_dev;
    l.X_hi = sub->Xt_hi;
    l.X_lo = sub->Xt_lo;
    l.X_off = sub->ld128 * 24;
    L[b] = l;
  }
  CK(tc2_batch_upload_args(L.data(), B, (char*)ctx->b_tc_args + k * tc2_batch_args_bytes(B),
                           ctx->stream));
  return ULISSE_OK;
}

// One batched K V over all problems: the tensor-core launch (slot of its arguments) or the
// persistent FP32 launch (its descriptor array), for at most r_max live columns.
static cudaError_t batch_kv_launch(ulisse_ctx* ctx, int slot, BatchKmvDesc* desc, int r_max,
                                   cudaStream_t st) {
  const int B = (int)ctx->subs.size();
  if (ctx->cfg.precision == ULISSE_PREC_MIXED)
    return launch_kmv_tc2_batch((char*)ctx->b_tc_args + slot * tc2_batch_args_bytes(B), B,
                                ctx->b_tc_items, ctx->b_tc_n_items, r_max, st);
  return launch_kmv_batch(desc, ctx->b_items, ctx->b_n_items, ctx->b_queue,
                          kBatchWidths[batch_width_bucket(r_max)], ctx->num_sms,
                          ctx->status_dev, st);
}

}  // extern "C++"

ulisse_status ulisse_batch_kmv(ulisse_ctx* ctx, const double* psi, const float* const* V, int R,
                               float* const* U) {
  BATCHED_ONLY(ctx);
  if (!V || !U || R < 1 || R > 32) return fail(ctx, ULISSE_ERR_ARG, "V/U null or R out of 1..32");
  const int B = (int)ctx->subs.size();
  for (int b = 0; b < B; ++b)
    if (!V[b] || !U[b]) return fail(ctx, ULISSE_ERR_ARG, "V[b] or U[b] is null");
  CKS(batch_set_psi(ctx, psi));
  CKS(batch_clear_status(ctx));
  graph_release(ctx);   // the products below may reallocate the problems' buffers
  std::vector<BatchKmvDesc> desc(B);
  std::vector<int> rc(B, R);
  double entries = 0.0;
  for (int b = 0; b < B; ++b) {
    ulisse_ctx* sub = ctx->subs[b];
    SUBS(ctx, sub, prescale(sub));
    SUBS(ctx, sub, ensure_columns(sub, R, R));
    CK(cudaMemcpy2DAsync(sub->D, sub->ldn * 4, V[b], sub->n * 4, sub->n * 4, R,
                         cudaMemcpyDeviceToDevice, ctx->stream));
    desc[b] = BatchKmvDesc{(const float*)sub->xhat, sub->n, sub->DP, 0, sub->params,
                           (const float*)sub->D, sub->ldn, sub->iota, (float*)sub->KD, sub->ldn,
                           sub->iota, ctx->b_rcount + b};
    entries += (double)sub->n * (double)sub->n * R;
  }
  CK(cudaMemcpyAsync(ctx->b_kdesc, desc.data(), sizeof(BatchKmvDesc) * B, cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaMemcpyAsync(ctx->b_rcount, rc.data(), sizeof(int) * B, cudaMemcpyHostToDevice,
                     ctx->stream));
  if (ctx->cfg.precision == ULISSE_PREC_MIXED) {
    CKS(batch_tc_upload(ctx, 2, [R](int, ulisse_ctx* sub, TcLaunch& l) {
      l.V = sub->D;
      l.vmap = sub->iota;
      l.R = R;
      l.U = sub->KD;
      l.umap = sub->iota;
    }));
    CK(batch_kv_launch(ctx, 2, nullptr, R, ctx->stream));
  } else {
    CK(launch_kmv_batch(ctx->b_kdesc, ctx->b_items, ctx->b_n_items, ctx->b_queue, R,
                        ctx->num_sms, ctx->status_dev, ctx->stream));
  }
  ctx->launches++;
  ctx->mvp_rounds++;
  ctx->entry_rhs += entries;
  for (int b = 0; b < B; ++b) {
    ulisse_ctx* sub = ctx->subs[b];
    CK(cudaMemcpy2DAsync(U[b], sub->n * 4, sub->KD, sub->ldn * 4, sub->n * 4, R,
                         cudaMemcpyDeviceToDevice, ctx->stream));
  }
  int st = 0;
  CKS(batch_read_status(ctx, &st));
  return status_to_result(ctx, st);
}

// Streams and counting flags of a batch and all its problems (capture redirects both).
static void batch_set_stream(ulisse_ctx* ctx, cudaStream_t s, bool capturing) {
  ctx->stream = s;
  ctx->capturing = capturing;
  for (ulisse_ctx* sub : ctx->subs) {
    sub->stream = s;
    sub->capturing = capturing;
  }
}

// Host-side preparation of a batched step (idempotent): every problem's buffers, gradient
// maps, column metadata, identity M and zero prior; the descriptor arrays of the batched
// launches; the chain slot.  Nothing here may run inside a capture.
static ulisse_status batch_prepare(ulisse_ctx* ctx) {
  const int B = (int)ctx->subs.size();
  const int nr = ctx->cfg.n_probes, R = 1 + nr;
  for (ulisse_ctx* sub : ctx->subs) {
    SUBS(ctx, sub, ensure_columns(sub, R, R + 1));
    SUBS(ctx, sub, ensure_grad_maps(sub, nr));
    if (sub->meta_grad_R != R) {
      std::vector<int> n_est(R, 1);
      n_est[0] = 2;
      int tot = 0;
      SUBS(ctx, sub, upload_meta(sub, R, n_est.data(), &tot));
      sub->meta_grad_R = R;
    }
    const int p = sub->d + 2;
    if (!sub->m_identity) {
      std::vector<double> I((size_t)p * p, 0.0);
      for (int i = 0; i < p; ++i) I[(size_t)i * p + i] = 1.0;
      CK(cudaMemcpyAsync(sub->M_dev, I.data(), sizeof(double) * p * p, cudaMemcpyHostToDevice,
                         ctx->stream));
      sub->m_identity = true;
    }
    if (!sub->prior_zero) {
      CK(cudaMemsetAsync(sub->prior_dev, 0, sizeof(double) * p, ctx->stream));
      sub->prior_zero = true;
    }
  }
  const bool warm = ctx->cfg.warm_start_probes != 0;
  if (!ctx->b_cgargs) {
    CKS(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->b_kdesc0), sizeof(BatchKmvDesc) * B));
    CKS(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->b_cgargs), sizeof(CgArgs<float>) * B));
    CKS(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->b_cgprob), sizeof(BatchCgProb) * B));
    CKS(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->b_rmax), sizeof(int)));
    int np = 0;
    for (ulisse_ctx* sub : ctx->subs) np += sub->d + 2;
    ctx->b_np = np;
    CKS(dev_alloc(ctx, reinterpret_cast<void**>(&ctx->b_psi), sizeof(double) * np));
    if (cudaMallocHost(&ctx->b_h_rmax, sizeof(int)) != cudaSuccess)
      return fail(ctx, ULISSE_ERR_NOMEM, "cudaMallocHost failed");
    prime_kmv_batch();
    prime_grad_batch();
  }
  CKS(graph_alloc(ctx));
  std::vector<CgArgs<float>> args(B);
  std::vector<BatchCgProb> probs(B);
  std::vector<BatchKmvDesc> kd(B), kd0(B);
  const std::vector<int> rcount(B, R);
  std::vector<BatchGradDesc> gd(B);
  int slot0 = 0, maxch = 1;
  for (int b = 0; b < B; ++b) {
    ulisse_ctx* sub = ctx->subs[b];
    CgArgs<float> a = cg_args<float>(sub, 0, 0);
    a.cs = ctx->chain;
    // 4096 rows per CTA, more when the problem would need over kMaxCgChunks chunks
    a.chunk = std::max<long long>(kBatchCgChunk,
                                  ((sub->n + kMaxCgChunks - 1) / kMaxCgChunks + 255) / 256 * 256);
    a.nchunk = (int)((sub->n + a.chunk - 1) / a.chunk);
    a.n_live = sub->n_live_dev;
    if (warm) a.warm_refresh = ctx->cfg.probe_refresh;
    maxch = std::max(maxch, a.nchunk);
    args[b] = a;
    probs[b] = BatchCgProb{sub->st, sub->st_next, sub->live, sub->n_live_dev, R, sub->n};
    kd[b] = BatchKmvDesc{(const float*)sub->xhat, sub->n, sub->DP, 0, sub->params,
                         (const float*)sub->D, sub->ldn, sub->live, (float*)sub->KD, sub->ldn,
                         sub->live, sub->n_live_dev};
    // K s_0 of warm-started solves: s_0 from Sbest (cap columns after S)
    kd0[b] = BatchKmvDesc{(const float*)sub->xhat, sub->n, sub->DP, 0, sub->params,
                          (const float*)sub->S, sub->ldn, sub->warm_map, (float*)sub->KD,
                          sub->ldn, sub->iota, ctx->b_rcount + b};
    const int nslots = (int)((sub->n + kBatchBM - 1) / kBatchBM);
    gd[b] = BatchGradDesc{(const float*)sub->xhat, sub->n, sub->DP, sub->d, sub->params,
                          (const float*)sub->SE, sub->amap, (const float*)sub->sa_dev,
                          (const float*)sub->B, sub->bmap, sub->ldn, R, slot0, nslots, 0,
                          ctx->b_g + (long long)b * kMaxP};
    slot0 += nslots;
  }
  ctx->b_maxch = maxch;
  CK(cudaMemcpyAsync(ctx->b_cgargs, args.data(), sizeof(CgArgs<float>) * B, cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaMemcpyAsync(ctx->b_cgprob, probs.data(), sizeof(BatchCgProb) * B, cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaMemcpyAsync(ctx->b_kdesc, kd.data(), sizeof(BatchKmvDesc) * B, cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaMemcpyAsync(ctx->b_kdesc0, kd0.data(), sizeof(BatchKmvDesc) * B, cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaMemcpyAsync(ctx->b_rcount, rcount.data(), sizeof(int) * B, cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaMemcpyAsync(ctx->b_gdesc, gd.data(), sizeof(BatchGradDesc) * B, cudaMemcpyHostToDevice,
                     ctx->stream));
  if (ctx->cfg.precision == ULISSE_PREC_MIXED) {
    prime_kmv_tc2_batch();
    CKS(batch_tc_upload(ctx, 0, [](int, ulisse_ctx* sub, TcLaunch& l) {
      l.V = sub->D;
      l.vmap = sub->live;
      l.R_dev = sub->n_live_dev;
      l.U = sub->KD;
      l.umap = sub->live;
    }));
    CKS(batch_tc_upload(ctx, 1, [ctx](int b, ulisse_ctx* sub, TcLaunch& l) {
      l.V = sub->S;
      l.vmap = sub->warm_map;
      l.R_dev = ctx->b_rcount + b;
      l.U = sub->KD;
      l.umap = sub->iota;
    }));
    // the tensor-core gradient pass: per width group the problems' operands, in group order
    int off = 0;
    for (size_t g = 0; g < ctx->b_gt_groups.size(); ++g) {
      const std::vector<int>& grp = ctx->b_gt_groups[g];
      std::vector<GradLaunch> gl(grp.size());
      std::vector<int> ns(grp.size());
      for (size_t li = 0; li < grp.size(); ++li) {
        const int b = grp[li];
        ulisse_ctx* sub = ctx->subs[b];
        GradLaunch L{};
        L.xhat = sub->xhat;
        L.n = sub->n;
        L.ldn = sub->ldn;
        L.d = sub->d;
        L.DP = sub->DP;
        L.A = sub->SE;
        L.amap = sub->amap;
        L.sa = sub->sa_dev;
        L.B = sub->B;
        L.bmap = sub->bmap;
        L.ld = sub->ldn;
        L.M = R;
        L.params = sub->params;
        L.partials = ctx->b_gt_part + ctx->b_gt_part_off[b];
        L.counter = ctx->b_gt_cnt + b;
        L.g_out = ctx->b_g + (long long)b * kMaxP;
        L.status = ctx->status_dev;
        L.bneg = sub->bneg;
        L.tc_hi = sub->Gt_hi;
        L.tc_lo = sub->Gt_lo;
        L.tc_ld = sub->ld128;
        set_grad_images(L, sub);
        gl[li] = L;
        ns[li] = ctx->b_gt_nsplit[b];
      }
      CK(gt_batch_upload_args(gl.data(), ns.data(), (int)grp.size(),
                              (char*)ctx->b_gt_args + off * gt_batch_args_bytes(1), ctx->stream));
      CK(launch_grad_tc_batch(nullptr, 0, nullptr, 0, ctx->b_gt_dp[g], R, ctx->stream, true));
      off += (int)grp.size();
    }
  }
  return ULISSE_OK;
}

// One batched step on ctx->stream: per problem its parameters from the packed vector, the
// prescale, y and the probes, the CG start; then CG + ULISSE in lock-step rounds (one
// batched compaction, one persistent K V over all live columns of all problems, three
// batched CG launches per round); then the persistent gradient sweep and, with sgld, every
// problem's update and the packed parameters back.  The host loop and the step graph run
// exactly these launches; in the graph the round loop is a WHILE node whose compaction sets
// the loop condition and a SWITCH over the K V width.
static ulisse_status batch_step_body(ulisse_ctx* ctx, bool sgld, bool in_graph) {
  const int B = (int)ctx->subs.size();
  const int nr = ctx->cfg.n_probes, R = 1 + nr;
  int off = 0;
  for (int b = 0; b < B; ++b) {
    ulisse_ctx* sub = ctx->subs[b];
    const int p = sub->d + 2;
    CK(cudaMemcpyAsync(sub->psi_dev, ctx->b_psi + off, sizeof(double) * p,
                       cudaMemcpyDeviceToDevice, ctx->stream));
    off += p;
    SUBS(ctx, sub, prescale(sub));
    CK(cudaMemcpyAsync(sub->B, sub->y, sub->ldn * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    dim3 pg((unsigned)std::min<long long>((sub->n + 255) / 256, 2LL * ctx->num_sms), nr);
    probes_kernel<float><<<pg, 256, 0, ctx->stream>>>((float*)sub->B, sub->ldn, sub->n, nr,
                                                      ctx->cfg.probe_kind, sub->cfg.seed, 0,
                                                      ctx->chain, ctx->cfg.probe_refresh);
  }
  CK(cudaGetLastError());
  // warm-started solves: every problem's K s_0 in one persistent launch, then the starts
  const bool warm = ctx->cfg.warm_start_probes != 0;
  if (warm) CK(batch_kv_launch(ctx, 1, ctx->b_kdesc0, R, ctx->stream));
  for (int b = 0; b < B; ++b) {
    ulisse_ctx* sub = ctx->subs[b];
    CgArgs<float> a = cg_args<float>(sub, 0, 0);
    a.cs = ctx->chain;
    if (warm) a.warm_refresh = ctx->cfg.probe_refresh;
    CK(launch_cg_init(a, R, ctx->num_sms, ctx->stream));
    CK(cudaMemsetAsync(sub->n_live_dev, 0, sizeof(int), ctx->stream));
  }
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(ctx->gstat + 3, 0, sizeof(long long), ctx->stream));
  const dim3 cg_grid(ctx->b_maxch, R, B);
  auto cg_round = [&](cudaStream_t s) {
    cg_dot_batch_kernel<float><<<cg_grid, kCgChunkNT, 0, s>>>(ctx->b_cgargs);
    cg_update_batch_kernel<float><<<cg_grid, kCgChunkNT, 0, s>>>(ctx->b_cgargs);
    cg_finish_batch_kernel<float><<<cg_grid, kCgChunkNT, 0, s>>>(ctx->b_cgargs);
    return cudaGetLastError();
  };
  const int max_rounds = ctx->cfg.max_iter + 2;
  if (!in_graph) {
    for (int it = 0; it < max_rounds + 1; ++it) {
      compact_batch_kernel<<<1, 256, 0, ctx->stream>>>(ctx->b_cgprob, B, ctx->b_rmax, 0, 0, 0,
                                                       max_rounds, ctx->gstat, ctx->status_dev);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(ctx->b_h_rmax, ctx->b_rmax, sizeof(int), cudaMemcpyDeviceToHost,
                         ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      const int rmax = *ctx->b_h_rmax;
      if (rmax == 0) break;
      CK(batch_kv_launch(ctx, 0, ctx->b_kdesc, rmax, ctx->stream));
      CK(cg_round(ctx->stream));
    }
  } else {
    cudaStreamCaptureStatus cst;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    CK(cudaStreamGetCaptureInfo(ctx->stream, &cst, nullptr, &g, &deps, nullptr, &ndeps));
    cudaGraphConditionalHandle h_loop, h_branch;
    CK(cudaGraphConditionalHandleCreate(&h_loop, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = h_loop;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode;
    CK(cudaGraphAddNode(&wnode, g, deps, nullptr, ndeps, &wp));
    CK(cudaStreamUpdateCaptureDependencies(ctx->stream, &wnode, nullptr, 1,
                                           cudaStreamSetCaptureDependencies));
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    CK(cudaGraphConditionalHandleCreate(&h_branch, body, 5, cudaGraphCondAssignDefault));
    cudaStream_t s2 = ctx->cap_stream2;
    CK(cudaStreamBeginCaptureToGraph(s2, body, nullptr, nullptr, 0,
                                     cudaStreamCaptureModeThreadLocal));
    compact_batch_kernel<<<1, 256, 0, s2>>>(ctx->b_cgprob, B, ctx->b_rmax, 1, h_loop, h_branch,
                                            max_rounds, ctx->gstat, ctx->status_dev);
    cudaError_t e = cudaGetLastError();
    const cudaGraphNode_t* bdeps = nullptr;
    size_t nbdeps = 0;
    cudaGraph_t bg = nullptr;
    if (e == cudaSuccess)
      e = cudaStreamGetCaptureInfo(s2, &cst, nullptr, &bg, &bdeps, nullptr, &nbdeps);
    cudaGraphNodeParams sp = {};
    sp.type = cudaGraphNodeTypeConditional;
    sp.conditional.handle = h_branch;
    sp.conditional.type = cudaGraphCondTypeSwitch;
    sp.conditional.size = 5;
    cudaGraphNode_t snode;
    if (e == cudaSuccess) e = cudaGraphAddNode(&snode, bg, bdeps, nullptr, nbdeps, &sp);
    if (e == cudaSuccess)
      e = cudaStreamUpdateCaptureDependencies(s2, &snode, nullptr, 1,
                                              cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) e = cg_round(s2);
    cudaGraph_t tmp = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(s2, &tmp);
    CK(e);
    CK(e2);
    for (int k = 0; k < 5; ++k) {
      CK(cudaStreamBeginCaptureToGraph(s2, sp.conditional.phGraph_out[k], nullptr, nullptr, 0,
                                       cudaStreamCaptureModeThreadLocal));
      const cudaError_t e3 = batch_kv_launch(ctx, 0, ctx->b_kdesc, kBatchWidths[k], s2);
      const cudaError_t e4 = cudaStreamEndCapture(s2, &tmp);
      CK(e3);
      CK(e4);
    }
  }
  // the second estimate of K^{-1} y as the right factor; the gradient sweep
  for (ulisse_ctx* sub : ctx->subs) {
    if (warm) CK(cudaMemsetAsync(sub->warm_valid, 0x01, sizeof(int), ctx->stream));
    CK(cudaMemcpyAsync(sub->B, (char*)sub->SE + sub->ldn * 4, sub->ldn * 4,
                       cudaMemcpyDeviceToDevice, ctx->stream));
  }
  if (ctx->cfg.precision == ULISSE_PREC_MIXED) {
    int off = 0;
    for (size_t g = 0; g < ctx->b_gt_groups.size(); ++g) {
      const int nb = (int)ctx->b_gt_groups[g].size();
      CK(launch_grad_tc_batch((char*)ctx->b_gt_args + off * gt_batch_args_bytes(1), nb,
                              ctx->b_gt_items + ctx->b_gt_item_off[g], ctx->b_gt_item_n[g],
                              ctx->b_gt_dp[g], R, ctx->stream));
      off += nb;
    }
  } else {
    CK(launch_grad_batch(ctx->b_gdesc, B, ctx->b_items, ctx->b_n_items, ctx->b_queue,
                         ctx->b_gpart, R, ctx->num_sms, ctx->status_dev, ctx->stream));
  }
  if (sgld) {
    off = 0;
    for (int b = 0; b < B; ++b) {
      ulisse_ctx* sub = ctx->subs[b];
      const int p = sub->d + 2;
      sgld_chain_kernel<<<1, 32, 0, ctx->stream>>>(sub->psi_dev, ctx->b_g + (long long)b * kMaxP,
                                                   sub->M_dev, sub->prior_dev, p, sub->cfg.seed,
                                                   ctx->chain, sub->status_dev, 0, ctx->b_np, off);
      off += p;
    }
    chain_advance_kernel<<<1, 32, 0, ctx->stream>>>(ctx->chain);
    CK(cudaGetLastError());
    off = 0;
    for (int b = 0; b < B; ++b) {
      ulisse_ctx* sub = ctx->subs[b];
      const int p = sub->d + 2;
      CK(cudaMemcpyAsync(ctx->b_psi + off, sub->psi_dev, sizeof(double) * p,
                         cudaMemcpyDeviceToDevice, ctx->stream));
      off += p;
    }
  }
  return ULISSE_OK;
}

// Work of one batched step outside the round loop (the loop's share is counted on the device).
static void batch_count_fixed(ulisse_ctx* ctx, int steps, bool sgld) {
  const int B = (int)ctx->subs.size();
  const int R = 1 + ctx->cfg.n_probes;
  const bool warm = ctx->cfg.warm_start_probes != 0;
  double ent = 0.0;
  for (ulisse_ctx* sub : ctx->subs) ent += (double)sub->n * (double)sub->n * R;
  // per problem prescale (+ the tensor-core row images), probes, CG start; the gradient
  // sweep; the updates; the warm starts' product (mixed: every K V launch packs V first)
  const bool mixed = ctx->cfg.precision == ULISSE_PREC_MIXED;
  const long long grad_launches = mixed ? 2LL * (long long)ctx->b_gt_groups.size() : 2LL;
  long long init_launches = 0;   // the CG starts' (cg_init_launch_count) beyond one per problem
  for (ulisse_ctx* sub : ctx->subs) init_launches += cg_init_launch_count(sub->n, R, ctx->num_sms) - 1;
  ctx->launches += (long long)steps * ((mixed ? 5LL : 3LL) * B + init_launches + grad_launches +
                                       (sgld ? B + 1 : 0) + (warm ? (mixed ? 2 : 1) : 0));
  ctx->entry_rhs += steps * ent * (warm ? 2.0 : 1.0);
  if (warm) ctx->mvp_rounds += steps;
}

static ulisse_status batch_fold_gstat(ulisse_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->h_gstat, ctx->gstat, sizeof(long long) * 4, cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->mvp_rounds += ctx->h_gstat[0];
  ctx->entry_rhs += (double)ctx->h_gstat[1];
  ctx->launches += ctx->h_gstat[2];
  // the device counts one K V launch per round; the mixed path also packs V each round
  if (ctx->cfg.precision == ULISSE_PREC_MIXED) ctx->launches += ctx->h_gstat[0];
  CK(cudaMemsetAsync(ctx->gstat, 0, sizeof(long long) * 3, ctx->stream));
  return ULISSE_OK;
}

static ulisse_status batch_graph_build(ulisse_ctx* ctx) {
  graph_release(ctx);
  if (!ctx->cap_stream) {
    CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&ctx->cap_stream2, cudaStreamNonBlocking));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  cudaStream_t saved = ctx->stream;
  batch_set_stream(ctx, ctx->cap_stream, true);
  ulisse_status r = ULISSE_OK;
  cudaError_t e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) r = batch_step_body(ctx, true, true);
  cudaGraph_t graph = nullptr;
  const cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(ctx->cap_stream, &graph) : e;
  batch_set_stream(ctx, saved, false);
  if (r != ULISSE_OK) {
    if (graph) cudaGraphDestroy(graph);
    return r;
  }
  if (e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(ctx, ULISSE_ERR_CUDA, std::string("batched step graph capture: ") + cudaGetErrorString(e2));
  }
  ctx->step_graph = graph;
  CK(cudaGraphInstantiate(&ctx->step_exec, graph, 0));
  ctx->graph_key = 1000;
  return ULISSE_OK;
}

// n_steps batched SGLD steps from the packed parameters already in b_psi, with the chain
// slot already set: one graph launch per step, or the host loop.
static ulisse_status batch_run_steps(ulisse_ctx* ctx, int n_steps) {
  if (ctx->graph_enabled) {
    if (ctx->graph_key != 1000) CKS(batch_graph_build(ctx));
    for (int k = 0; k < n_steps; ++k) CK(cudaGraphLaunch(ctx->step_exec, ctx->stream));
  } else {
    for (int k = 0; k < n_steps; ++k) CKS(batch_step_body(ctx, true, false));
  }
  batch_count_fixed(ctx, n_steps, true);
  return ULISSE_OK;
}

static ulisse_status batch_set_chain(ulisse_ctx* ctx, unsigned long long step0,
                                     const double* eps_dev, double* trace_dev) {
  const ChainSlot cs{0, step0, eps_dev, trace_dev};
  CK(cudaMemcpyAsync(ctx->chain, &cs, sizeof(ChainSlot), cudaMemcpyHostToDevice, ctx->stream));
  return ULISSE_OK;
}

ulisse_status ulisse_batch_grad(ulisse_ctx* ctx, const double* psi, unsigned long long step,
                                double* g, ulisse_col_stats* stats) {
  BATCHED_ONLY(ctx);
  if (!g) return fail(ctx, ULISSE_ERR_ARG, "g is null");
  CKS(batch_set_psi(ctx, psi));
  CKS(batch_clear_status(ctx));
  CKS(batch_prepare(ctx));
  CK(cudaMemcpyAsync(ctx->b_psi, psi, sizeof(double) * ctx->b_np, cudaMemcpyHostToDevice,
                     ctx->stream));
  CKS(batch_set_chain(ctx, step, ctx->eps_one, nullptr));
  CKS(batch_step_body(ctx, false, false));
  batch_count_fixed(ctx, 1, false);
  const int B = (int)ctx->subs.size();
  std::vector<double> gall((size_t)B * kMaxP);
  CK(cudaMemcpyAsync(gall.data(), ctx->b_g, sizeof(double) * gall.size(), cudaMemcpyDeviceToHost,
                     ctx->stream));
  CKS(batch_fold_gstat(ctx));
  int st = 0;
  CKS(batch_read_status(ctx, &st));
  for (int b = 0; b < B; ++b)
    for (int k = 0; k < ctx->subs[b]->d + 2; ++k) g[ctx->sub_p_off[b] + k] = gall[(size_t)b * kMaxP + k];
  if (stats) {
    const int R = 1 + ctx->cfg.n_probes;
    for (int b = 0; b < B; ++b) SUBS(ctx, ctx->subs[b], copy_stats(ctx->subs[b], stats + (size_t)b * R, R));
  }
  return status_to_result(ctx, st);
}

ulisse_status ulisse_batch_sgld_step(ulisse_ctx* ctx, double* psi_inout, double eps_t,
                                     unsigned long long step, double* g_out) {
  BATCHED_ONLY(ctx);
  if (!(eps_t >= 0.0) || !std::isfinite(eps_t)) return fail(ctx, ULISSE_ERR_ARG, "eps_t invalid");
  CKS(batch_set_psi(ctx, psi_inout));
  CKS(batch_clear_status(ctx));
  CKS(batch_prepare(ctx));
  CK(cudaMemcpyAsync(ctx->b_psi, psi_inout, sizeof(double) * ctx->b_np, cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaMemcpyAsync(ctx->eps_one, &eps_t, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  CKS(batch_set_chain(ctx, step, ctx->eps_one, nullptr));
  CKS(batch_run_steps(ctx, 1));
  CKS(batch_fold_gstat(ctx));
  int st = 0;
  CKS(batch_read_status(ctx, &st));
  ulisse_status r = status_to_result(ctx, st);
  if (r == ULISSE_ERR_ARG) return r;
  CK(cudaMemcpyAsync(psi_inout, ctx->b_psi, sizeof(double) * ctx->b_np, cudaMemcpyDeviceToHost,
                     ctx->stream));
  if (g_out) {
    const int B = (int)ctx->subs.size();
    std::vector<double> gall((size_t)B * kMaxP);
    CK(cudaMemcpyAsync(gall.data(), ctx->b_g, sizeof(double) * gall.size(), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int b = 0; b < B; ++b)
      for (int k = 0; k < ctx->subs[b]->d + 2; ++k)
        g_out[ctx->sub_p_off[b] + k] = gall[(size_t)b * kMaxP + k];
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return r;
}

ulisse_status ulisse_batch_sgld_chain(ulisse_ctx* ctx, double* psi_dev, const double* eps_dev,
                                      int n_steps, unsigned long long step0, double* trace_dev) {
  BATCHED_ONLY(ctx);
  if (!psi_dev || !eps_dev || n_steps < 0) return fail(ctx, ULISSE_ERR_ARG, "bad chain arguments");
  CKS(batch_clear_status(ctx));
  CKS(batch_prepare(ctx));
  CK(cudaMemcpyAsync(ctx->b_psi, psi_dev, sizeof(double) * ctx->b_np, cudaMemcpyDeviceToDevice,
                     ctx->stream));
  CKS(batch_set_chain(ctx, step0, eps_dev, trace_dev));
  CKS(batch_run_steps(ctx, n_steps));
  CK(cudaMemcpyAsync(psi_dev, ctx->b_psi, sizeof(double) * ctx->b_np, cudaMemcpyDeviceToDevice,
                     ctx->stream));
  CKS(batch_fold_gstat(ctx));
  int st = 0;
  CKS(batch_read_status(ctx, &st));
  return status_to_result(ctx, st);
}

// ---------------------------------------------------------------------------------------
// Autotuner: for every live column count, the K V launch configuration that runs fastest
// on this context's data and device, timed with CUDA events on the context's stream.
// ---------------------------------------------------------------------------------------
// Median time of `reps` K V launches over nl columns in the given configuration (width 0:
// the default choices); *nsplit_out gets the split count the configuration used.
static ulisse_status time_kmv_config(ulisse_ctx* ctx, int nl, int width, int tm, int nsplit,
                                     int cross, int reps, float* ms_out, int* nsplit_out) {
  if ((int)ctx->tune.size() < nl)
    ctx->tune.resize((size_t)nl, ulisse_ctx::KmvTune{0, 0, 0, 0.f, 0.f, 0});
  const ulisse_ctx::KmvTune saved = ctx->tune[nl - 1];
  ctx->tune[nl - 1] = ulisse_ctx::KmvTune{width, tm, nsplit, 0.f, 0.f, cross};
  ctx->planning = true;
  ulisse_status r = run_kmv(ctx, ctx->D, ctx->iota, nl, ctx->KD, ctx->iota, kModeK, -1);
  ctx->planning = false;
  if (nsplit_out) *nsplit_out = ctx->last_nsplit;
  cudaEvent_t a = nullptr, b = nullptr;
  if (r == ULISSE_OK && (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess))
    r = fail(ctx, ULISSE_ERR_CUDA, "cudaEventCreate failed");
  const long long l0 = ctx->launches;
  const double e0 = ctx->entry_rhs;
  std::vector<float> t;
  if (r == ULISSE_OK) r = run_kmv(ctx, ctx->D, ctx->iota, nl, ctx->KD, ctx->iota, kModeK, -1);
  for (int k = 0; k < reps && r == ULISSE_OK; ++k) {
    cudaEventRecord(a, ctx->stream);
    r = run_kmv(ctx, ctx->D, ctx->iota, nl, ctx->KD, ctx->iota, kModeK, -1);
    cudaEventRecord(b, ctx->stream);
    float ms = 0.f;
    if (r == ULISSE_OK && (cudaEventSynchronize(b) != cudaSuccess ||
                           cudaEventElapsedTime(&ms, a, b) != cudaSuccess))
      r = fail(ctx, ULISSE_ERR_CUDA, "event timing failed");
    t.push_back(ms);
  }
  ctx->launches = l0;      // tuning launches are not part of the method's work
  ctx->entry_rhs = e0;
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  ctx->tune[nl - 1] = saved;
  if (r != ULISSE_OK) return r;
  std::sort(t.begin(), t.end());
  *ms_out = t[t.size() / 2];
  return ULISSE_OK;
}

ulisse_status ulisse_autotune(ulisse_ctx* ctx, const double* psi, int max_cols, int reps,
                              ulisse_tune_entry* out) {
  if (!ctx) return ULISSE_ERR_ARG;
  if (ctx->batched) return fail(ctx, ULISSE_ERR_ARG, "batched context: use the ulisse_batch_* calls");
  if (max_cols < 1 || max_cols > kMaxRChunk || reps < 1 || reps > 100)
    return fail(ctx, ULISSE_ERR_ARG, "max_cols must be 1..32 and reps 1..100");
  if (ctx->f64) return fail(ctx, ULISSE_ERR_ARG, "the autotuner covers the FP32 and mixed paths");
  CKS(set_psi_host(ctx, psi));
  CKS(prescale(ctx));
  CKS(ensure_columns(ctx, max_cols, max_cols));
  const bool prof = ctx->prof;
  ctx->prof = false;
  ctx->tune.assign((size_t)max_cols, ulisse_ctx::KmvTune{0, 0, 0, 0.f, 0.f, 0});
  std::vector<ulisse_ctx::KmvTune> table((size_t)max_cols);
  ulisse_status r = ULISSE_OK;
  for (int nl = 1; nl <= max_cols && r == ULISSE_OK; ++nl) {
    // the default configuration first (what the launch plan picks untuned)
    float ms_def = 0.f;
    int split_def = 1;
    r = time_kmv_config(ctx, nl, 0, 0, 0, 0, reps, &ms_def, &split_def);
    if (r != ULISSE_OK) break;
    const int cross_def =
        ctx->mixed ? (ctx->cfg.tc_cross_term != 0 ? ctx->cfg.tc_cross_term : kCrossTensor) : 0;
    ulisse_ctx::KmvTune best{0, 0, 0, ms_def, ms_def, cross_def};
    // candidates: the compiled width (tensor cores: the MMA N; SIMT: the smallest
    // instantiation >= nl, or a larger one), rows per thread (SIMT) or where the cross term
    // is formed (tensor cores, unless the configuration fixes it), then the j split
    std::vector<int> widths, tms, crosses;
    if (ctx->mixed) {
      for (int wd : {16, 32, 64})
        if (wd >= nl) widths.push_back(wd);
      tms = {0};
      if (ctx->cfg.tc_cross_term != 0) crosses = {ctx->cfg.tc_cross_term};
      else crosses = {kCrossPipe, kCrossTensor};
    } else {
      widths = {nl, nl + 1, nl + 4};
      tms = {2, 4};
      crosses = {0};
    }
    for (int wd : widths) {
      for (int tm : tms) {
        for (int cr : crosses) {
          float ms = 0.f;
          int sp = 1;
          r = time_kmv_config(ctx, nl, wd, tm, 0, cr, reps, &ms, &sp);
          if (r != ULISSE_OK) break;
          if (ms < best.ms) best = ulisse_ctx::KmvTune{wd, tm, 0, ms, ms_def, cr};
        }
        if (r != ULISSE_OK) break;
      }
      if (r != ULISSE_OK) break;
    }
    if (r != ULISSE_OK) break;
    const int wd = best.width > 0 ? best.width : nl;
    float ms_base = 0.f;
    int base = 1;
    r = time_kmv_config(ctx, nl, wd, best.tm, 0, best.cross, 1, &ms_base, &base);   // its planned split
    for (int sp : {base / 2, base * 2}) {
      if (r != ULISSE_OK || sp < 1 || sp == base) continue;
      float ms = 0.f;
      int used = sp;
      r = time_kmv_config(ctx, nl, wd, best.tm, sp, best.cross, reps, &ms, &used);
      if (r == ULISSE_OK && ms < best.ms)
        best = ulisse_ctx::KmvTune{wd, best.tm, sp, ms, ms_def, best.cross};
    }
    if (r != ULISSE_OK) break;
    if (best.width == 0) best.width = nl;
    if (best.tm == 0) best.tm = ctx->cfg.kmv_rows_per_thread;
    table[nl - 1] = best;
  }
  ctx->prof = prof;
  if (r != ULISSE_OK) {
    ctx->tune.clear();
    return r;
  }
  ctx->tune = table;
  ctx->graph_key = -1;   // a captured step graph holds the old configuration
  if (out)
    for (int nl = 1; nl <= max_cols; ++nl) {
      const ulisse_ctx::KmvTune& t = table[nl - 1];
      out[nl - 1] = ulisse_tune_entry{nl, t.width, t.tm, t.nsplit, t.ms, t.ms_default, t.cross};
    }
  CK(cudaStreamSynchronize(ctx->stream));
  return ULISSE_OK;
}

ulisse_status ulisse_set_tune(ulisse_ctx* ctx, const ulisse_tune_entry* table, int n) {
  if (!ctx) return ULISSE_ERR_ARG;
  if (ctx->batched) return fail(ctx, ULISSE_ERR_ARG, "batched context: no K V table");
  if (ctx->f64) return fail(ctx, ULISSE_ERR_ARG, "the K V table covers the FP32 and mixed paths");
  if (n < 0 || n > kMaxRChunk || (n > 0 && !table))
    return fail(ctx, ULISSE_ERR_ARG, "n must be 0..32 (and the table non-null)");
  std::vector<ulisse_ctx::KmvTune> t((size_t)n);
  for (int k = 0; k < n; ++k) {
    const ulisse_tune_entry& e = table[k];
    const int nl = k + 1;
    bool ok = e.width >= nl && e.width <= 64 && e.nsplit >= 0 && e.nsplit <= 64;
    if (ctx->mixed)
      ok = ok && (e.cross_term == kCrossPipe || e.cross_term == kCrossTensor);
    else
      ok = ok && (e.rows_per_thread == 2 || e.rows_per_thread == 4) && e.cross_term == 0;
    if (!ok) return fail(ctx, ULISSE_ERR_ARG, "invalid K V table entry " + std::to_string(k));
    t[k] = ulisse_ctx::KmvTune{e.width, e.rows_per_thread, e.nsplit, e.ms, e.ms_default,
                               e.cross_term};
  }
  ctx->tune = t;
  ctx->graph_key = -1;   // a captured step graph holds the old configuration
  return ULISSE_OK;
}

// One CTA waits on an mbarrier that expects two arrivals and gets one: the wait, bounded by
// the SM clock here (2^30 cycles, about half a second), runs out and the timeout is recorded
// in the status word as every kernel records it.
__global__ void selftest_wait_timeout_kernel(int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 2);
    fence_barrier_init();
    mbar_arrive_expect_tx(&bar, 0);   // one arrival (no bytes) of the two it waits for
    bool done = false;
    const long long t0 = clock64();
    while (!done && clock64() - t0 < (1LL << 30)) done = mbar_try_wait(&bar, 0);
    if (!done) atomicOr(status, kStatusTimeout);
  }
}

ulisse_status ulisse_selftest_wait_timeout(ulisse_ctx* ctx) {
  if (!ctx) return ULISSE_ERR_ARG;
  CK(cudaMemsetAsync(ctx->status_dev, 0, sizeof(int), ctx->stream));
  selftest_wait_timeout_kernel<<<1, 32, 0, ctx->stream>>>(ctx->status_dev);
  CK(cudaGetLastError());
  int st = 0;
  CKS(read_status(ctx, &st));
  return status_to_result(ctx, st);
}

ulisse_status ulisse_counters(const ulisse_ctx* ctx, long long* mvp_rounds, double* entry_rhs,
                              long long* kernel_launches) {
  if (!ctx) return ULISSE_ERR_ARG;
  const long long launches = ctx->launches;
  if (mvp_rounds) *mvp_rounds = ctx->mvp_rounds;
  if (entry_rhs) *entry_rhs = ctx->entry_rhs;
  if (kernel_launches) *kernel_launches = launches;
  return ULISSE_OK;
}

ulisse_status ulisse_profile_enable(ulisse_ctx* ctx, int enable) {
  if (!ctx) return ULISSE_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  prof_drain(ctx);
  ctx->prof = enable != 0;
  ctx->totals = ulisse_profile{};
  return ULISSE_OK;
}

ulisse_status ulisse_profile_read(ulisse_ctx* ctx, ulisse_profile* out, int reset) {
  if (!ctx || !out) return ULISSE_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  prof_drain(ctx);
  *out = ctx->totals;
  if (reset) ctx->totals = ulisse_profile{};
  return ULISSE_OK;
}

const char* ulisse_last_error(const ulisse_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

void ulisse_destroy(ulisse_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (void** p : {reinterpret_cast<void**>(&ctx->st_next), reinterpret_cast<void**>(&ctx->part1),
                   reinterpret_cast<void**>(&ctx->part2), reinterpret_cast<void**>(&ctx->bneg),
                   &ctx->Vt_hi, &ctx->Vt_lo, &ctx->Gt_hi, &ctx->Gt_lo,
                   reinterpret_cast<void**>(&ctx->Xt_hi), reinterpret_cast<void**>(&ctx->Xt_lo),
                   reinterpret_cast<void**>(&ctx->q_map), &ctx->q_sa, &ctx->pcg_buf, &ctx->pred_xs,
                   reinterpret_cast<void**>(&ctx->pcg_aux), reinterpret_cast<void**>(&ctx->pcg_live)})
    dev_free(*p);
  for (void** p : {reinterpret_cast<void**>(&ctx->X), &ctx->y, &ctx->xhat,
                   reinterpret_cast<void**>(&ctx->params), reinterpret_cast<void**>(&ctx->psi_dev),
                   &ctx->B, &ctx->S, &ctx->E, &ctx->D, &ctx->KD, &ctx->SE,
                   reinterpret_cast<void**>(&ctx->st), reinterpret_cast<void**>(&ctx->live),
                   reinterpret_cast<void**>(&ctx->n_live_dev), reinterpret_cast<void**>(&ctx->iota),
                   &ctx->partials, reinterpret_cast<void**>(&ctx->counters),
                   reinterpret_cast<void**>(&ctx->gpart), reinterpret_cast<void**>(&ctx->gcounter),
                   reinterpret_cast<void**>(&ctx->g_dev), &ctx->sa_dev,
                   reinterpret_cast<void**>(&ctx->amap), reinterpret_cast<void**>(&ctx->bmap),
                   reinterpret_cast<void**>(&ctx->M_dev), reinterpret_cast<void**>(&ctx->prior_dev),
                   reinterpret_cast<void**>(&ctx->status_dev),
                   reinterpret_cast<void**>(&ctx->warm_valid)})
    dev_free(*p);
  for (void* p : ctx->ws_allocs) cudaFree(p);
  ctx->ws_allocs.clear();
  for (ulisse_ctx* sub : ctx->subs) ulisse_destroy(sub);
  ctx->subs.clear();
  graph_release(ctx);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->cap_stream2) cudaStreamDestroy(ctx->cap_stream2);
  dev_free(reinterpret_cast<void*&>(ctx->chain));
  dev_free(reinterpret_cast<void*&>(ctx->gstat));
  dev_free(reinterpret_cast<void*&>(ctx->eps_one));
  if (ctx->h_gstat) cudaFreeHost(ctx->h_gstat);
  for (void** p : {reinterpret_cast<void**>(&ctx->b_cgargs), reinterpret_cast<void**>(&ctx->b_cgprob),
                   reinterpret_cast<void**>(&ctx->b_kdesc0),
                   reinterpret_cast<void**>(&ctx->b_rmax), reinterpret_cast<void**>(&ctx->b_psi)})
    dev_free(*p);
  if (ctx->b_h_rmax) cudaFreeHost(ctx->b_h_rmax);
  for (void** p : {reinterpret_cast<void**>(&ctx->b_items), reinterpret_cast<void**>(&ctx->b_kdesc),
                   reinterpret_cast<void**>(&ctx->b_gdesc), reinterpret_cast<void**>(&ctx->b_queue),
                   reinterpret_cast<void**>(&ctx->b_nlive), reinterpret_cast<void**>(&ctx->b_rcount),
                   reinterpret_cast<void**>(&ctx->b_gpart), reinterpret_cast<void**>(&ctx->b_g),
                   reinterpret_cast<void**>(&ctx->b_tc_items), &ctx->b_tc_args,
                   reinterpret_cast<void**>(&ctx->b_tc_part), reinterpret_cast<void**>(&ctx->b_tc_cnt),
                   reinterpret_cast<void**>(&ctx->b_gt_items), &ctx->b_gt_args,
                   reinterpret_cast<void**>(&ctx->b_gt_part), reinterpret_cast<void**>(&ctx->b_gt_cnt)})
    dev_free(*p);
  if (ctx->b_h_nlive) cudaFreeHost(ctx->b_h_nlive);
  if (ctx->b_h_status) cudaFreeHost(ctx->b_h_status);
  prof_drain(ctx);
  for (auto& e : ctx->free_events) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  if (ctx->h_n_live) cudaFreeHost(ctx->h_n_live);
  if (ctx->h_status) cudaFreeHost(ctx->h_status);
  delete ctx;
}

}  // extern "C"
