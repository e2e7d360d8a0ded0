#!/usr/bin/env python
"""SGLD + ULISSE benchmark on the Census-shaped workload (n = 50,000, d = 8, 16 probes).

One step = one pass of the whole path: parameter unpack and prescale, probe generation,
the batched ULISSE solves of K s = y (two estimators) and K s = r_j (j = 1..16), the fused
gradient pass and the SGLD update -- all in libulisse's CUDA kernels, launched through the
C ABI.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The headline is the chosen path -- tensor-core (tcgen05) mixed-precision K V, every step one
CUDA-graph launch, probes reused for 20 steps with warm-started solves -- in SGLD steps/s;
the plain FP32 path (SIMT K V, same graph form) is timed the same way beside it, and both
report K V entry*RHS/s from an event-timed pass.  The roofline of the dominant K V kernel
counts the method's work (n(n+1)/2 distinct exponentials per product) against the
exponential unit's rate measured on the device in the same run.

At N = 1 the same line carries the other configurations as keys: the gradient error of the
paths (Sec. 5's measure, dense FP64 Cholesky reference on the device), the near-duplicate
K V at full size (n = 200,000, d = 16, 64 RHS) with its error against oracle rows, the
64-problem uneven batch, the 2-D FP64 100-step chain beside the oracle's full chain, and
preconditioned CG (Sec. 3) against plain CG with cold solves (--no-extras skips them).

--impl reference times the FP64 CPU oracle on the host cores instead (a bounded sample of
the same workload, scaled to SGLD steps/s).  With N > 1 (torchrun) every rank runs an
independent chain (replicas: the method's path for one problem runs on one GPU).
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "census_like"
N_PROBES = 16
EPS_T = 1e-4
L2_FLUSH_BYTES = 512 << 20          # > 129 MB L2: written between timed steps
FP32_FMA_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x 2 x max clock
EX2_PEAK_DERIVED_TENTRIES = 152 * 32 * 2.070e9 / 1e12    # SMs x ex2 per clock x max clock
WORK_FILE = os.path.join(ROOT, "profiles", "census_like_step_work.txt")
# per K V kernel: its ncu traffic summary and the sources whose hash it was taken for
KMV_KERNELS = {
    "fp32": ("kmv_kernel (tile-generating K V, FP32 SIMT)",
             os.path.join(ROOT, "profiles", "kmv_census_like_traffic.txt"),
             ["paper_1501_05427_gb300/csrc/kmv_kernel.cuh",
              "paper_1501_05427_gb300/csrc/kmv_launch.cuh",
              "paper_1501_05427_gb300/csrc/kmv_f32.cu",
              "paper_1501_05427_gb300/csrc/ulisse_internal.cuh"]),
    "mixed_pipe": ("kmv_tc_kernel (tile-generating K V, tcgen05 BF16x3 contraction, "
                   "FP32-FMA cross term)",
                   os.path.join(ROOT, "profiles", "kmv_tc_census_like_traffic.txt"),
                   ["paper_1501_05427_gb300/csrc/kmv_tc.cu",
                    "paper_1501_05427_gb300/csrc/tc_common.cuh",
                    "paper_1501_05427_gb300/csrc/kmv_kernel.cuh",
                    "paper_1501_05427_gb300/csrc/ulisse_internal.cuh"]),
    "mixed_tensor": ("kmv_tc2_kernel (tile-generating K V, tcgen05 3xTF32 cross term and "
                     "BF16x3 contraction, FP32 accumulation)",
                     os.path.join(ROOT, "profiles", "kmv_tc2_census_like_traffic.txt"),
                     ["paper_1501_05427_gb300/csrc/kmv_tc2.cu",
                      "paper_1501_05427_gb300/csrc/kmv_tc.cu",
                      "paper_1501_05427_gb300/csrc/tc_common.cuh",
                      "paper_1501_05427_gb300/csrc/kmv_kernel.cuh",
                      "paper_1501_05427_gb300/csrc/ulisse_internal.cuh"]),
}
CROSS_KEY = {1: "mixed_pipe", 2: "mixed_tensor"}


def generated_entries(n):
    """Covariance entries the tensor-core K V kernel generates per launch (every (i, j))."""
    return float(n) * n


def kernel_key(path, tune_table=None, live_cols=None):
    """KMV_KERNELS key of the K V kernel a path runs at live_cols columns: the tensor-core path
    forms the cross term where the autotuner chose (default: on the tensor cores)."""
    if path == "fp32":
        return "fp32"
    if tune_table and live_cols and tune_table[live_cols - 1].get("cross_term"):
        return CROSS_KEY[tune_table[live_cols - 1]["cross_term"]]
    return "mixed_tensor"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=150)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target host time of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--path", choices=["fp32", "mixed"], default="mixed",
                    help="chosen K V path: tensor-core mixed precision or FP32 SIMT")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip timing the plain FP32 path beside the chosen one")
    ap.add_argument("--no-graph", action="store_true",
                    help="run the steps from the host loop instead of one graph launch each")
    ap.add_argument("--workload", choices=["census_like", "uneven_batch"], default="census_like",
                    help="census_like: the headline; uneven_batch: 64 problems of uneven size "
                         "advanced together (batched context, one graph launch per step)")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the K V autotuner (untuned launch configurations)")
    ap.add_argument("--refresh", type=int, default=20,
                    help="chosen path: redraw the probes every this many steps (Sec. 5.1 uses 20)")
    ap.add_argument("--no-warm", action="store_true",
                    help="chosen path: start every solve from zero (no warm-started solves)")
    ap.add_argument("--profile-steps", type=int, default=8,
                    help="steps of the event-timed pass (per-launch K V times)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other configurations' keys (gradient error, near-duplicate "
                         "K V, uneven batch, 2-D FP64 chain)")
    ap.add_argument("--c3-rows", type=int, default=4000,
                    help="output rows of the near-duplicate K V the oracle evaluates")
    ap.add_argument("--c5-steps", type=int, default=1000,
                    help="steps of the learned warm start's recording trajectory (0: skip)")
    ap.add_argument("--grad-reps", type=int, default=100,
                    help="repetitions of the gradient-error measurement")
    return ap.parse_args()


def _kv_file(path):
    out = {}
    if not os.path.exists(path):
        return out
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#") and "=" in line:
            k, v = line.split("=", 1)
            out[k.strip()] = v.strip()
    return out


def kmv_source_hash(key="fp32"):
    h = hashlib.sha256()
    for f in KMV_KERNELS[key][2]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# ----------------------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = list(csv.reader(io.StringIO(self.tmp.read())))
        self.tmp.close()
        os.unlink(self.tmp.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for name, flag in zip(names, r[5:9]):
                if flag.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------------------
# oracle timing on the host cores (bounded sample, scaled to steps/s)
# ----------------------------------------------------------------------------------------
_ORACLE_CAL = {}   # per problem size: inputs and per-row times of the oracle (one calibration)


def oracle_sample(prob, work, target_s, rng_seed=0):
    """Time the oracle's two O(n^2) kernels on a row sample of the full-size workload:
    K V with 17 right-hand sides (all n columns) and the all-parameter derivative products
    of the gradient, each for m output rows; scale each by n/m and by the per-step work."""
    import numpy as np

    import oracle
    n, d = prob.n, prob.d
    R = 1 + N_PROBES
    rng = np.random.default_rng(rng_seed)
    cal = _ORACLE_CAL.get(n)
    if cal is None:
        # once per run: build, inputs, and a calibration on a few hundred rows (threads warm)
        oracle.build()
        Xd = prob.X.astype(np.float64)
        V = np.random.default_rng(0).standard_normal((n, R))
        cores = oracle.omp_threads()
        oracle.kmv_rows(Xd, prob.psi_true, V, np.arange(cores))
        m0 = 8 * cores
        t0 = time.perf_counter()
        oracle.kmv_rows(Xd, prob.psi_true, V, np.arange(m0))
        t_row = max(time.perf_counter() - t0, 1e-4) / m0
        t0 = time.perf_counter()
        oracle.dkmv_all_rows(Xd, prob.psi_true, V, np.arange(2 * cores))
        t_row_g = max(time.perf_counter() - t0, 1e-4) / (2 * cores)
        cal = _ORACLE_CAL[n] = (Xd, V, cores, t_row, t_row_g)
    Xd, V, cores, t_row, t_row_g = cal
    m_kv = int(max(8 * cores, min(n, 0.6 * target_s / t_row)))
    m_g = int(max(2 * cores, min(n, 0.4 * target_s / t_row_g)))
    rows = np.sort(rng.choice(n, m_kv, replace=False))
    t0 = time.perf_counter()
    oracle.kmv_rows(Xd, prob.psi_true, V, rows)
    t_kv = time.perf_counter() - t0
    rows_g = np.sort(rng.choice(n, m_g, replace=False))
    t0 = time.perf_counter()
    oracle.dkmv_all_rows(Xd, prob.psi_true, V, rows_g)
    t_g = time.perf_counter() - t0
    kv_rate = m_kv * n * R / t_kv                 # entry x RHS per second
    grad_rate = m_g * n / t_g                     # gradient entries per second
    t_step = work["mvp_entry_rhs"] / kv_rate + work["grad_entries"] / grad_rate
    return {
        "steps_per_s": 1.0 / t_step,
        "kv_entry_rhs_per_s": kv_rate,
        "cores": oracle.omp_threads(),
        "sample": ("oracle K V (R=%d) on %d of %d output rows and all-parameter derivative "
                   "products on %d rows of the full-size workload, %.1f s of host time; scaled "
                   "by n/m and by the per-step work (%.4g K V entry-RHS in %.1f rounds, %.4g "
                   "gradient entries)" % (R, m_kv, n, m_g, t_kv + t_g, work["mvp_entry_rhs"],
                                         work["mvp_rounds"], work["grad_entries"])),
        "host_seconds": t_kv + t_g,
    }


def _work_from_file():
    kv = _kv_file(WORK_FILE)
    if not kv:
        return None
    return {"mvp_entry_rhs": float(kv["mvp_entry_rhs_per_step"]),
            "grad_entries": float(kv["grad_entries_per_step"]),
            "mvp_rounds": float(kv["mvp_rounds_per_step"])}


# ----------------------------------------------------------------------------------------
# distributed helpers (replicas)
# ----------------------------------------------------------------------------------------
def max_over_ranks(v, world, device):
    """The largest of v over all ranks (the slowest rank's time); v itself with one rank."""
    if world <= 1:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def dist_setup(args, backend):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return world, rank, local


def run_reference(args):
    world, rank, _ = dist_setup(args, "gloo")
    if rank != 0:
        return 0
    from paper_1501_05427_gb300 import workloads as w
    prob = w.census_like()
    work = _work_from_file()
    if work is None:
        raise SystemExit("missing %s (per-step work of the workload)" % WORK_FILE)
    per_step = max(0.5, args.cpu_seconds / max(args.steps, 1))   # whole run: a minute or two
    for _ in range(args.warmup):
        oracle_sample(prob, work, per_step / 4)
    rates, host = [], 0.0
    t0 = time.perf_counter()
    for k in range(args.steps):
        r = oracle_sample(prob, work, per_step, rng_seed=k)
        rates.append(r)
        host += r["host_seconds"]
    wall = time.perf_counter() - t0
    t_step = statistics.mean(1.0 / r["steps_per_s"] for r in rates)
    value = 1.0 / t_step
    line = {
        "impl": "reference", "metric": "SGLD steps/s", "value": value, "unit": "steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * t_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": prob.n, "d": prob.d, "n_probes": N_PROBES},
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": rates[-1]["cores"],
                         "kind": "oracle", "sample": rates[-1]["sample"],
                         "extrapolated": True},
        "extrapolated": True,
        "extrapolation": ("each step is a timed sample of the oracle's two O(n^2) routines on "
                          "a row subset of the full workload, scaled by n/m and by the "
                          "chosen GPU path's work per step; no full step of the oracle runs "
                          "(one would take minutes)"),
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }
    print(json.dumps(line))
    return 0


def _timed_steps(ctx, dev, stream, psi0, K, W, step_base, flush, barrier, sampler=None):
    """W untimed steps, then K steps each bracketed by CUDA events on the library's stream,
    with an L2 flush (outside the spans) before each.  Every step starts from psi0 with its
    own step number (its own probes and truncation draws): with a constant step size the
    heavy-tailed gradient estimate lets a long chain jump far from the posterior, and the
    throughput is measured at the workload's parameters."""
    import torch
    psi_start = torch.tensor(psi0, dtype=torch.float64, device=dev)
    psi_dev = psi_start.clone()
    eps_dev = torch.full((max(K, W, 1),), EPS_T, dtype=torch.float64, device=dev)
    for k in range(W):
        psi_dev.copy_(psi_start)
        ctx.sgld_chain(psi_dev, eps_dev[:1], step0=step_base + k)
    c0 = ctx.counters()
    events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(K)]
    if sampler:
        sampler.start()
    barrier()
    torch.cuda.synchronize(dev)
    rounds = []
    for k in range(K):
        psi_dev.copy_(psi_start)          # every step from the same parameters (see DESIGN)
        flush.zero_()
        events[k][0].record(stream)
        ctx.sgld_chain(psi_dev, eps_dev[k:k + 1], step0=step_base + W + k)
        events[k][1].record(stream)
        rounds.append(ctx.counters()[0])
    torch.cuda.synchronize(dev)
    barrier()
    clocks = sampler.stop() if sampler else None
    c1 = ctx.counters()
    rounds = [b - a for a, b in zip([c0[0]] + rounds[:-1], rounds)]
    step_ms = [a.elapsed_time(b) for a, b in events]
    return {"step_ms": step_ms, "total_ms": sum(step_ms), "rounds": rounds,
            "counters": tuple(b - a for a, b in zip(c0, c1)), "clocks": clocks}


def _fit_step_time(step_ms, rounds):
    """Least-squares step_ms = fixed + per_round * rounds over the timed steps: the two paths
    follow different CG trajectories (different round counts), so they are also compared
    at the same number of rounds."""
    import numpy as np
    r = np.asarray(rounds, dtype=np.float64)
    t = np.asarray(step_ms, dtype=np.float64)
    if len(r) < 3 or np.ptp(r) == 0:
        return None
    A = np.column_stack([np.ones_like(r), r])
    (a, b), *_ = np.linalg.lstsq(A, t, rcond=None)
    return {"fixed_ms": float(a), "ms_per_round": float(b)}


def _profile_pass(ctx, dev, psi0, P, step_base, n, R):
    """P steps with event timing of every O(n^2) launch (this runs the host loop)."""
    import torch
    psi_dev = torch.tensor(psi0, dtype=torch.float64, device=dev)
    eps_dev = torch.full((max(P, 1),), EPS_T, dtype=torch.float64, device=dev)
    ctx.profile_enable(True)
    c0 = ctx.counters()
    ctx.sgld_chain(psi_dev, eps_dev[:P], step0=step_base)
    c1 = ctx.counters()
    prof = ctx.profile_read(reset=True)
    ctx.profile_enable(False)
    grad_entries = float(n) * n * R
    mvp_erhs = (c1[1] - c0[1]) - grad_entries * P
    return {
        "kmv_ms": prof["kmv_ms"], "kmv_flop": prof["kmv_flop"], "kmv_launches": prof["kmv_launches"],
        "grad_ms": prof["grad_ms"], "grad_flop": prof["grad_flop"],
        "mvp_entry_rhs": mvp_erhs, "rounds": c1[0] - c0[0], "steps": P,
        "kv_entry_rhs_per_s": mvp_erhs / (prof["kmv_ms"] / 1e3) if prof["kmv_ms"] > 0 else None,
        "kmv_tflops": (prof["kmv_flop"] / (prof["kmv_ms"] / 1e3) / 1e12
                       if prof["kmv_ms"] > 0 else None),
    }


# ----------------------------------------------------------------------------------------
# the other configurations (keys of the same line; rank 0 at N = 1)
# ----------------------------------------------------------------------------------------
def _exact_gradient_torch(X, y, psi, dev):
    """g_i = -1/2 Tr(K^-1 dK_i) + 1/2 y^T K^-1 dK_i K^-1 y in FP64 on the device (dense
    Cholesky through torch.linalg): the reference of the gradient-error measurement, n a few
    thousand.  Parameters psi = (log l_1..log l_d, log sigma^2, log lambda)."""
    import torch
    Xt = torch.from_numpy(X).to(dev, torch.float64)
    yt = torch.from_numpy(y).to(dev, torch.float64)
    n, d = Xt.shape
    ell = torch.tensor(psi[:d], dtype=torch.float64, device=dev).exp()
    s2, lam = math.exp(psi[d]), math.exp(psi[d + 1])
    Xs = Xt / ell
    diff2 = [(Xs[:, k, None] - Xs[None, :, k]) ** 2 for k in range(d)]
    Ks = s2 * torch.exp(-0.5 * sum(diff2))
    K = Ks + lam * torch.eye(n, dtype=torch.float64, device=dev)
    L = torch.linalg.cholesky(K)
    Kinv = torch.cholesky_inverse(L)
    a = torch.cholesky_solve(yt[:, None], L)[:, 0]
    g = []
    for dK in [Ks * diff2[k] for k in range(d)] + [Ks]:
        g.append(float(-0.5 * torch.sum(Kinv * dK) + 0.5 * a @ (dK @ a)))
    g.append(float(-0.5 * lam * torch.trace(Kinv) + 0.5 * lam * (a @ a)))
    return np.array(g)


def grad_error_leg(dev, stream, reps, prob=None):
    """Sec. 5's gradient error ||g - g~||^2 / ||g||^2 over `reps` seeded repetitions on a
    problem small enough for a dense Cholesky (default: Census-shaped, n = 4,000; 16 probes),
    at the generating parameters + 0.3 (where ||g|| is not ~0).  Paths: plain FP32 (probes
    redrawn every step, cold solves), mixed (tensor cores, same options) and the chosen form
    (mixed, probes reused for 20 steps, warm-started solves); same seeds on every path."""
    import torch

    from paper_1501_05427_gb300 import ulisse as u
    from paper_1501_05427_gb300 import workloads as w
    prob = prob if prob is not None else w.census_like(n=4000, seed=20150124)
    psi = prob.psi_true + 0.3
    t0 = time.perf_counter()
    g = _exact_gradient_torch(prob.X, prob.y, psi, dev)
    t_exact = time.perf_counter() - t0
    X = torch.from_numpy(prob.X).to(dev)
    y = torch.from_numpy(prob.y).to(dev)
    out = {"statistic": "||g - g~||^2 / ||g||^2 over %d seeded repetitions, %s "
                        "n=%d, d=%d, 16 probes, q=1, psi = truth + 0.3"
                        % (reps, prob.name, prob.n, prob.d),
           "g_norm": float(np.linalg.norm(g)),
           "reference": "dense FP64 Cholesky on the device (%.1f s)" % t_exact}
    legs = (("plain_fp32", u.PREC_FP32, 1, 0), ("mixed", u.PREC_MIXED, 1, 0),
            ("chosen", u.PREC_MIXED, 20, 1))
    for name, prec, refresh, warm in legs:
        cfg = u.ulisse_config_default(n_probes=16, precision=prec, seed=77,
                                      probe_refresh=refresh, warm_start_probes=warm,
                                      max_iter=1000)
        errs, rounds = [], []
        with u.Context(X, y, cfg, stream=stream) as ctx:
            for k in range(reps):
                r0 = ctx.counters()[0]
                gk, _ = ctx.grad(psi, step=k, allow=(u.ULISSE_ERR_MAXITER,))
                rounds.append(ctx.counters()[0] - r0)
                errs.append(float(np.sum((gk - g) ** 2) / np.sum(g * g)))
        e = np.array(errs)
        r = float(np.mean(rounds))
        out[name] = {"mean": float(e.mean()), "se": float(e.std(ddof=1) / math.sqrt(len(e))),
                     "median": float(np.median(e)), "p90": float(np.percentile(e, 90)),
                     "mvp_rounds_per_step": r,
                     # averaging m independent unbiased estimates divides the error by m at
                     # m times the rounds, so error x rounds is the cost of a given error
                     "median_x_rounds": float(np.median(e)) * r,
                     "p90_x_rounds": float(np.percentile(e, 90)) * r}
    base = out["plain_fp32"]
    out["rounds_at_equal_error_plain_over"] = {
        k: {"median": base["median_x_rounds"] / out[k]["median_x_rounds"],
            "p90": base["p90_x_rounds"] / out[k]["p90_x_rounds"]} for k in ("mixed", "chosen")}
    return out


def near_duplicates_subproblem_leg(dev, stream, reps):
    """The near-duplicate inputs (d = 16, 1% jittered copies) at n = 4,000, where a dense FP64
    Cholesky gives the exact values: the error of a converged solve K^{-1} y (q = 0) per path
    against the Cholesky solution, and the gradient-error statistic of grad_error_leg."""
    import torch

    from paper_1501_05427_gb300 import ulisse as u
    from paper_1501_05427_gb300 import workloads as w
    prob = w.near_duplicates(n=4000)
    psi = prob.psi_true + 0.3
    Xd = torch.from_numpy(prob.X).to(dev, torch.float64)
    yd = torch.from_numpy(prob.y).to(dev, torch.float64)
    ell = torch.tensor(psi[:prob.d], dtype=torch.float64, device=dev).exp()
    s2, lam = math.exp(psi[prob.d]), math.exp(psi[prob.d + 1])
    Xs = Xd / ell
    K = s2 * torch.exp(-0.5 * torch.cdist(Xs, Xs) ** 2) + lam * torch.eye(prob.n, device=dev,
                                                                           dtype=torch.float64)
    s_exact = torch.linalg.solve(K, yd)
    cond = float(torch.linalg.cond(K))
    X = torch.from_numpy(prob.X).to(dev)
    y = torch.from_numpy(prob.y).to(dev)
    out = {"workload": "near_duplicates", "n": prob.n, "d": prob.d,
           "duplicates": int(prob.meta["duplicates"]), "cond_K": cond, "solve": {}}
    for name, prec in (("fp32", u.PREC_FP32), ("mixed", u.PREC_MIXED)):
        cfg = u.ulisse_config_default(precision=prec, q=0.0, eps=1e-3, max_iter=5000)
        with u.Context(X, y, cfg, stream=stream) as ctx:
            S, st = ctx.solve(psi, y[:, None], allow=(u.ULISSE_ERR_MAXITER,))
        sv = S[:, 0].double()
        out["solve"][name] = {
            "iterations": int(st[0][1]),
            "rel_error_vs_cholesky": float(torch.linalg.norm(sv - s_exact) /
                                           torch.linalg.norm(s_exact)),
            "rel_residual": float(torch.linalg.norm(yd - K @ sv) / torch.linalg.norm(yd))}
    out["solve"]["stopping_rule"] = ("||y - K s|| < 1e-3 (FP32 vectors); the solution error "
                                     "is bounded by that residual / lambda_min(K)")
    out["gradient_error"] = grad_error_leg(dev, stream, reps, prob)
    return out


def learned_warm_start_leg(dev, stream, rec_steps=1000, rec_every=4, n_eval=16, var_cols=8,
                           var_calls=3):
    """The learned warm start x0 = K_s(X, Z) c, c = MLP(psi), at the workload it is meant for
    (n = 100,000, d = 8, 16 probes, noise variance 0.05): pairs are recorded along the first
    `rec_steps` steps of a parameter trajectory (every `rec_every`-th step, at most 256 pairs),
    the network is trained on them, and on held-out parameters the y solve (q = 1, two
    estimators) is run from x0 = 0, from the pooled constant c (the network's starting point)
    and from the trained network: CG iterations (= K V products) of each, and the variance of
    the y term 1/2 s1^T dK s2 of the gradient with and without the learned start.

    The trajectory is a seeded AR(1) walk around the generating parameters (stationary s.d.
    0.046 per coordinate), a stand-in for the chain's states: a free-running chain at a
    constant step size is thrown by the heavy-tailed gradient estimates (see the chain
    test), and the walk gives the network the same kind of parameter spread to learn from."""
    import torch

    from paper_1501_05427_gb300 import ulisse as u
    from paper_1501_05427_gb300 import workloads as w
    prob = w.warm_start_problem()
    n, p = prob.n, prob.d + 2
    rng = np.random.default_rng(20150105)
    walk, z = [], np.zeros(p)
    for _ in range(rec_steps + rec_every * n_eval):
        z = 0.9 * z + 0.02 * rng.standard_normal(p)
        walk.append(prob.psi_true + z)
    X = torch.from_numpy(prob.X).to(dev)
    y = torch.from_numpy(prob.y).to(dev)
    cfg = u.ulisse_config_default(precision=u.PREC_MIXED, n_probes=16, probe_refresh=20,
                                  warm_start_probes=1, seed=55, max_iter=3000)
    allow = (u.ULISSE_ERR_MAXITER,)
    out = {"workload": "warm_start (census_like shape)", "n": n, "d": prob.d, "n_probes": 16,
           "network": "MLP %d -> 256 -> 256 -> 512 (tanh), 512 anchors, FP32 training, BF16 "
                      "inference" % p,
           "trajectory": "AR(1) walk around the generating parameters, s.d. 0.046",
           "recorded": "%d pairs from the first %d steps (every %d-th)"
                       % (min(256, rec_steps // rec_every), rec_steps, rec_every)}
    with u.Context(X, y, cfg, stream=stream) as ctx:
        ctx.ws_init(n_anchors=512, hidden=256, n_rows=1024, max_pairs=256, seed=1)
        # a recorded pair (psi_t, rows, y_rows, K(X_rows, X) K_s(X, Z)) does not depend on the
        # step's solves, so only the recorded steps are run (plus a few plain ones, timed for
        # the recording's cost)
        t_rec = t_plain = 0.0
        n_rec = n_plain = 0
        for t in range(rec_steps):
            rec = (t % rec_every == 0)
            if not rec and n_plain >= 20:
                continue
            ctx.ws_set(record=rec, use=False)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.grad(walk[t], step=t, allow=allow)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            if rec:
                t_rec += dt
                n_rec += 1
            else:
                t_plain += dt
                n_plain += 1
        out["step_ms_recording"] = 1e3 * t_rec / max(n_rec, 1)
        out["step_ms_not_recording"] = 1e3 * t_plain / max(n_plain, 1)
        ctx.ws_set(record=False, use=False)
        held = [walk[rec_steps + rec_every * k] for k in range(n_eval)]
        # held-out loss of the pooled constant: one Adam step of negligible size, validated
        # against the pooled start it begins from
        out["pooled_heldout_loss"] = ctx.ws_train(steps=1, batch=64, lr=1e-12)
        ctx.ws_train(steps=0, batch=64)
        x_pool = [ctx.ws_x0(ps, bf16=True).clone() for ps in held]
        t0 = time.perf_counter()
        loss = ctx.ws_train(steps=600, batch=64, lr=2e-3)
        out["training_s"] = time.perf_counter() - t0
        out["training_heldout_loss"] = loss
        x_net = [ctx.ws_x0(ps, bf16=True).clone() for ps in held]
        its = {"x0_zero": [], "pooled_constant": [], "network": []}
        for k, ps in enumerate(held):
            for name, s0 in (("x0_zero", None), ("pooled_constant", x_pool[k][:, None]),
                             ("network", x_net[k][:, None])):
                _, st = ctx.solve(ps, y[:, None], n_est=[2], S0=s0, step=50_000 + k,
                                  allow=allow)
                its[name].append(int(st[0][1]))
        out["y_solve_iterations_heldout"] = {
            k: {"mean": float(np.mean(v)), "median": float(np.median(v))} for k, v in its.items()}
        out["kv_products_saved_vs_x0_zero"] = {
            k: 1.0 - float(np.mean(its[k])) / float(np.mean(its["x0_zero"]))
            for k in ("pooled_constant", "network")}
        # variance of the y term of the gradient at one held-out point: var_cols columns of y
        # per call (independent truncation draws per column), var_calls calls
        ps = held[0]
        B = y[:, None].repeat(1, var_cols)
        terms = {"x0_zero": [], "pooled_constant": [], "network": []}
        iters = {"x0_zero": [], "pooled_constant": [], "network": []}
        for name, s0 in (("x0_zero", None),
                         ("pooled_constant", x_pool[0][:, None].repeat(1, var_cols)),
                         ("network", x_net[0][:, None].repeat(1, var_cols))):
            for c in range(var_calls):
                S, st = ctx.solve(ps, B, n_est=[2] * var_cols, S0=s0, step=60_000 + c,
                                  allow=allow)
                iters[name] += [int(e[1]) for e in st]
                for j in range(var_cols):
                    terms[name].append(ctx.dk_bilinear(ps, S[:, 2 * j:2 * j + 1],
                                                       S[:, 2 * j + 1:2 * j + 2], [0.5]))
        var = {k: float(np.var(np.array(v), axis=0, ddof=1).sum()) for k, v in terms.items()}
        it = {k: float(np.mean(v)) for k, v in iters.items()}
        out["y_term_gradient_variance"] = {
            "samples": var_cols * var_calls,
            "trace": var, "iterations": it,
            "variance_ratio_over_x0_zero": {k: var[k] / var["x0_zero"]
                                            for k in ("pooled_constant", "network")},
            "variance_x_iterations_ratio_over_x0_zero": {
                k: var[k] * it[k] / (var["x0_zero"] * it["x0_zero"])
                for k in ("pooled_constant", "network")}}
    return out


def _event_time(fn, stream, flush, reps, warm=2):
    """Median CUDA-event time (ms) of fn() on `stream`, L2 flushed before each launch."""
    import torch
    for _ in range(warm):
        fn()
    ts = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def near_duplicates_leg(dev, stream, flush, rows_oracle):
    """K V at the near-duplicate workload's full size (n = 200,000, d = 16, 1% jittered
    copies, 64 right-hand sides): entry-RHS/s of the tensor-core path and of the FP32 SIMT
    path, and their error against the FP64 oracle on `rows_oracle` sampled output rows (the
    oracle's time for those rows is its CPU baseline at this size)."""
    import torch

    from paper_1501_05427_gb300 import ulisse as u
    from paper_1501_05427_gb300 import workloads as w
    prob = w.near_duplicates()
    n, d, R = prob.n, prob.d, 64
    X = torch.from_numpy(prob.X).to(dev)
    y = torch.from_numpy(prob.y).to(dev)
    V = torch.from_numpy(np.random.default_rng(64).standard_normal((n, R)).astype(np.float32))
    Vd = V.to(dev).t().contiguous().t()          # column-major, as the library takes it
    out = {"workload": "near_duplicates", "n": n, "d": d, "rhs": R,
           "duplicates": int(prob.meta["duplicates"])}
    res = {}
    for name, prec in (("mixed", u.PREC_MIXED), ("fp32", u.PREC_FP32)):
        cfg = u.ulisse_config_default(precision=prec, n_probes=16)
        with u.Context(X, y, cfg, stream=stream) as ctx:
            U = torch.empty((R, n), dtype=torch.float32, device=dev).t()
            ms = _event_time(lambda: ctx.kmv(prob.psi_true, Vd, out=U), stream, flush, 5)
            res[name] = U.cpu().numpy()
        out[name] = {"ms_per_launch": ms, "entry_rhs_per_s": float(n) * n * R / (ms / 1e3)}
    out["speedup_mixed_over_fp32"] = out["fp32"]["ms_per_launch"] / out["mixed"]["ms_per_launch"]
    if rows_oracle > 0:
        import oracle
        oracle.build()
        rows = np.sort(np.random.default_rng(7).choice(n, rows_oracle, replace=False))
        t0 = time.perf_counter()
        ref = oracle.kmv_rows(prob.X.astype(np.float64), prob.psi_true,
                              V.numpy().astype(np.float64), rows)
        t_orc = time.perf_counter() - t0
        for name in ("mixed", "fp32"):
            Ur = res[name][rows].astype(np.float64)
            out[name]["error_vs_oracle"] = {
                "rows": int(rows_oracle),
                "frobenius_rel": float(np.linalg.norm(Ur - ref) / np.linalg.norm(ref)),
                "max_col_rel": float(np.max(np.linalg.norm(Ur - ref, axis=0) /
                                            np.linalg.norm(ref, axis=0))),
                "max_abs_over_max_ref": float(np.max(np.abs(Ur - ref)) / np.max(np.abs(ref)))}
        out["cpu_baseline"] = {"value": rows_oracle * float(n) * R / t_orc,
                               "unit": "entry·RHS/s", "cores": oracle.omp_threads(),
                               "kind": "oracle", "extrapolated": False,
                               "sample": "oracle K V of %d output rows against all %d inputs, "
                                         "64 RHS, %.1f s" % (rows_oracle, n, t_orc)}
    return out


def small_2d_leg(dev, stream, n_steps=100):
    """The 2-D FP64 configuration: n = 1,000, 4 Gaussian probes, 100 SGLD steps at step size
    1e-4 from the generating parameters, as one chain (one graph launch per step) on the FP64
    and the FP32 path, and the oracle's full 100-step chain on the host cores (timed, not
    extrapolated)."""
    import torch

    import oracle
    from paper_1501_05427_gb300 import ulisse as u
    from paper_1501_05427_gb300 import workloads as w
    prob = w.small_2d()
    X = torch.from_numpy(prob.X).to(dev)
    y = torch.from_numpy(prob.y).to(dev)
    p = prob.d + 2
    out = {"workload": "small_2d", "n": prob.n, "d": prob.d, "n_probes": 4,
           "probe_kind": "gaussian", "steps": n_steps, "eps_t": 1e-4}
    finals = {}
    for name, prec in (("fp64", u.PREC_FP64), ("fp32", u.PREC_FP32)):
        cfg = u.ulisse_config_default(precision=prec, n_probes=4, probe_kind=u.PROBE_GAUSSIAN,
                                      q=1.0, beta=1.0, max_iter=2000, seed=20150122)
        with u.Context(X, y, cfg, stream=stream) as ctx:
            eps = torch.full((n_steps,), 1e-4, dtype=torch.float64, device=dev)
            psi = torch.tensor(prob.psi_true, dtype=torch.float64, device=dev)
            ctx.sgld_chain(psi, eps[:5], step0=10_000)          # warm-up (graph build)
            psi.copy_(torch.tensor(prob.psi_true, dtype=torch.float64))
            r0 = ctx.counters()[0]
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            a.record(stream)
            ctx.sgld_chain(psi, eps, step0=0, allow=(u.ULISSE_ERR_MAXITER,))
            b.record(stream)
            b.synchronize()
            ms = a.elapsed_time(b)
            # the same chain again with its trace (outside the timed span)
            trace = torch.zeros((n_steps, p), dtype=torch.float64, device=dev)
            psi.copy_(torch.tensor(prob.psi_true, dtype=torch.float64))
            ctx.sgld_chain(psi, eps, step0=0, trace_dev=trace, allow=(u.ULISSE_ERR_MAXITER,))
            finals[name] = trace.cpu().numpy()
            out[name] = {"steps_per_s": n_steps / (ms / 1e3), "ms_per_step": ms / n_steps,
                         "mvp_rounds_per_step": (ctx.counters()[0] - r0) / n_steps}
    oracle.build()
    Xd, yd = prob.X.astype(np.float64), prob.y.astype(np.float64)
    psi = prob.psi_true.copy()
    orc_trace = []
    t0 = time.perf_counter()
    for k in range(n_steps):
        psi, _, _ = oracle.sgld_step(Xd, yd, psi, 1e-4, nr=4, probe_kind=1, q=1.0, beta=1.0,
                                     max_iter=2000, seed=20150122, step=k)
        orc_trace.append(psi)
    t_orc = time.perf_counter() - t0
    orc_trace = np.array(orc_trace)
    out["cpu_baseline"] = {"value": n_steps / t_orc, "unit": "steps/s",
                           "cores": oracle.omp_threads(), "kind": "oracle",
                           "extrapolated": False,
                           "sample": "the oracle's full %d-step chain (%.1f s)" % (n_steps, t_orc)}
    # the chains run the same draws; the FP64 one follows the oracle's chain until rounding
    # flips a discrete decision (an early stop near its threshold) on an ill-conditioned solve
    track = {}
    for k, tr in finals.items():
        dif = np.max(np.abs(tr - orc_trace), axis=1)
        off = np.nonzero(dif > 1e-6)[0]
        track[k] = {"steps_within_1e-6": int(off[0]) if len(off) else n_steps,
                    "max_abs_diff_first_10": float(dif[:10].max()),
                    "final_max_abs_diff": float(dif[-1])}
    out["psi_vs_oracle_chain"] = track
    return out


def pcg_leg(dev, stream, flush, X, y, psi0, steps=6, warm=2):
    """Sec. 3's preconditioned CG (J = K + delta I, inner CG to ||r|| <= 0.1 ||e||) with ULISSE
    on the outer iteration, against plain CG, both with cold solves (probes redrawn every
    step: every step is a probe-epoch start) on the tensor-core path, from the host loop:
    K V rounds per step (outer and inner) and steps/s, for a few delta (the paper tunes
    delta for the fewest iterations)."""
    import torch

    from paper_1501_05427_gb300 import ulisse as u
    out = {"solves": "cold (zero start), probes redrawn every step", "inner_tol": 0.1,
           "inner_max": 50, "step_form": "host loop"}
    legs = [("cg", 0.0)] + [("pcg_delta_%g" % dl, dl) for dl in (0.1, 0.5, 2.0)]
    for name, dl in legs:
        cfg = u.ulisse_config_default(n_probes=N_PROBES, precision=u.PREC_MIXED, q=1.0, beta=1.0,
                                      max_iter=1000, seed=20150123, pcg_delta=dl,
                                      pcg_inner_tol=0.1, pcg_inner_max=50)
        with u.Context(X, y, cfg, stream=stream) as ctx:
            ctx.set_graph(False)
            for k in range(warm):
                ctx.sgld_step(psi0, EPS_T, step=10_000 + k, allow=(u.ULISSE_ERR_MAXITER,))
            r0 = ctx.counters()[0]
            ms = []
            for k in range(steps):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize(dev)
                a.record(stream)
                ctx.sgld_step(psi0, EPS_T, step=k, allow=(u.ULISSE_ERR_MAXITER,))
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
            out[name] = {"steps_per_s": 1000.0 * steps / sum(ms),
                         "mvp_rounds_per_step": (ctx.counters()[0] - r0) / steps}
    best = min((k for k in out if k.startswith("pcg_")), key=lambda k: out[k]["mvp_rounds_per_step"])
    out["fewest_rounds"] = best
    out["rounds_pcg_over_cg"] = out[best]["mvp_rounds_per_step"] / out["cg"]["mvp_rounds_per_step"]
    return out


def uneven_batch_leg(args, dev, stream, flush, K=5, W=2):
    """The 64-problem uneven batch, one graph launch per batched step (see run_batch): the
    chosen path's line, with the other precision's measurement beside it."""
    line = _batch_measure(args, dev, stream, flush, K, W, sampler=None)
    other = "fp32" if args.path == "mixed" else "mixed"
    o = _batch_measure(args, dev, stream, flush, K, W, sampler=None, path=other)
    line[other] = {k: o[k] for k in ("value", "ms_per_step", "mvp_rounds_per_step", "dtype",
                                      "steps_with_a_column_cut_at_max_iter")}
    return line


def run_ours(args):
    import numpy as np
    import torch

    from paper_1501_05427_gb300 import ulisse as u
    from paper_1501_05427_gb300 import workloads as w

    world, rank, local = dist_setup(args, "nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prob = w.census_like()
    n, d = prob.n, prob.d
    p, R = d + 2, 1 + N_PROBES
    X = torch.from_numpy(prob.X).to(dev)
    y = torch.from_numpy(prob.y).to(dev)
    stream = torch.cuda.current_stream(dev)
    K, W = args.steps, args.warmup
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    tuned = {}

    def make_ctx(path, refresh, warm, key):
        prec = u.PREC_MIXED if path == "mixed" else u.PREC_FP32
        cfg = u.ulisse_config_default(n_probes=N_PROBES, probe_kind=u.PROBE_RADEMACHER, q=1.0,
                                      beta=1.0, eps=1e-8, max_iter=1000,
                                      seed=20150123 + rank, precision=prec,
                                      probe_refresh=refresh, warm_start_probes=int(warm))
        c = u.Context(X, y, cfg, stream=stream)
        c.set_graph(not args.no_graph)
        if not args.no_tune:
            tuned[key] = c.autotune(prob.psi_true, R, reps=3)
        return c

    def max_ranks(v):
        return max_over_ranks(v, world, dev)

    # the exponential unit's throughput on this device (the mixed path's roofline)
    ex2_rate, ex2_ms = u.ulisse_measure_ex2_rate(stream, reps=20)

    # chosen path: the timed region
    warm = not args.no_warm
    ctx = make_ctx(args.path, args.refresh, warm, "chosen")
    res = _timed_steps(ctx, dev, stream, prob.psi_true, K, W, 0, flush, barrier,
                       ClockSampler(local))
    total_ms = max_ranks(res["total_ms"])
    value = world * K / (total_ms / 1000.0)
    rounds, erhs, launches = res["counters"]

    # per-launch K V and gradient times (event-timed pass of the same workload)
    prof = _profile_pass(ctx, dev, prob.psi_true, args.profile_steps, 50_000, n, R)

    # end to end through the host-buffer API (psi in, psi and g out every step), replaying
    # exactly the timed steps: same parameters, same step numbers, so the same draws and rounds
    for k in range(W):
        ctx.sgld_step(prob.psi_true.copy(), EPS_T, step=k)
    barrier()
    torch.cuda.synchronize(dev)
    r_e0 = ctx.counters()[0]
    t0 = time.perf_counter()
    for k in range(K):
        psi_h, g_h = ctx.sgld_step(prob.psi_true.copy(), EPS_T, step=W + k)
    torch.cuda.synchronize(dev)
    e2e_s = max_ranks(time.perf_counter() - t0)
    e2e_rounds = (ctx.counters()[0] - r_e0) / max(K, 1)
    e2e_value = world * K / e2e_s
    ctx.close()

    # plain FP32 path (probes redrawn every step, cold solves: the method as stated), and
    # FP32 with the chosen path's method options (isolates the arithmetic), same form
    def other_leg(path, refresh, warm_leg, key):
        octx = make_ctx(path, refresh, warm_leg, key)
        ores = _timed_steps(octx, dev, stream, prob.psi_true, K, W, 0, flush, barrier)
        oprof = _profile_pass(octx, dev, prob.psi_true, args.profile_steps, 50_000, n, R)
        octx.close()
        ototal = max_ranks(ores["total_ms"])
        return {"value": world * K / (ototal / 1000.0), "unit": "steps/s",
                "ms_per_step": ototal / K,
                "mvp_rounds_per_step": ores["counters"][0] / K,
                "step_time_fit": _fit_step_time(ores["step_ms"], ores["rounds"]),
                "kv_entry_rhs_per_s": oprof["kv_entry_rhs_per_s"],
                "kmv_ms_per_round": (oprof["kmv_ms"] / oprof["rounds"] if oprof["rounds"] else None),
                "kernel": KMV_KERNELS[kernel_key(path, tuned.get(key), R)][0],
                "probe_refresh": refresh,
                "warm_started_solves": bool(warm_leg)}

    plain = same_method = None
    if not args.no_plain:
        plain = other_leg("fp32", 1, False, "plain_fp32")
        if args.path != "fp32" or warm or args.refresh != 1:
            same_method = other_leg("fp32", args.refresh, warm, "fp32_same_method")

    fit = _fit_step_time(res["step_ms"], res["rounds"])
    # the arithmetic alone: chosen vs FP32 with the same method options, at the same rounds
    at_equal = None
    ref = same_method or plain
    if ref and fit and ref.get("step_time_fit"):
        r_bar = rounds / K
        t_c = fit["fixed_ms"] + fit["ms_per_round"] * r_bar
        t_p = ref["step_time_fit"]["fixed_ms"] + ref["step_time_fit"]["ms_per_round"] * r_bar
        at_equal = {"rounds_per_step": r_bar, "chosen_steps_per_s": 1000.0 / t_c,
                    "fp32_steps_per_s": 1000.0 / t_p, "speedup": t_p / t_c,
                    "fp32_leg": "fp32_same_method" if same_method else "plain_fp32"}
    kkey = kernel_key(args.path, tuned.get("chosen"), R)
    name, traffic_file, _ = KMV_KERNELS[kkey]
    traffic = None
    tf = _kv_file(traffic_file)
    if tf and tf.get("kmv_source_hash") == kmv_source_hash(kkey):
        traffic = float(tf["dram_bytes_per_launch"])
    kmv_s = prof["kmv_ms"] / 1e3
    launches_kv = prof["kmv_launches"]
    # algorithmic work per K V launch (the method's, Sec. 3): k_ij = k_ji, so n(n+1)/2
    # distinct kernel values (distance and exponential), and the n^2 R multiply-adds of the
    # contraction
    distinct = float(n) * (n + 1) / 2.0
    alg_flop = launches_kv * (distinct * (3.0 * d + 2.0) + 2.0 * R * float(n) * n)
    alg_tflops = alg_flop / kmv_s / 1e12 if kmv_s > 0 else None
    flop_view = {"unit": "TFLOP/s", "achieved": alg_tflops, "peak": FP32_FMA_PEAK_TFLOPS,
                 "frac": (alg_tflops / FP32_FMA_PEAK_TFLOPS) if alg_tflops else None,
                 "flop_per_launch": "n(n+1)/2 (3d + 2) + 2 R n^2 (distinct kernel values, "
                                    "contraction)",
                 "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop/FMA x 2070 MHz"}
    ex2_peak = ex2_rate / 1e12
    if kkey == "mixed_tensor":
        # the cross term and the contraction run on the tensor cores; what every kernel value
        # still needs on the CUDA cores is one exponential (ex2 on the XU pipe)
        exps = launches_kv * distinct / kmv_s if kmv_s > 0 else None
        gen = launches_kv * generated_entries(n) / kmv_s if kmv_s > 0 else None
        roofline = {
            "bound": "alu",
            "kernel": name,
            "achieved": exps / 1e12 if exps else None,
            "peak": ex2_peak,
            "unit": "T exp/s",
            "frac": (exps / 1e12 / ex2_peak) if exps else None,
            "work_per_launch": "n(n+1)/2 exponentials (the distinct kernel values; k_ij = "
                               "k_ji), n = %d" % n,
            "peak_source": "measured: ulisse_measure_ex2_rate, best of 20 launches of "
                           "independent ex2.approx.ftz.f32 on every SM (%.3f ms); derived "
                           "152 x 32/clk x 2070 MHz = %.2f" % (ex2_ms, EX2_PEAK_DERIVED_TENTRIES),
            "generated_entries_per_s": gen / 1e12 if gen else None,
            "generated_entries_per_launch": generated_entries(n),
            "traffic": traffic,
            "fp32_equivalent_flops": flop_view,
        }
    else:
        roofline = {
            "bound": "alu",
            "kernel": name,
            "achieved": alg_tflops,
            "peak": FP32_FMA_PEAK_TFLOPS,
            "peak_source": flop_view["peak_source"],
            "unit": "TFLOP/s",
            "frac": flop_view["frac"],
            "traffic": traffic,
            "flop_per_launch": flop_view["flop_per_launch"],
            "ex2_peak_measured": ex2_peak,
        }
    roofline.update({
        "traffic_unit": "DRAM bytes per launch (ncu capture of the dominant instance; see its file)",
        "measured_in": "event-timed pass of %d steps (host loop, one event pair per launch)"
                       % prof["steps"],
        "kmv_launches": prof["kmv_launches"],
        "kmv_ms_per_round": prof["kmv_ms"] / prof["rounds"] if prof["rounds"] else None,
        "kmv_ms_per_launch": prof["kmv_ms"] / prof["kmv_launches"] if prof["kmv_launches"] else None,
        "grad_ms_per_step": prof["grad_ms"] / prof["steps"],
        "grad_tflops": (prof["grad_flop"] / (prof["grad_ms"] / 1e3) / 1e12
                        if prof["grad_ms"] > 0 else None),
        "grad_flop_per_launch": ("n(n+1)/2 (5d + 4 + 4M): each unordered pair once, 2M factor "
                                 "products" if args.path == "mixed"
                                 else "n^2 (5d + 4 + 2M): every ordered pair"),
    })
    extras = {}
    if world == 1 and not args.no_extras:
        extras["gradient_error"] = grad_error_leg(dev, stream, args.grad_reps)
        extras["near_duplicates_kv"] = near_duplicates_leg(dev, stream, flush, args.c3_rows)
        extras["near_duplicates_subproblem"] = near_duplicates_subproblem_leg(
            dev, stream, max(10, args.grad_reps // 2))
        if args.c5_steps > 0:
            extras["learned_warm_start"] = learned_warm_start_leg(dev, stream, args.c5_steps)
        extras["uneven_batch"] = uneven_batch_leg(args, dev, stream, flush)
        extras["small_2d_fp64_chain"] = small_2d_leg(dev, stream)
        extras["pcg"] = pcg_leg(dev, stream, flush, X, y, prob.psi_true)
    line = {
        "metric": "SGLD steps/s", "value": value, "unit": "steps/s", "n_gpus": world,
        "steps": K, "warmup": W, "ms_per_step": total_ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x3/f32" if args.path == "mixed" else "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "d": d, "n_probes": N_PROBES, "q": 1.0,
                   "beta": 1.0, "eps_t": EPS_T,
                   "path": ("tcgen05 mixed precision: K V with the exponent's dot product "
                            "by 3xTF32 and the contraction by 3xBF16, gradient pass by 3xBF16, "
                            "FP32 accumulation"
                            if args.path == "mixed" else "fp32 SIMT K V and gradient"),
                   "step_form": "host loop" if args.no_graph else "one CUDA graph launch per step",
                   "probe_refresh": args.refresh, "warm_started_solves": warm,
                   "steps_start_at": "the generating parameters (own step number each)",
                   "l2": "flushed between timed steps (512 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "kv_throughput": {"value": prof["kv_entry_rhs_per_s"], "unit": "entry·RHS/s",
                          "plain_fp32": plain["kv_entry_rhs_per_s"] if plain else None},
        "plain_fp32": plain,
        "fp32_same_method": same_method,
        "autotune": ({path: {"tuned_over_untuned_ms": [round(e["ms"] / e["ms_default"], 3)
                                                      for e in tab],
                             "cross_term": [e["cross_term"] for e in tab],
                             "width": [e["width"] for e in tab],
                             "nsplit": [e["nsplit"] for e in tab]}
                      for path, tab in tuned.items()} if tuned else None),
        "gradient_error": extras.get("gradient_error"),
        "near_duplicates_kv": extras.get("near_duplicates_kv"),
        "near_duplicates_subproblem": extras.get("near_duplicates_subproblem"),
        "learned_warm_start": extras.get("learned_warm_start"),
        "uneven_batch": extras.get("uneven_batch"),
        "small_2d_fp64_chain": extras.get("small_2d_fp64_chain"),
        "pcg": extras.get("pcg"),
        "mvp_rounds_per_step": rounds / K,
        "step_time_fit": fit,
        "at_equal_rounds": at_equal,
        "rounds_per_step": res["rounds"],
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": "steps/s", "h2d_bytes_per_step": 8 * p + 8 + 32,
                "d2h_bytes_per_step": 16 * p + 32 + 4, "mvp_rounds_per_step": e2e_rounds,
                "api": "ulisse_sgld_step (host psi in, host psi and g out)",
                "steps": "the timed steps replayed (same start and step numbers)"},
        "gpu_launches": int(launches),
        "clocks": res["clocks"],
        "step_ms": res["step_ms"],
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        work = {"mvp_entry_rhs": erhs / K - float(n) * n * R, "grad_entries": float(n) * n,
                "mvp_rounds": rounds / K}
        cb = oracle_sample(prob, work, args.cpu_seconds)
        line["cpu_baseline"] = {"value": cb["steps_per_s"], "unit": "steps/s",
                                "cores": cb["cores"], "kind": "oracle", "sample": cb["sample"],
                                "extrapolated": True,
                                "extrapolation": "timed oracle rows scaled by n/m and by this "
                                                 "run's measured work per step",
                                "kv_entry_rhs_per_s": cb["kv_entry_rhs_per_s"]}
        line["work_per_step"] = {"mvp_entry_rhs_per_step": work["mvp_entry_rhs"],
                                 "grad_entries_per_step": work["grad_entries"],
                                 "mvp_rounds_per_step": work["mvp_rounds"]}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _batch_measure(args, dev, stream, flush, K, W, sampler=None, world=1, rank=0, path=None):
    """The 64-problem uneven workload: one batched SGLD step of all problems per graph launch
    (mixed: every CG round's K V of all problems on the tensor cores in one launch; FP32: one
    persistent K V launch; the gradient sweep in one persistent FP32 launch).  Returns the
    measurement."""
    import torch

    from paper_1501_05427_gb300 import ulisse as u
    from paper_1501_05427_gb300 import workloads as w
    probs = w.uneven_batch()
    # the slowest of 576 columns decides a batched step's rounds; a column that has not
    # stopped after max_iter CG iterations is cut off (reported, not fatal)
    warm = not args.no_warm
    path = path or args.path
    prec = u.PREC_MIXED if path == "mixed" else u.PREC_FP32
    cfg = u.ulisse_config_default(precision=prec, n_probes=8, probe_kind=u.PROBE_RADEMACHER,
                                  q=1.0, beta=1.0,
                                  eps=1e-8, max_iter=3000, seed=20150126 + 1000 * rank,
                                  probe_refresh=args.refresh, warm_start_probes=int(warm))
    allow = (u.ULISSE_ERR_MAXITER,)
    cut = 0
    Xs = [torch.from_numpy(p.X).to(dev) for p in probs]
    ys = [torch.from_numpy(p.y).to(dev) for p in probs]
    bc = u.BatchContext(Xs, ys, cfg, stream=stream)
    bc.set_graph(not args.no_graph)
    psi = torch.tensor(np.concatenate([p.psi_true for p in probs]), dtype=torch.float64,
                       device=dev)
    eps = torch.full((max(K, W, 1),), EPS_T, dtype=torch.float64, device=dev)
    psi_start = psi.clone()
    for k in range(W):
        psi.copy_(psi_start)
        bc.sgld_chain(psi, eps[:1], step0=k, allow=allow)
    c0 = bc.counters()
    events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(K)]
    if sampler:
        sampler.start()
    torch.cuda.synchronize(dev)
    rounds = []
    for k in range(K):
        psi.copy_(psi_start)
        flush.zero_()
        events[k][0].record(stream)
        st = bc.sgld_chain_status(psi, eps[k:k + 1], step0=W + k)
        events[k][1].record(stream)
        cut += int(st == u.ULISSE_ERR_MAXITER)
        rounds.append(bc.counters()[0])
    torch.cuda.synchronize(dev)
    clocks = sampler.stop() if sampler else None
    c1 = bc.counters()
    rounds = [b - a for a, b in zip([c0[0]] + rounds[:-1], rounds)]
    step_ms = [a.elapsed_time(b) for a, b in events]
    total_ms = sum(step_ms)
    n_sum = sum(p.n for p in probs)
    bc.close()
    return {
        "metric": "SGLD steps/s", "value": world * K * len(probs) / (total_ms / 1000.0),
        "unit": "problem-steps/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3/f32" if path == "mixed" else "f32",
        "data": "synthetic",
        "config": {"workload": "uneven_batch", "problems": len(probs), "n_total": n_sum,
                   "path": path,
                   "n_min": min(p.n for p in probs), "n_max": max(p.n for p in probs),
                   "dims": sorted(set(p.d for p in probs)), "n_probes": 8,
                   "step_form": "host loop" if args.no_graph else "one CUDA graph launch per batched step",
                   "probe_refresh": args.refresh, "warm_started_solves": warm,
                   "l2": "flushed between timed steps (512 MiB write)"},
        "batched_steps_per_s": K / (total_ms / 1000.0),
        "kv_throughput": {"value": (c1[1] - c0[1]) / (total_ms / 1000.0),
                          "unit": "entry·RHS/s (whole step: K V rounds and the gradient sweep)"},
        "mvp_rounds_per_step": (c1[0] - c0[0]) / K,
        "rounds_per_step": rounds,
        "steps_with_a_column_cut_at_max_iter": cut,
        "gpu_launches": int(c1[2] - c0[2]),
        "clocks": clocks,
        "step_ms": step_ms,
    }


def run_batch(args):
    """--workload uneven_batch: the batched line on its own."""
    import torch
    world, rank, local = dist_setup(args, "nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    line = _batch_measure(args, dev, stream, flush, args.steps, args.warmup,
                          sampler=ClockSampler(local), world=world, rank=rank)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "uneven_batch":
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
