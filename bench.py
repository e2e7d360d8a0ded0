#!/usr/bin/env python
"""SGLD + ULISSE benchmark on the Census-shaped workload (n = 50,000, d = 8, 16 probes).

One step = one pass of the whole path: parameter unpack and prescale, probe generation,
the batched ULISSE solves of K s = y (two estimators) and K s = r_j (j = 1..16), the fused
gradient pass and the SGLD update -- all in libulisse's CUDA kernels, launched through the
C ABI.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "census_like"
N_PROBES = 16
EPS_T = 1e-4
L2_FLUSH_BYTES = 512 << 20          # > 129 MB L2: written between timed steps
FP32_FMA_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x 2 x max clock
WORK_FILE = os.path.join(ROOT, "profiles", "census_like_step_work.txt")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "kmv_census_like_traffic.txt")
KMV_SOURCES = ["paper_1501_05427_gb300/csrc/kmv_kernel.cuh",
               "paper_1501_05427_gb300/csrc/kmv_launch.cuh",
               "paper_1501_05427_gb300/csrc/kmv_f32.cu",
               "paper_1501_05427_gb300/csrc/ulisse_internal.cuh"]


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target host time of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--path", choices=["fp32", "mixed"], default="fp32",
                    help="K V path: FP32 SIMT or tensor-core mixed precision")
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


def kmv_source_hash():
    h = hashlib.sha256()
    for f in KMV_SOURCES:
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
def oracle_sample(prob, work, target_s, rng_seed=0):
    """Time the oracle's two O(n^2) kernels on a row sample of the full-size workload:
    K V with 17 right-hand sides (all n columns) and the all-parameter derivative products
    of the gradient, each for m output rows; scale each by n/m and by the per-step work."""
    import numpy as np

    import oracle
    oracle.build()
    n, d = prob.n, prob.d
    Xd = prob.X.astype(np.float64)
    rng = np.random.default_rng(rng_seed)
    R = 1 + N_PROBES
    V = rng.standard_normal((n, R))
    # calibrate on a few hundred rows (threads warm), then size the sample to the target
    cores = oracle.omp_threads()
    oracle.kmv_rows(Xd, prob.psi_true, V, np.arange(cores))
    m0 = 8 * cores
    t0 = time.perf_counter()
    oracle.kmv_rows(Xd, prob.psi_true, V, np.arange(m0))
    t_cal = max(time.perf_counter() - t0, 1e-4)
    m_kv = int(max(m0, min(n, m0 * 0.6 * target_s / t_cal)))
    t0 = time.perf_counter()
    oracle.dkmv_all_rows(Xd, prob.psi_true, V, np.arange(2 * cores))
    t_cal_g = max(time.perf_counter() - t0, 1e-4)
    m_g = int(max(2 * cores, min(n, 2 * cores * 0.4 * target_s / t_cal_g)))
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
    per_step = max(2.0, args.cpu_seconds / max(args.steps, 1))
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
                         "kind": "oracle", "sample": rates[-1]["sample"]},
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }
    print(json.dumps(line))
    return 0


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
    p = d + 2
    prec = u.PREC_MIXED if args.path == "mixed" else u.PREC_FP32
    cfg = u.ulisse_config_default(n_probes=N_PROBES, probe_kind=u.PROBE_RADEMACHER, q=1.0,
                                  beta=1.0, eps=1e-8, max_iter=1000, seed=20150123 + rank,
                                  precision=prec)
    X = torch.from_numpy(prob.X).to(dev)
    y = torch.from_numpy(prob.y).to(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = u.Context(X, y, cfg, stream=stream)
    K, W = args.steps, args.warmup
    psi_dev = torch.tensor(prob.psi_true, dtype=torch.float64, device=dev)
    eps_dev = torch.full((max(K, W, 1),), EPS_T, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for k in range(W):
        ctx.sgld_chain(psi_dev, eps_dev[:1], step0=k)
    ctx.profile_enable(True)
    rounds0, erhs0, launches0 = ctx.counters()
    events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(K)]
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    torch.cuda.synchronize(dev)
    rounds_per_step = []
    for k in range(K):
        flush.zero_()                     # L2 flush, outside the timed spans
        events[k][0].record(stream)
        ctx.sgld_chain(psi_dev, eps_dev[k:k + 1], step0=W + k)
        events[k][1].record(stream)
        rounds_per_step.append(ctx.counters()[0])
    torch.cuda.synchronize(dev)
    rounds_per_step = [b - a for a, b in zip([rounds0] + rounds_per_step[:-1], rounds_per_step)]
    barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in events]
    total_ms = sum(step_ms)
    rounds1, erhs1, launches1 = ctx.counters()
    prof = ctx.profile_read(reset=True)
    ctx.profile_enable(False)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * K / (total_ms / 1000.0)

    # end to end through the host-buffer API: psi in, (psi, g) out every step
    e2e_steps = args.e2e_steps
    psi_h = prob.psi_true.copy()
    ctx.sgld_step(psi_h, EPS_T, step=10_000)          # warm
    barrier()
    torch.cuda.synchronize(dev)
    r_e0 = ctx.counters()[0]
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        psi_h, g_h = ctx.sgld_step(psi_h, EPS_T, step=W + K + 1 + k)
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    e2e_rounds = (ctx.counters()[0] - r_e0) / max(e2e_steps, 1)
    if world > 1:
        t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = world * e2e_steps / e2e_s

    mvp_rounds = (rounds1 - rounds0) / K
    grad_entries = float(n) * n
    mvp_erhs = (erhs1 - erhs0) / K - grad_entries * (1 + N_PROBES)
    kmv_tflops = prof["kmv_flop"] / (prof["kmv_ms"] / 1e3) / 1e12 if prof["kmv_ms"] > 0 else None
    traffic = None
    tf = _kv_file(TRAFFIC_FILE)
    if tf and tf.get("kmv_source_hash") == kmv_source_hash() and prof["kmv_launches"] > 0:
        # captured launch: bytes per launch for R_cap right-hand sides; scale to this run's
        # mean right-hand sides per launch (X^ and V tiles grow with R, X^ does not)
        traffic = float(tf["dram_bytes_per_launch"])
    roofline = {
        "bound": "alu",
        "kernel": ("kmv_tc_kernel (tile-generating K V, tcgen05)" if args.path == "mixed"
                   else "kmv_kernel (tile-generating K V, FP32 SIMT)"),
        "achieved": kmv_tflops,
        "peak": FP32_FMA_PEAK_TFLOPS,
        "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop/FMA x 2070 MHz max SM clock",
        "unit": "TFLOP/s",
        "frac": (kmv_tflops / FP32_FMA_PEAK_TFLOPS) if kmv_tflops else None,
        "traffic": traffic,
        "kmv_launches": prof["kmv_launches"],
        "kmv_ms_per_step": prof["kmv_ms"] / K,
        "grad_ms_per_step": prof["grad_ms"] / K,
        "grad_tflops": (prof["grad_flop"] / (prof["grad_ms"] / 1e3) / 1e12
                        if prof["grad_ms"] > 0 else None),
        "share_of_step": (prof["kmv_ms"] / total_ms) if world == 1 else None,
    }
    line = {
        "metric": "SGLD steps/s", "value": value, "unit": "steps/s", "n_gpus": world,
        "steps": K, "warmup": W, "ms_per_step": total_ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "d": d, "n_probes": N_PROBES, "q": 1.0,
                   "beta": 1.0, "eps_t": EPS_T,
                   "path": ("tcgen05 mixed K V (3xTF32 cross term, 3xBF16 contraction)"
                            if args.path == "mixed" else "fp32 SIMT K V"),
                   "l2": "flushed between timed steps (512 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "kv_throughput": {"value": (mvp_erhs * K) / (prof["kmv_ms"] / 1e3)
                          if prof["kmv_ms"] > 0 else None, "unit": "entry·RHS/s"},
        "mvp_rounds_per_step": mvp_rounds,
        "rounds_per_step": rounds_per_step,
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": "steps/s", "h2d_bytes_per_step": 8 * p,
                "d2h_bytes_per_step": 16 * p, "mvp_rounds_per_step": e2e_rounds,
                "api": "ulisse_sgld_step (host psi in, host psi and g out)"},
        "gpu_launches": int(launches1 - launches0),
        "clocks": clocks,
        "step_ms": step_ms,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        work = {"mvp_entry_rhs": mvp_erhs, "grad_entries": grad_entries,
                "mvp_rounds": mvp_rounds}
        cb = oracle_sample(prob, work, args.cpu_seconds)
        line["cpu_baseline"] = {"value": cb["steps_per_s"], "unit": "steps/s",
                                "cores": cb["cores"], "kind": "oracle", "sample": cb["sample"],
                                "kv_entry_rhs_per_s": cb["kv_entry_rhs_per_s"]}
        line["work_per_step"] = {"mvp_entry_rhs_per_step": mvp_erhs,
                                 "grad_entries_per_step": grad_entries,
                                 "mvp_rounds_per_step": mvp_rounds}
    ctx.close()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
