"""Batched contexts (ulisse_create_batched): many problems of uneven size, the O(n^2) passes of
all of them in one persistent launch.  Each problem is checked against the FP64 oracle with
the generator seed the batch gives it (cfg.seed + b), and against a single context."""
import math
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU runs deselect this module
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1501_05427_gb300 import ulisse as u  # noqa: E402
from paper_1501_05427_gb300 import workloads as w  # noqa: E402


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _batch(probs, **cfg):
    Xs = [torch.from_numpy(p.X).cuda() for p in probs]
    ys = [torch.from_numpy(p.y).cuda() for p in probs]
    return u.BatchContext(Xs, ys, u.ulisse_config_default(**cfg))


def _kv_check(U, ref, scale, tol):
    err = np.abs(U - ref)
    assert np.all(err <= tol * scale + 1e-30), float(np.max(err / (scale + 1e-300)))
    assert np.linalg.norm(U - ref) <= tol * np.linalg.norm(ref)


def _mixed_problems():
    # ragged sizes (one point, under one tile, several 256-row blocks) and widths 1..8
    spec = [(1, 1), (63, 2), (300, 3), (1000, 4), (2500, 8), (777, 5), (129, 8)]
    return [w.random_problem(n, d, seed=2000 + 7 * n + d) for n, d in spec]


@pytest.mark.parametrize("R", [1, 5, 9, 17, 32])
def test_batch_kmv_matches_oracle(orc, R):
    probs = _mixed_problems()
    rng = np.random.default_rng(R)
    Vs = [rng.standard_normal((p.n, R)).astype(np.float32) for p in probs]
    psi = np.concatenate([p.psi_true for p in probs])
    with _batch(probs) as bc:
        Us = bc.kmv(psi, [torch.from_numpy(V).cuda() for V in Vs])
        Us = [U.cpu().numpy().astype(np.float64) for U in Us]
    for p, V, U in zip(probs, Vs, Us):
        Xd, Vd = p.X.astype(np.float64), V.astype(np.float64)
        K = orc.cov_matrix(Xd, p.psi_true)
        _kv_check(U, K @ Vd, np.abs(K) @ np.abs(Vd), 1e-5)


def test_batch_kmv_uneven_workload_sampled_rows(orc):
    """The 64-problem workload (n from 2,000 to 40,000, d in {2, 4, 8}), 9 right-hand sides,
    in the launch configuration of the batched step: sampled rows of every problem against
    the oracle, which evaluates them one by one."""
    probs = w.uneven_batch()
    rng = np.random.default_rng(5)
    Vs = []
    for p in probs:
        V = rng.choice([-1.0, 1.0], (p.n, 9)).astype(np.float32)
        V[:, 0] = p.y
        Vs.append(V)
    psi = np.concatenate([p.psi_true for p in probs])
    with _batch(probs, n_probes=8) as bc:
        Us = bc.kmv(psi, [torch.from_numpy(V).cuda() for V in Vs])
        Us = [U.cpu().numpy() for U in Us]
    for p, V, U in zip(probs, Vs, Us):
        rows = np.sort(rng.choice(p.n, 6, replace=False))
        rows[-1] = p.n - 1
        Xd, Vd = p.X.astype(np.float64), V.astype(np.float64)
        ref = orc.kmv_rows(Xd, p.psi_true, Vd, rows)
        scale = orc.kmv_rows(Xd, p.psi_true, Vd, rows, absolute=True)
        _kv_check(U[rows].astype(np.float64), ref, scale, 1e-5)


def _short_problems():
    # Census-shaped inputs of widths 8, 4 and 2 and uneven sizes
    return [w.census_like(n=900, d=8, seed=3001), w.census_like(n=1700, d=8, seed=3002),
            w.census_like(n=400, d=4, seed=3003), w.census_like(n=1200, d=2, seed=3004)]


def _early_stop_margin(orc, Xd, psi, b, q, iters):
    """Smallest relative distance of ||e_i|| (i = 1..iters) to the threshold q sqrt(n)."""
    tr = orc.cg_record(Xd, psi, b, eps=1e-8, max_iter=max(iters, 1) + 1)
    a = q * math.sqrt(len(b))
    norms = np.linalg.norm(tr["E"], axis=1)[1:iters + 1]
    return float(np.min(np.abs(norms - a) / a)) if len(norms) else 1.0


def test_batch_grad_matches_oracle_per_problem(orc):
    """Census-shaped problems of four sizes in one batch (short trajectories, as in the
    single-context FP32 parity test): each problem's seeded gradient within 1e-4 of the
    oracle's with seed cfg.seed + b; integer outcomes equal unless the oracle's early-stop
    test lies within 1e-4 of alpha."""
    probs = [w.census_like(n=n, d=8, seed=500 + n) for n in (800, 1500, 2000, 2500)]
    nr, seed = 8, 41
    psi = np.concatenate([p.psi_true for p in probs])
    checked = 0
    with _batch(probs, n_probes=nr, max_iter=500, seed=seed) as bc:
        for step in (0, 1):
            g, stats = bc.grad(psi, step=step)
            for b, (p, gb) in enumerate(zip(probs, bc.split(g))):
                Xd, yd = p.X.astype(np.float64), p.y.astype(np.float64)
                gref, st_ref = orc.grad_estimate(Xd, yd, p.psi_true, nr=nr, q=1.0, beta=1.0,
                                                 max_iter=500, seed=seed + b, step=step)
                if any(tuple(stats[b][c][:4]) != tuple(int(v) for v in st_ref[c, :4])
                       for c in range(1 + nr)):
                    B = np.column_stack([yd, orc.probes(p.n, nr, 0, seed + b, step)])
                    margins = [_early_stop_margin(orc, Xd, p.psi_true, B[:, c], 1.0,
                                                  int(st_ref[c, 1])) for c in range(1 + nr)]
                    assert min(margins) < 1e-4, (b, step, stats[b], st_ref)
                    continue
                rel = np.linalg.norm(gb - gref) / np.linalg.norm(gref)
                assert rel <= 1e-4, (b, step, gb, gref, rel)
                checked += 1
    assert checked >= 4


def test_batch_matches_single_contexts(orc):
    """Problem b of a batch and a single context with seed cfg.seed + b take the same
    integer decisions and agree to FP32 rounding (the batch sums the j range in one pass,
    the single context may split it)."""
    probs = _short_problems()
    nr, seed = 8, 7
    psi = np.concatenate([p.psi_true for p in probs])
    with _batch(probs, n_probes=nr, seed=seed) as bc:
        g, stats = bc.grad(psi, step=3)
        psi_new, g2 = bc.sgld_step(psi, 1e-4, step=4)
    for b, p in enumerate(probs):
        X = torch.from_numpy(p.X).cuda()
        y = torch.from_numpy(p.y).cuda()
        with u.Context(X, y, u.ulisse_config_default(n_probes=nr, seed=seed + b)) as ctx:
            gs, st = ctx.grad(p.psi_true, step=3)
            ps, gs2 = ctx.sgld_step(p.psi_true, 1e-4, step=4)
        assert [tuple(s[:4]) for s in st] == [tuple(s[:4]) for s in stats[b]]
        assert np.linalg.norm(bc.split(g)[b] - gs) <= 1e-4 * np.linalg.norm(gs)
        assert np.linalg.norm(bc.split(g2)[b] - gs2) <= 1e-4 * np.linalg.norm(gs2)
        # psi' = psi + eps/2 g + sqrt(eps) xi with the same xi: the difference is eps/2 dg
        assert np.max(np.abs(bc.split(psi_new)[b] - ps)) <= 1e-4 * 0.5e-4 * np.linalg.norm(gs2) + 1e-12


def test_batch_uneven_workload_step_runs(orc):
    """One batched SGLD step of the 64-problem workload: finite results, every problem's
    solves finished, and the work counters account for all problems."""
    probs = w.uneven_batch()
    psi = np.concatenate([p.psi_true for p in probs])
    with _batch(probs, n_probes=8, seed=5) as bc:
        g, stats = bc.grad(psi, step=0)
        rounds, entries, launches = bc.counters()
    assert np.all(np.isfinite(g))
    for st in stats:
        assert all(s[2] == 0 for s in st)               # outcome ok
        assert all(s[1] >= 1 for s in st)
    assert launches > 64
    n2 = sum(float(p.n) ** 2 for p in probs)
    assert entries >= n2 * 9 * 2                        # at least one K V round and the gradient


def test_batch_argument_errors():
    probs = _short_problems()[:2]
    Xs = [torch.from_numpy(p.X).cuda() for p in probs]
    ys = [torch.from_numpy(p.y).cuda() for p in probs]
    with pytest.raises(u.UlisseError):     # FP64 batches are not offered
        u.BatchContext(Xs, ys, u.ulisse_config_default(precision=u.PREC_FP64))
    big = w.random_problem(100, 12, seed=1)
    with pytest.raises(u.UlisseError):
        _batch([probs[0], big])
    with _batch(probs) as bc:
        lib = u.load()
        g = np.zeros(bc.n_params)
        psi = np.concatenate([p.psi_true for p in probs])
        # single-problem calls refuse a batched context
        assert lib.ulisse_grad(bc._h, u._hptr(psi), 0, u._hptr(g), None) == u.ULISSE_ERR_ARG
        bad = psi.copy()
        bad[3] = math.nan
        with pytest.raises(u.UlisseError):
            bc.grad(bad)
        n, p = u.ulisse_batch_size(bc)
        assert (n, p) == (2, bc.n_params)


def test_batch_graph_chain_matches_host_loop():
    """Every batched step as one graph launch (WHILE / SWITCH nodes around the persistent
    launches) reproduces the host loop bit for bit: trace, final parameters, counters."""
    spec = [(2200, 2), (700, 4), (3100, 8), (150, 8), (1800, 4)]
    probs = [w.random_problem(n, d, seed=4000 + n) for n, d in spec]
    psi0 = np.concatenate([p.psi_true for p in probs])
    out = []
    with _batch(probs, n_probes=8, seed=12) as bc:
        for graph in (False, True, True):
            bc.set_graph(graph)
            psi = torch.tensor(psi0, dtype=torch.float64, device="cuda")
            eps = torch.full((4,), 1e-3, dtype=torch.float64, device="cuda")
            tr = torch.zeros((4, bc.n_params), dtype=torch.float64, device="cuda")
            c0 = bc.counters()
            bc.sgld_chain(psi, eps, step0=20, trace_dev=tr)
            c1 = bc.counters()
            out.append((tr.cpu().numpy(), psi.cpu().numpy(),
                        tuple(b - a for a, b in zip(c0, c1))))
        # one step through the host-buffer call equals the chain's first step
        bc.set_graph(True)
        psi_h, g_h = bc.sgld_step(psi0, 1e-3, step=20)
    (tr_h, psi_hl, w_h), (tr_g, psi_g, w_g), (tr_g2, _, w_g2) = out
    assert np.array_equal(tr_g, tr_h) and np.array_equal(psi_g, psi_hl)
    assert np.array_equal(tr_g2, tr_h)
    assert w_g == w_h == w_g2
    assert np.array_equal(psi_h, tr_h[0])


def test_batch_graph_uneven_workload():
    """The 64-problem workload, two batched steps as graph launches: finite parameters,
    the same trace as the host loop."""
    probs = w.uneven_batch()
    psi0 = np.concatenate([p.psi_true for p in probs])
    traces = []
    with _batch(probs, n_probes=8, seed=5) as bc:
        for graph in (True, False):
            bc.set_graph(graph)
            psi = torch.tensor(psi0, dtype=torch.float64, device="cuda")
            eps = torch.full((2,), 1e-4, dtype=torch.float64, device="cuda")
            tr = torch.zeros((2, bc.n_params), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            bc.sgld_chain(psi, eps, step0=0, trace_dev=tr)
            torch.cuda.synchronize()
            print("uneven batch (64 problems), %s: %.1f ms per batched step"
                  % ("graph" if graph else "host loop", 1e3 * (time.perf_counter() - t0) / 2))
            traces.append(tr.cpu().numpy())
    assert np.all(np.isfinite(traces[0]))
    assert np.array_equal(traces[0], traces[1])


def test_batch_warm_solves_graph_and_single_contexts():
    """Warm-started solves in a batch: the graph chain equals the host loop bit for bit, and
    over consecutive gradient steps each problem follows a warm-started single context with
    seed cfg.seed + b (same integer decisions, gradients within FP32 rounding)."""
    spec = [(1800, 8), (900, 4), (2600, 2)]
    probs = [w.census_like(n=n, d=d, seed=5000 + n) for n, d in spec]
    psi0 = np.concatenate([p.psi_true for p in probs])
    cfg = dict(n_probes=8, seed=21, probe_refresh=3, warm_start_probes=1)
    traces = []
    for graph in (False, True):
        # a fresh batch each time: the warm starts carry state from step to step
        with _batch(probs, **cfg) as bc:
            bc.set_graph(graph)
            psi = torch.tensor(psi0, dtype=torch.float64, device="cuda")
            eps = torch.full((5,), 1e-3, dtype=torch.float64, device="cuda")
            tr = torch.zeros((5, bc.n_params), dtype=torch.float64, device="cuda")
            bc.sgld_chain(psi, eps, step0=7, trace_dev=tr)
            traces.append(tr.cpu().numpy())
    assert np.array_equal(traces[0], traces[1])
    with _batch(probs, **cfg) as bc:
        out_b = [bc.grad(psi0, step=s) for s in range(4)]
    for b, p in enumerate(probs):
        X = torch.from_numpy(p.X).cuda()
        y = torch.from_numpy(p.y).cuda()
        c = dict(cfg, seed=cfg["seed"] + b)
        with u.Context(X, y, u.ulisse_config_default(**c)) as ctx:
            out_s = [ctx.grad(p.psi_true, step=s) for s in range(4)]
        for (gb, stb), (gs, sts) in zip(out_b, out_s):
            assert [tuple(s[:4]) for s in sts] == [tuple(s[:4]) for s in stb[b]]
            assert np.linalg.norm(bc.split(gb)[b] - gs) <= 1e-4 * np.linalg.norm(gs)
