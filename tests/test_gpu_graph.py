"""One SGLD step as a CUDA graph (ulisse_set_graph / ulisse_sgld_chain): the graph holds the
data-dependent CG loop as conditional nodes and launches exactly the host loop's kernels, so a
chain run from the graph must reproduce the host-loop chain bit for bit -- trace, final psi
and work counters -- in every precision, with the learned warm start on, after a call that
reallocated the context's buffers, and when a solve runs into max_iter."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU runs deselect this module
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1501_05427_gb300 import ulisse as u  # noqa: E402
from paper_1501_05427_gb300 import workloads as w  # noqa: E402


def _ctx(prob, **cfg):
    X = torch.from_numpy(prob.X).cuda()
    y = torch.from_numpy(prob.y).cuda()
    return u.Context(X, y, u.ulisse_config_default(**cfg))


def _chain(ctx, psi0, eps, step0, graph, allow=()):
    ctx.set_graph(graph)
    psi_dev = torch.tensor(psi0, dtype=torch.float64, device="cuda")
    eps_dev = torch.tensor(eps, dtype=torch.float64, device="cuda")
    trace = torch.zeros((len(eps), len(psi0)), dtype=torch.float64, device="cuda")
    c0 = ctx.counters()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.sgld_chain(psi_dev, eps_dev, step0=step0, trace_dev=trace, allow=allow)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    c1 = ctx.counters()
    work = tuple(b - a for a, b in zip(c0, c1))
    return trace.cpu().numpy(), psi_dev.cpu().numpy(), work, dt


@pytest.mark.parametrize("precision,prob_fn,nr,kind", [
    (u.PREC_FP32, lambda: w.census_like(n=3000, seed=7001), 8, 0),
    (u.PREC_MIXED, lambda: w.census_like(n=3000, seed=7002), 16, 0),
    (u.PREC_FP64, lambda: w.small_2d(n=1000), 4, 1),
])
def test_graph_chain_matches_host_loop(precision, prob_fn, nr, kind):
    prob = prob_fn()
    eps = [2e-3] * 6
    with _ctx(prob, precision=precision, n_probes=nr, probe_kind=kind, seed=3) as ctx:
        tr_h, psi_h, work_h, dt_h = _chain(ctx, prob.psi_true, eps, 40, graph=False)
        tr_g, psi_g, work_g, dt_g = _chain(ctx, prob.psi_true, eps, 40, graph=True)
        tr_g2, psi_g2, work_g2, dt_g2 = _chain(ctx, prob.psi_true, eps, 40, graph=True)
    print("%s n=%d: host loop %.2f ms/step, graph %.2f ms/step (first launch incl. capture "
          "%.2f ms/step); rounds %d" % (prob.name, prob.n, 1e3 * dt_h / len(eps),
                                        1e3 * dt_g2 / len(eps), 1e3 * dt_g / len(eps), work_h[0]))
    assert np.array_equal(tr_g, tr_h)
    assert np.array_equal(psi_g, psi_h)
    assert np.array_equal(tr_g2, tr_h)
    assert work_g[0] == work_h[0] and work_g[1] == work_h[1]
    assert work_g[2] == work_h[2]
    assert work_g2 == work_g


def test_graph_chain_with_warm_start():
    prob = w.census_like(n=2500, seed=7003)
    with _ctx(prob, n_probes=4, seed=5) as ctx:
        ctx.ws_init(n_anchors=96, hidden=32, n_rows=128, max_pairs=32, seed=2)
        ctx.ws_set(record=True)
        rng = np.random.default_rng(1)
        for k in range(16):
            ctx.grad((prob.psi_true + 0.05 * rng.standard_normal(prob.d + 2)), step=k)
        ctx.ws_train(steps=0, batch=8)
        ctx.ws_set(record=False, use=True)
        eps = [1e-3] * 4
        tr_h, psi_h, work_h, _ = _chain(ctx, prob.psi_true, eps, 100, graph=False)
        tr_g, psi_g, work_g, _ = _chain(ctx, prob.psi_true, eps, 100, graph=True)
    assert np.array_equal(tr_g, tr_h)
    assert work_g == work_h


def test_graph_rebuilt_after_reallocation():
    """A solve with more columns reallocates the vectors; the next chain captures again."""
    prob = w.census_like(n=1800, seed=7004)
    eps = [1e-3] * 3
    with _ctx(prob, n_probes=4, seed=6) as ctx:
        tr1, _, _, _ = _chain(ctx, prob.psi_true, eps, 0, graph=True)
        B = torch.randn((prob.n, 40), device="cuda")
        ctx.solve(prob.psi_true, B, step=1)
        tr2, _, _, _ = _chain(ctx, prob.psi_true, eps, 0, graph=True)
        tr3, _, _, _ = _chain(ctx, prob.psi_true, eps, 0, graph=False)
    assert np.array_equal(tr1, tr2)
    assert np.array_equal(tr2, tr3)


def test_graph_chain_reports_max_iter():
    """q = 0 (no early stop) and max_iter = 3: every solve is cut off; the graph path reports
    ULISSE_ERR_MAXITER like the host loop and gives the same trace."""
    prob = w.census_like(n=1500, seed=7005)
    eps = [1e-3] * 2
    allow = (u.ULISSE_ERR_MAXITER,)
    with _ctx(prob, n_probes=4, q=0.0, max_iter=3, seed=8) as ctx:
        tr_h, _, work_h, _ = _chain(ctx, prob.psi_true, eps, 0, graph=False, allow=allow)
        tr_g, _, work_g, _ = _chain(ctx, prob.psi_true, eps, 0, graph=True, allow=allow)
        ctx.set_graph(True)
        psi_dev = torch.tensor(prob.psi_true, dtype=torch.float64, device="cuda")
        with pytest.raises(u.UlisseError) as ei:
            ctx.sgld_chain(psi_dev, torch.tensor(eps, dtype=torch.float64, device="cuda"))
        assert ei.value.args[0].startswith("ulisse status %d" % u.ULISSE_ERR_MAXITER)
    assert np.array_equal(tr_g, tr_h)
    assert work_g == work_h
