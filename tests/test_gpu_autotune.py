"""Autotuner of the K V launch configuration (ulisse_autotune): the chosen configuration
is never slower than the untuned one, the tuned products keep their parity with the FP64
oracle, and a step graph captured after tuning still reproduces the host loop."""
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


def _ctx(prob, **cfg):
    X = torch.from_numpy(prob.X).cuda()
    y = torch.from_numpy(prob.y).cuda()
    return u.Context(X, y, u.ulisse_config_default(**cfg))


@pytest.mark.parametrize("precision,tol", [(u.PREC_FP32, 1e-5), (u.PREC_MIXED, 1e-4)])
def test_autotune_table_and_parity(orc, precision, tol):
    prob = w.census_like(n=20_000, seed=8101)
    n = prob.n
    rng = np.random.default_rng(4)
    Xd = prob.X.astype(np.float64)
    rows = np.sort(rng.choice(n, 24, replace=False))
    rows[-1] = n - 1
    with _ctx(prob, precision=precision, n_probes=16) as ctx:
        table = ctx.autotune(prob.psi_true, 17, reps=3)
        for e in table:
            print("tune %s nl=%2d width=%2d tm=%d split=%2d  %.3f ms (untuned %.3f ms)"
                  % ("fp32" if precision == u.PREC_FP32 else "mixed", e["live_cols"],
                     e["width"], e["rows_per_thread"], e["nsplit"], e["ms"], e["ms_default"]))
            assert 0 < e["ms"] <= e["ms_default"]
        for R in (1, 5, 16, 17):
            V = rng.standard_normal((n, R)).astype(np.float32)
            U = ctx.kmv(prob.psi_true, torch.from_numpy(V).cuda()).cpu().numpy()[rows]
            ref = orc.kmv_rows(Xd, prob.psi_true, V.astype(np.float64), rows)
            scale = orc.kmv_rows(Xd, prob.psi_true, V.astype(np.float64), rows, absolute=True)
            err = np.abs(U - ref)
            assert np.all(err <= tol * scale), float(np.max(err / scale))


def test_graph_after_tuning_matches_host_loop():
    prob = w.census_like(n=6000, seed=8102)
    eps = torch.full((4,), 1e-3, dtype=torch.float64, device="cuda")
    traces = []
    with _ctx(prob, n_probes=16, seed=4) as ctx:
        ctx.autotune(prob.psi_true, 17, reps=2)
        for graph in (False, True):
            ctx.set_graph(graph)
            psi = torch.tensor(prob.psi_true, dtype=torch.float64, device="cuda")
            tr = torch.zeros((4, prob.d + 2), dtype=torch.float64, device="cuda")
            ctx.sgld_chain(psi, eps, step0=3, trace_dev=tr)
            traces.append(tr.cpu().numpy())
    assert np.array_equal(traces[0], traces[1])
