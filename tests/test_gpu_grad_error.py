"""Gradient error of the chosen path against the plain FP32 path, by the paper's measure
(Sec. 5: the mean over repetitions of ||g - g~||^2 / ||g||^2, g the exact gradient), on a
Census-shaped problem small enough for the oracle's Cholesky (n = 4,000, d = 8, 16 probes).
The parameters are the generating ones shifted by +0.3 in every log coordinate (at the
generating parameters the exact gradient is close to zero and the ratio is meaningless).
Both paths run the same seeds -- the same probes and the same truncation draws -- so they
differ only by their arithmetic; the learned warm start is measured on the mixed path too
(reported, not bounded: its unbiasedness is tested in test_gpu_warm_start.py).  bench.py
measures the same statistic in its run (key gradient_error)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU runs deselect this module
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1501_05427_gb300 import ulisse as u  # noqa: E402
from paper_1501_05427_gb300 import workloads as w  # noqa: E402

REPS = 100


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _errors(prob, psi, g_exact, precision, warm_start=False):
    X = torch.from_numpy(prob.X).cuda()
    y = torch.from_numpy(prob.y).cuda()
    cfg = u.ulisse_config_default(n_probes=16, precision=precision, seed=77)
    errs, rounds = [], []
    with u.Context(X, y, cfg) as ctx:
        if warm_start:
            ctx.ws_init(n_anchors=512, hidden=256, n_rows=1024, max_pairs=64, seed=3)
            ctx.ws_set(record=True)
            rng = np.random.default_rng(9)
            for k in range(40):
                ctx.grad(psi + 0.05 * rng.standard_normal(prob.d + 2), step=10_000 + k)
            ctx.ws_train(steps=0, batch=8)
            ctx.ws_set(record=False, use=True)
        for s in range(REPS):
            r0 = ctx.counters()[0]
            g, _ = ctx.grad(psi, step=s)
            rounds.append(ctx.counters()[0] - r0)
            errs.append(np.sum((g - g_exact) ** 2) / np.sum(g_exact ** 2))
    return np.array(errs), np.array(rounds)


def test_mixed_path_has_the_plain_gradient_error(orc):
    prob = w.census_like(n=4000, seed=20150124)
    psi = prob.psi_true + 0.3
    g_exact = orc.exact_gradient(prob.X.astype(np.float64), prob.y.astype(np.float64), psi)
    e32, r32 = _errors(prob, psi, g_exact, u.PREC_FP32)
    emx, rmx = _errors(prob, psi, g_exact, u.PREC_MIXED)
    ews, rws = _errors(prob, psi, g_exact, u.PREC_MIXED, warm_start=True)
    def se(e):
        return e.std(ddof=1) / np.sqrt(len(e))
    print("\ngradient error ||g - g~||^2 / ||g||^2 over %d seeded repetitions "
          "(census_like n=4000, d=8, 16 probes, q=1, beta=1, psi = truth + 0.3; "
          "||g|| = %.4g):" % (REPS, np.linalg.norm(g_exact)))
    for name, e, r in (("plain_fp32", e32, r32), ("mixed", emx, rmx),
                       ("mixed_warm_start", ews, rws)):
        print("  %-17s mean %.4e  se %.2e  median %.4e  p90 %.4e  K V rounds/step %.2f"
              % (name, e.mean(), se(e), np.median(e), np.percentile(e, 90), r.mean()))
    # The truncation weights make the error heavy-tailed (a single repetition can hold most
    # of the mean), and past ~15 CG iterations the two arithmetics follow different
    # trajectories, so they are compared by median and 90th percentile.
    assert np.median(emx) <= 1.25 * np.median(e32)
    assert np.percentile(emx, 90) <= 1.5 * np.percentile(e32, 90)
    assert np.all(np.isfinite(ews))
