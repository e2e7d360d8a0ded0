"""Degenerate and extreme solves through ulisse_solve, against the FP64 oracle (seeded, the
same Philox streams): a zero right-hand side among others (Algorithm 1 starts converged:
l = 0, no iteration, the estimate is s_0 = 0, and its neighbours are unaffected), a
one-point problem (K is the scalar sigma^2 + lambda), and 1,000 right-hand sides in one call
(more than the K V launches' column chunks of 32 and 64, and than the oracle's block of
512 accumulators).  Integer outcomes must equal the
oracle's; estimates within the path's solve tolerance (FP32 and mixed 1e-4, FP64 1e-6) on
these short-trajectory inputs."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU runs deselect this module
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1501_05427_gb300 import ulisse as u  # noqa: E402
from paper_1501_05427_gb300 import workloads as w  # noqa: E402

PRECS = [(u.PREC_FP32, 1e-4), (u.PREC_MIXED, 1e-4), (u.PREC_FP64, 1e-6)]


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _solve_both(orc, prob, B, n_est, precision, seed=3, step=0, eps=1e-8):
    Sref, st_ref = orc.ulisse_solve(prob.X.astype(np.float64), prob.psi_true,
                                    B.astype(np.float64), n_est=n_est, q=1.0, beta=1.0,
                                    eps=eps, max_iter=500, seed=seed, step=step)
    X = torch.from_numpy(prob.X).cuda()
    y = torch.from_numpy(prob.y).cuda()
    cfg = u.ulisse_config_default(precision=precision, q=1.0, eps=eps, max_iter=500, seed=seed)
    with u.Context(X, y, cfg) as ctx:
        S, st = ctx.solve(prob.psi_true, torch.from_numpy(B.astype(np.float32)).cuda(),
                          n_est=n_est, step=step)
    return S.cpu().numpy().astype(np.float64), st, Sref, st_ref


def _rel_cols(S, Sref):
    out = []
    for k in range(Sref.shape[1]):
        nr = np.linalg.norm(Sref[:, k])
        out.append(np.linalg.norm(S[:, k] - Sref[:, k]) / nr if nr > 0 else
                   float(np.max(np.abs(S[:, k]))))
    return np.array(out)


@pytest.mark.parametrize("precision,tol", PRECS)
def test_zero_right_hand_side(orc, precision, tol):
    prob = w.census_like(n=700, seed=1000)
    B = np.random.default_rng(1).choice([-1.0, 1.0], (prob.n, 3)).astype(np.float32)
    B[:, 0] = prob.y
    B[:, 1] = 0.0
    n_est = np.array([2, 1, 1], dtype=np.int32)
    S, st, Sref, st_ref = _solve_both(orc, prob, B, n_est, precision)
    assert [tuple(s[:4]) for s in st] == [tuple(int(v) for v in r[:4]) for r in st_ref]
    assert tuple(st[1][:3]) == (0, 0, u.ULISSE_OK)
    assert np.all(S[:, 2] == 0.0)          # the zero column's estimate (estimator offset 2)
    assert np.all(_rel_cols(S, Sref) <= tol)


@pytest.mark.parametrize("precision,tol", PRECS)
def test_one_point_problem(orc, precision, tol):
    """CG solves a 1 x 1 system exactly in one step; the convergence threshold is one that
    the precision can reach after it (FP32 vectors leave a residual of ~1e-7 |b|, above the
    paper's absolute 1e-8), so the integer outcomes are comparable."""
    prob = w.random_problem(1, 2, seed=5)
    B = np.array([[prob.y[0], 1.0, -1.0]], dtype=np.float32)
    n_est = np.array([2, 1, 1], dtype=np.int32)
    eps = 1e-8 if precision == u.PREC_FP64 else 1e-5
    S, st, Sref, st_ref = _solve_both(orc, prob, B, n_est, precision, eps=eps)
    assert [tuple(s[:4]) for s in st] == [tuple(int(v) for v in r[:4]) for r in st_ref]
    assert np.all(_rel_cols(S, Sref) <= tol)


@pytest.mark.parametrize("precision,tol", PRECS)
def test_thousand_right_hand_sides(orc, precision, tol):
    prob = w.census_like(n=400, seed=1100, noise=0.3)
    R = 1000
    B = np.random.default_rng(2).choice([-1.0, 1.0], (prob.n, R)).astype(np.float32)
    B[:, 0] = prob.y
    n_est = np.ones(R, dtype=np.int32)
    n_est[0] = 2
    S, st, Sref, st_ref = _solve_both(orc, prob, B, n_est, precision)
    same = [tuple(s[:4]) == tuple(int(v) for v in r[:4]) for s, r in zip(st, st_ref)]
    print("1,000 right-hand sides, precision %d: %d of %d columns with equal integer outcomes, "
          "worst estimate error %.2e" % (precision, sum(same), R, _rel_cols(S, Sref).max()))
    assert all(same)
    assert np.all(_rel_cols(S, Sref) <= tol)
