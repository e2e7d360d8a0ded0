"""Posterior predictive (Sec. 2, Eq. monte:carlo:integration) through ulisse_predict, against
the oracle's exact predictive (dense Cholesky; pinned in test_oracle_pins.py).

* Converged solves (q = 0): every column runs Algorithm 1 to its threshold, so the result is
  the exact predictive up to that threshold.  FP64: mean within 1e-7 of its scale, variance
  within 1e-7 of sigma^2 + lambda.  FP32 and mixed on a Census-shaped problem: the FP32 CG
  stops at eps = 1e-3 (FP32 vectors cannot take ||e|| much lower), so the solves carry an error
  K^{-1} e, ||e|| < eps; the test states that bound per test input
  (|k*_j| eps / lambda for the mean) and checks each output against it.
* ULISSE solves (q > 0): mean and the k*^T K^{-1} k* term are unbiased; the mean of 2,000
  seeded predictions is within 4 standard errors of the exact values (noise 0.3, q = 0.1, where
  the sample standard error carries the truncation weights' expectation).
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU runs deselect this module
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1501_05427_gb300 import sampler  # noqa: E402
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


def test_predict_fp64_converged(orc):
    prob = w.small_2d(n=500)
    Xs = np.random.default_rng(5).uniform(0, 1, (50, 2)).astype(np.float32)
    mref, vref = orc.predict(prob.X.astype(np.float64), prob.y.astype(np.float64),
                             prob.psi_true, Xs.astype(np.float64))
    with _ctx(prob, precision=u.PREC_FP64, q=0.0, eps=1e-10, max_iter=5000) as ctx:
        m, v = ctx.predict(prob.psi_true, torch.from_numpy(Xs).cuda())
    m, v = m.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    s2l = np.exp(prob.psi_true[-2]) + np.exp(prob.psi_true[-1])
    print("FP64 predictive: mean err %.2e (scale %.2e), var err %.2e"
          % (np.max(np.abs(m - mref)), np.max(np.abs(mref)), np.max(np.abs(v - vref))))
    assert np.max(np.abs(m - mref)) <= 1e-7 * max(1.0, np.max(np.abs(mref)))
    assert np.max(np.abs(v - vref)) <= 1e-7 * s2l


@pytest.mark.parametrize("precision", [u.PREC_FP32, u.PREC_MIXED])
def test_predict_fp32_mixed_converged(orc, precision):
    prob = w.census_like(n=2000, seed=909)
    Xs = np.random.default_rng(6).standard_normal((40, 8)).astype(np.float32)
    Xd = prob.X.astype(np.float64)
    mref, vref = orc.predict(Xd, prob.y.astype(np.float64), prob.psi_true, Xs.astype(np.float64))
    eps = 1e-3
    with _ctx(prob, precision=precision, q=0.0, eps=eps, max_iter=5000) as ctx:
        m, v = ctx.predict(prob.psi_true, torch.from_numpy(Xs).cuda())
    m, v = m.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    lam = np.exp(prob.psi_true[-1])
    kn = np.linalg.norm(orc.cross_signal(Xd, Xs.astype(np.float64), prob.psi_true), axis=0)
    # |k*^T K^{-1} e| <= |k*| |e| / lambda_min(K) <= |k*| eps / lambda, plus FP32 rounding
    bound_m = kn * eps / lam + 1e-4 * np.maximum(1.0, np.abs(mref))
    # the variance's solve K^{-1} k* stops at |e| < eps as well: |k*| eps / lambda again
    bound_v = kn * eps / lam + 1e-4
    print("precision %d: mean err / bound max %.3f, var err / bound max %.3f"
          % (precision, np.max(np.abs(m - mref) / bound_m), np.max(np.abs(v - vref) / bound_v)))
    assert np.all(np.abs(m - mref) <= bound_m)
    assert np.all(np.abs(v - vref) <= bound_v)


def test_predict_ulisse_unbiased(orc):
    prob = w.census_like(n=600, seed=62, noise=0.3)
    Xs = np.random.default_rng(7).standard_normal((6, 8)).astype(np.float32)
    mref, vref = orc.predict(prob.X.astype(np.float64), prob.y.astype(np.float64),
                             prob.psi_true, Xs.astype(np.float64))
    N = 2000
    Xt = torch.from_numpy(Xs).cuda()
    with _ctx(prob, q=0.1, max_iter=600, seed=17) as ctx:
        out = [ctx.predict(prob.psi_true, Xt, step=s) for s in range(N)]
    M = np.array([o[0].cpu().numpy() for o in out], dtype=np.float64)
    V = np.array([o[1].cpu().numpy() for o in out], dtype=np.float64)
    zm = (M.mean(axis=0) - mref) / (M.std(axis=0, ddof=1) / math.sqrt(N))
    zv = (V.mean(axis=0) - vref) / (V.std(axis=0, ddof=1) / math.sqrt(N))
    print("ULISSE predictions: max |z| mean %.2f, var %.2f" % (np.max(np.abs(zm)),
                                                               np.max(np.abs(zv))))
    assert np.max(np.abs(zm)) < 4.0 and np.max(np.abs(zv)) < 4.0


def test_posterior_predictive_mixture(orc):
    """Eq. monte:carlo:integration end to end: the mixture over posterior samples of the
    library's predictives equals the mixture of the oracle's exact predictives (q = 0)."""
    prob = w.small_2d(n=300)
    rng = np.random.default_rng(8)
    psis = prob.psi_true + 0.05 * rng.standard_normal((5, 4))
    Xs = rng.uniform(0, 1, (10, 2)).astype(np.float32)
    with _ctx(prob, precision=u.PREC_FP64, q=0.0, eps=1e-10, max_iter=5000) as ctx:
        M, V = sampler.posterior_predictive(ctx, psis, torch.from_numpy(Xs).cuda())
    ref = [orc.predict(prob.X.astype(np.float64), prob.y.astype(np.float64), p,
                       Xs.astype(np.float64)) for p in psis]
    Mr = np.array([r[0] for r in ref])
    Vr = np.array([r[1] for r in ref])
    mu, var = sampler.mixture_moments(M, V)
    mur, varr = sampler.mixture_moments(Mr, Vr)
    assert np.max(np.abs(mu - mur)) < 1e-6 and np.max(np.abs(var - varr)) < 1e-6
    ys = mur + 0.3
    assert np.allclose(sampler.mixture_density(ys, M, V), sampler.mixture_density(ys, Mr, Vr),
                       rtol=1e-5)
