"""Host-side SGLD control (paper_1501_05427_gb300/sampler.py, Sec. 2.1 and Sec. 5.1): the
step-size schedule, the Langevin-phase noise ratio and freeze, and the preconditioner from a
subset.  The FP64 likelihood code there is an implementation of its own; the oracle's
independent one pins it."""
import math

import numpy as np
import pytest

from paper_1501_05427_gb300 import sampler as S


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def test_step_size_schedule_endpoints():
    a, b = S.step_size_schedule(1e-1, 1e-4, 40_000)
    assert math.isclose(S.step_size(a, b, 0), 1e-1, rel_tol=1e-12)
    assert math.isclose(S.step_size(a, b, 39_999), 1e-4, rel_tol=1e-12)
    e = [S.step_size(a, b, t) for t in (0, 10, 1000, 39_999)]
    assert all(x > y for x, y in zip(e, e[1:]))
    with pytest.raises(ValueError):
        S.step_size_schedule(1e-4, 1e-1, 100)


def test_noise_ratio_is_the_definition():
    """eps/4 lambda_max(M^(1/2) V M^(1/2)) with the symmetric square root from scipy."""
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(1)
    for p in (2, 5, 10):
        A = rng.standard_normal((p, p))
        M = A @ A.T + p * np.eye(p)
        B = rng.standard_normal((p, p))
        V = B @ B.T
        Mh = np.real(scipy_linalg.sqrtm(M))
        want = 0.25 * 3e-3 * np.linalg.eigvalsh(Mh @ V @ Mh)[-1]
        assert math.isclose(S.noise_ratio(3e-3, M, V), want, rel_tol=1e-9)


def test_monitor_estimates_the_ratio_and_freezes():
    rng = np.random.default_rng(2)
    p = 4
    M = np.diag([1.0, 2.0, 0.5, 1.5])
    V0 = np.diag([4.0, 1.0, 9.0, 2.0])
    exact = lambda eps: S.noise_ratio(eps, M, V0)
    mon = S.LangevinMonitor(M, batch=4000, threshold=0.002)
    # a batch at a large step size: ratio above the threshold, no freeze
    eps1 = 4e-3
    for k in range(4000):
        r = mon.update(k, eps1, rng.multivariate_normal(np.zeros(p), V0))
        assert r is None
    assert mon.frozen_at is None and mon.ratios
    assert abs(mon.ratios[-1][1] / exact(eps1) - 1.0) < 0.1
    # a batch at a small one: ratio below the threshold, frozen at its last step
    eps2 = 2e-4
    out = None
    for k in range(4000, 8000):
        out = mon.update(k, eps2, rng.multivariate_normal(np.zeros(p), V0))
    assert exact(eps2) < 0.002
    assert mon.frozen_at == 7999 and out == eps2
    assert mon.update(8000, 1e-9, np.zeros(p)) == eps2     # stays frozen


def test_host_likelihood_matches_the_oracle(orc):
    rng = np.random.default_rng(3)
    X = rng.uniform(0, 1, (80, 3))
    y = rng.standard_normal(80)
    psi = np.log([0.4, 0.6, 0.9, 1.2, 0.2])
    assert math.isclose(S.log_marginal_likelihood(X, y, psi),
                        orc.log_marginal_likelihood(X, y, psi), rel_tol=1e-10)
    g = S.lml_gradient(X, y, psi)
    assert np.allclose(g, orc.exact_gradient(X, y, psi), rtol=1e-8, atol=1e-10)


def test_hessian_mode_and_preconditioner(orc):
    rng = np.random.default_rng(4)
    n = 120
    X = rng.uniform(0, 1, (n, 2))
    truth = np.log([0.3, 0.5, 1.0, 0.1])
    K = orc.cov_matrix(X, truth)
    y = np.linalg.cholesky(K) @ rng.standard_normal(n)
    psi = np.log([0.5, 0.5, 0.8, 0.2])
    # Hessian vs second differences of the oracle's likelihood
    H = S.lml_hessian(X, y, psi)
    h = 1e-3
    i, j = 0, 3
    e_i, e_j = np.eye(4)[i] * h, np.eye(4)[j] * h
    f = lambda q: orc.log_marginal_likelihood(X, y, q)
    fd = (f(psi + e_i + e_j) - f(psi + e_i - e_j) - f(psi - e_i + e_j) + f(psi - e_i - e_j)) / (4 * h * h)
    assert math.isclose(H[i, j], fd, rel_tol=1e-3, abs_tol=1e-3)
    # the mode: zero gradient (oracle's) and a higher likelihood than the start
    mode = S.posterior_mode(X, y, psi)
    assert np.max(np.abs(orc.exact_gradient(X, y, mode))) < 1e-5 * max(1.0, abs(f(mode)))
    assert f(mode) > f(psi)
    # M = (-H)^-1 at the mode of the (here: whole) subset, symmetric positive definite
    M, mode2 = S.preconditioner_from_subset(X, y, psi, m=n)
    assert np.allclose(mode2, mode, atol=1e-6)
    assert np.allclose(M @ (-S.lml_hessian(X, y, mode2)), np.eye(4), atol=1e-6)
    assert np.all(np.linalg.eigvalsh(M) > 0)


class _FakeContext:
    """sgld_step of a Gaussian target N(0, I) with a noisy gradient (variance s2 per
    coordinate): records the step sizes it is given."""

    def __init__(self, s2, seed=0):
        self.s2 = s2
        self.rng = np.random.default_rng(seed)
        self.eps = []

    def sgld_step(self, psi, eps, step, M=None, prior_grad=None):
        self.eps.append(eps)
        g = -psi + math.sqrt(self.s2) * self.rng.standard_normal(len(psi))
        return psi + 0.5 * eps * g + math.sqrt(eps) * self.rng.standard_normal(len(psi)), g


def test_run_sgld_freezes_the_step_size():
    ctx = _FakeContext(s2=5.0)
    trace, mon = S.run_sgld(ctx, np.ones(3), n_steps=3000, eps_first=1e-1, eps_last=1e-4,
                            batch=100, threshold=0.002)
    assert trace.shape == (3000, 3) and np.all(np.isfinite(trace))
    assert mon.frozen_at is not None
    t0 = mon.frozen_at
    # the schedule until the freeze, the frozen value after it
    a, b = S.step_size_schedule(1e-1, 1e-4, 3000)
    assert all(math.isclose(ctx.eps[t], S.step_size(a, b, t)) for t in range(t0 + 1))
    assert all(e == ctx.eps[t0] for e in ctx.eps[t0 + 1:])
    # frozen where eps/4 * s2 (the exact ratio here) first drops below 0.002, within the
    # batch's sampling error
    assert ctx.eps[t0] / 4 * 5.0 < 0.002 * 1.5


def test_mixture_moments_and_density():
    """The equal-weight mixture of Gaussians: its moments by the law of total variance agree
    with a large sample drawn from the mixture, and its density integrates to one and equals
    scipy's normal pdf averaged by hand."""
    from scipy.stats import norm
    from paper_1501_05427_gb300 import sampler
    rng = np.random.default_rng(4)
    means = rng.standard_normal((7, 3))
    varis = rng.uniform(0.1, 2.0, (7, 3))
    mu, v = sampler.mixture_moments(means, varis)
    k = rng.integers(0, 7, 400_000)
    draws = means[k] + np.sqrt(varis[k]) * rng.standard_normal((400_000, 3))
    assert np.all(np.abs(draws.mean(axis=0) - mu) < 5 * np.sqrt(v / 400_000))
    assert np.all(np.abs(draws.var(axis=0) / v - 1) < 0.02)
    ys = np.array([0.3, -1.0, 2.0])
    ref = np.mean([norm.pdf(ys, means[i], np.sqrt(varis[i])) for i in range(7)], axis=0)
    assert np.allclose(sampler.mixture_density(ys, means, varis), ref, rtol=1e-12)
    grid = np.linspace(-15, 15, 60001)
    dens = np.array([sampler.mixture_density(np.full(3, g), means, varis) for g in grid])
    assert np.allclose(np.trapezoid(dens, grid, axis=0), 1.0, atol=1e-6)


def test_posterior_predictive_calls_predict_per_sample():
    from paper_1501_05427_gb300 import sampler

    class FakeTensor:
        def __init__(self, a):
            self.a = a

        def cpu(self):
            return self

        def numpy(self):
            return self.a

    class FakeCtx:
        def __init__(self):
            self.calls = []

        def predict(self, psi, Xs, step=0, var=True):
            self.calls.append((psi.copy(), step))
            return FakeTensor(np.full(2, psi[0])), FakeTensor(np.full(2, 1.0 + step)) if var else None

    ctx = FakeCtx()
    psis = np.array([[0.5, 0.0], [1.5, 0.0]])
    m, v = sampler.posterior_predictive(ctx, psis, None, step0=10)
    assert [c[1] for c in ctx.calls] == [10, 11]
    assert np.allclose(m, [[0.5, 0.5], [1.5, 1.5]]) and np.allclose(v, [[11, 11], [12, 12]])
