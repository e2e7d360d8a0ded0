"""SGLD run control (Sec. 2.1 and the choices of Sec. 5.1) driving the library on the GPU:
sampler.run_sgld with the decreasing step size eps_t = a (b + t)^-1 from 1e-1 to 1e-4, the
Langevin-phase monitor on batches of 100 gradients with the step-size freeze at 0.002, and
the preconditioner M from the log-posterior mode of a 500-point subset, every step one
ulisse_sgld_step through a real context.

Checks: the freeze happens at the end of the first batch whose ratio eps_t/4 lambda_max(M^1/2
V M^1/2), recomputed here from the recorded gradients, is below 0.002, and every later step
uses the frozen step size; after the freeze the chain's step-to-step covariance has M's shape
(the injected noise N(0, eps M) dominates the move in the Langevin phase).

The workload is the 2-D one (the Concrete-sized stand-in, n = 1,000, FP64 products as in the
paper's Concrete run).  The early-stop threshold is alpha = 0.03 sqrt(n): at the paper's
alpha = sqrt(n) the truncation noise of these inputs keeps the ratio above 0.002 down to
eps ~ 1e-5, past the end of a 1e-1 -> 1e-4 schedule (the chain test in
test_gpu_chain_validation.py measures it).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU runs deselect this module
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1501_05427_gb300 import sampler  # noqa: E402
from paper_1501_05427_gb300 import ulisse as u  # noqa: E402
from paper_1501_05427_gb300 import workloads as w  # noqa: E402


def test_run_sgld_freezes_where_the_ratio_says_and_moves_with_M():
    prob = w.small_2d(n=1000)
    M, mode = sampler.preconditioner_from_subset(prob.X, prob.y, prob.psi_true, m=500, seed=3)
    X = torch.from_numpy(prob.X).cuda()
    y = torch.from_numpy(prob.y).cuda()
    cfg = u.ulisse_config_default(precision=u.PREC_FP64, n_probes=4, q=0.03, beta=1.0,
                                  max_iter=3000, seed=11)
    rec = []
    n_steps = 1500
    with u.Context(X, y, cfg) as ctx:
        trace, mon = sampler.run_sgld(ctx, mode, n_steps, eps_first=1e-1, eps_last=1e-4, M=M,
                                      batch=100, threshold=0.002, record=rec)
    eps = np.array([r[1] for r in rec])
    G = np.array([r[2] for r in rec])
    assert np.all(np.isfinite(trace)) and np.all(np.isfinite(G))
    # the ratios of the completed batches, recomputed from the recorded gradients
    expect_freeze = None
    for k, (step, ratio) in enumerate(mon.ratios):
        lo = step - 99
        V = np.cov(G[lo:step + 1], rowvar=False, ddof=1)
        r = sampler.noise_ratio(eps[step], M, V)
        assert abs(r - ratio) <= 1e-12 * max(1.0, r)
        if expect_freeze is None and r < 0.002:
            expect_freeze = step
    print("batch ratios %s; frozen at step %s with eps %s"
          % (["%.2g" % r for _, r in mon.ratios], mon.frozen_at, mon.frozen_eps))
    assert expect_freeze is not None and mon.frozen_at == expect_freeze
    assert np.all(eps[mon.frozen_at + 1:] == mon.frozen_eps)
    assert np.all(eps[:mon.frozen_at + 1] >= mon.frozen_eps)
    # after the freeze: Cov(psi_{t+1} - psi_t) ~ eps M (the drift term is (eps/2) M g~, whose
    # share is the ratio above); compare the whitened covariance with the identity
    D = np.diff(trace[mon.frozen_at + 1:], axis=0)
    C = np.cov(D, rowvar=False, ddof=1) / mon.frozen_eps
    L = np.linalg.cholesky(M)
    Li = np.linalg.inv(L)
    ev = np.linalg.eigvalsh(Li @ C @ Li.T)
    m = len(D)
    print("whitened step covariance eigenvalues %s over %d steps" % (np.round(ev, 3), m))
    # sampling spread of the eigenvalues of a p x p Wishart(m) / m: about 2 sqrt(p / m)
    assert ev.min() > 1 - 4 * np.sqrt(4 / m) and ev.max() < 1 + 4 * np.sqrt(4 / m)
