"""Preconditioned CG with J = K + delta I (Sec. 3) and ULISSE on its outer iteration (Sec. 4),
through the C ABI (ulisse_config.pcg_delta > 0), against the oracle's oracle/pcg.py.

Seeded parity: the GPU and the oracle draw the same J's (same counter-based streams as plain
CG), so the outer early-stop iteration l, the outer iteration count, J and the total count of
K V products (outer and inner) must agree, and the estimates agree up to the trajectory's
drift under the arithmetic:
  * FP64 path on ill-conditioned 2-D inputs, with inner solves of at most ~10 iterations:
    1e-6 (float output buffer), as plain CG.  A longer inner solve on these inputs separates
    two FP64 evaluations (different summation orders) geometrically, as plain CG does past
    ~15 iterations, and its truncated result z feeds the outer direction directly: with
    delta = 0.05 and 0.2 (20-30 inner iterations) the estimates differed by 1.5e-5 and
    1e-4, so those regimes are checked through the converged solve instead;
  * FP32 and mixed paths: the inner CG is held to a few iterations (inner_max; the relative
    tolerance set below what they reach), so that every preconditioner solve has the same
    length on both sides and the chain of products stays short; 1e-4 as for plain CG.
Where an integer outcome differs, the oracle's own decision must lie within rounding of its
threshold (the outer early-stop test within 1e-4 of alpha), as in the plain-CG tests.
Long trajectories are checked by what is unique: a converged PCG solve (q = 0) is the
Cholesky solution, and the mean of seeded PCG gradients is the exact gradient within 4 SE.
"""
import math

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


def _margin(Xd, psi, b, delta, tau, inner_max, q, iters):
    from oracle import pcg
    tr = pcg.pcg_record(Xd, psi, b, delta, tau, inner_max, eps=1e-8, max_iter=max(iters, 1) + 1)
    a = q * math.sqrt(len(b))
    norms = np.linalg.norm(tr["E"], axis=1)[1:iters + 1]
    return float(np.min(np.abs(norms - a) / a)) if len(norms) else 1.0


def _case(orc, prob, R, precision, delta, tau, inner_max, q, tol, seed=21, step=4):
    from oracle import pcg
    n = prob.n
    rng = np.random.default_rng(n + R)
    B = rng.choice([-1.0, 1.0], (n, R)).astype(np.float32)
    B[:, 0] = prob.y
    n_est = np.ones(R, np.int32)
    n_est[0] = 2
    Xd, Bd = prob.X.astype(np.float64), B.astype(np.float64)
    Sref, st_ref, rounds_ref = pcg.ulisse_pcg_solve(Xd, prob.psi_true, Bd, delta, tau, inner_max,
                                                    n_est=n_est, q=q, beta=1.0, eps=1e-8,
                                                    max_iter=500, seed=seed, step=step)
    with _ctx(prob, precision=precision, q=q, max_iter=500, seed=seed, pcg_delta=delta,
              pcg_inner_tol=tau, pcg_inner_max=inner_max) as ctx:
        r0 = ctx.counters()[0]
        Sg, st = ctx.solve(prob.psi_true, torch.from_numpy(B).cuda(), n_est=n_est, step=step)
        rounds = ctx.counters()[0] - r0
    Sg = Sg.cpu().numpy().astype(np.float64)
    col, checked, errs = 0, 0, []
    flips = False
    for c in range(R):
        if tuple(st[c][:4]) != tuple(int(v) for v in st_ref[c, :4]):
            m = _margin(Xd, prob.psi_true, Bd[:, c], delta, tau, inner_max, q, int(st_ref[c, 1]))
            assert m < 1e-4, (c, st[c], st_ref[c], m)
            flips = True
            col += n_est[c]
            continue
        for t in range(n_est[c]):
            ref = Sref[:, col + t]
            errs.append(np.linalg.norm(Sg[:, col + t] - ref) / np.linalg.norm(ref))
        checked += 1
        col += n_est[c]
    print("PCG %s delta=%g tau=%g inner_max=%d: outer iterations %s, K V rounds %d (oracle "
          "%d), max rel err %.2e" % (precision, delta, tau, inner_max, [s[1] for s in st],
                                     rounds, sum(rounds_ref), max(errs)))
    assert checked >= R - 1
    assert max(errs) <= tol
    # K V rounds: every live column shares a round.  The first preconditioner solve takes as
    # many rounds as its longest column; then each outer iteration one round (K d) and, for
    # the columns still running, as many as the longest of their next inner solves
    if not flips:
        inner = [pcg.pcg_record(Xd, prob.psi_true, Bd[:, c], delta, tau, inner_max, eps=1e-8,
                                max_iter=500)["inner"] for c in range(R)]
        iters = [int(v) for v in st_ref[:, 1]]
        expect = max(inner[c][0] for c in range(R))
        for t in range(1, max(iters) + 1):
            expect += 1
            more = [inner[c][t] for c in range(R) if iters[c] > t]
            expect += max(more) if more else 0
        assert rounds == expect, (rounds, expect)


@pytest.mark.parametrize("n,d,R,delta,tau", [(400, 2, 4, 1.0, 1e-1), (500, 2, 5, 0.5, 1e-1),
                                             (600, 3, 3, 2.0, 1e-1)])
def test_pcg_solve_parity_fp64(orc, n, d, R, delta, tau):
    prob = w.random_problem(n, d, seed=900 + n)
    _case(orc, prob, R, u.PREC_FP64, delta, tau, 100, 1.0, 1e-6)


@pytest.mark.parametrize("precision", [u.PREC_FP32, u.PREC_MIXED])
@pytest.mark.parametrize("n,R,delta,inner_max", [(700, 4, 0.5, 2), (1500, 9, 1.0, 3),
                                                 (1200, 6, 0.2, 2)])
def test_pcg_solve_parity_fp32_mixed(orc, precision, n, R, delta, inner_max):
    prob = w.census_like(n=n, seed=300 + n)
    _case(orc, prob, R, precision, delta, 1e-6, inner_max, 1.0, 1e-4)


def test_pcg_converged_solve_is_cholesky(orc):
    """No early stop (q = 0): the outer PCG runs to its threshold; its result is the unique
    solution K^{-1} b whatever the inner solves did."""
    prob = w.random_problem(800, 2, seed=1801)
    n = prob.n
    B = np.random.default_rng(3).standard_normal((n, 3)).astype(np.float32)
    B[:, 0] = prob.y
    with _ctx(prob, precision=u.PREC_FP64, q=0.0, eps=1e-10, max_iter=2000, seed=1,
              pcg_delta=0.1, pcg_inner_tol=1e-2, pcg_inner_max=200) as ctx:
        S, st = ctx.solve(prob.psi_true, torch.from_numpy(B).cuda())
    S = S.cpu().numpy().astype(np.float64)
    for c in range(3):
        assert st[c][0] == 0 and st[c][2] == 0
        ref = orc.exact_solve(prob.X.astype(np.float64), prob.psi_true,
                              B[:, c].astype(np.float64))
        assert np.linalg.norm(S[:, c] - ref) <= 1e-6 * np.linalg.norm(ref), c


def test_pcg_gradient_unbiased(orc):
    """E[g~] = g with the PCG solves: the mean of 3,000 seeded gradient estimates (FP32 path)
    is within 4 standard errors of the exact gradient, in the regime where the sample
    standard error carries the truncation weights' expectation (noise variance 0.3, q = 0.1;
    see test_gpu_warm_probes.py)."""
    prob = w.census_like(n=600, seed=62, noise=0.3)
    g_exact = orc.exact_gradient(prob.X.astype(np.float64), prob.y.astype(np.float64),
                                 prob.psi_true)
    N = 3000
    with _ctx(prob, n_probes=2, q=0.1, max_iter=600, seed=321, pcg_delta=0.3,
              pcg_inner_tol=1e-2, pcg_inner_max=50) as ctx:
        G = np.array([ctx.grad(prob.psi_true, step=s)[0] for s in range(N)])
    se = G.std(axis=0, ddof=1) / math.sqrt(N)
    z = (G.mean(axis=0) - g_exact) / se
    print("PCG gradient: max |z| = %.2f" % np.max(np.abs(z)))
    assert np.max(np.abs(z)) < 4.0, (G.mean(axis=0), g_exact, se)


def test_pcg_sgld_step_runs_from_the_host_loop(orc):
    """An SGLD step with PCG solves (the step graph is not used for them): the same step
    twice gives the same parameters, and the gradient matches the oracle's PCG solves fed to
    the oracle's bilinear form."""
    prob = w.census_like(n=900, seed=77)
    with _ctx(prob, n_probes=4, seed=5, max_iter=500, pcg_delta=0.5, pcg_inner_tol=1e-6,
              pcg_inner_max=2) as ctx:
        p1, g1 = ctx.sgld_step(prob.psi_true, 1e-4, step=3)
        p2, g2 = ctx.sgld_step(prob.psi_true, 1e-4, step=3)
    assert np.array_equal(p1, p2) and np.array_equal(g1, g2)
    assert np.all(np.isfinite(g1))
    from oracle import pcg
    Xd, yd = prob.X.astype(np.float64), prob.y.astype(np.float64)
    B = np.column_stack([yd, orc.probes(prob.n, 4, 0, 5, 3)])
    n_est = np.array([2, 1, 1, 1, 1])
    S, st, _ = pcg.ulisse_pcg_solve(Xd, prob.psi_true, B, 0.5, 1e-6, 2, n_est=n_est, q=1.0,
                                    beta=1.0, eps=1e-8, max_iter=500, seed=5, step=3)
    # g = 1/2 a1^T dK a2 - 1/(2 N_r) sum_j z_j^T dK r_j (Eq. gradient:unbiased)
    A = np.column_stack([S[:, 0]] + [S[:, 2 + j] for j in range(4)])
    Bf = np.column_stack([S[:, 1]] + [B[:, 1 + j] for j in range(4)])
    scale = np.array([0.5] + [-1.0 / 8.0] * 4)
    gref = orc.dk_bilinear(Xd, prob.psi_true, A, Bf, scale)
    assert np.linalg.norm(g1 - gref) <= 1e-4 * np.linalg.norm(gref)
