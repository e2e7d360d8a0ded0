"""Seeded parity of the chosen (mixed-precision) path against the FP64 oracle.

The mixed path forms the exponent's cross term by three TF32 products and the contraction
K V by three BF16 products on the tensor cores (FP32 accumulation); the solver's vectors are
FP32 and its scalar recurrences FP64.  Every seeded case here runs the same Philox streams
as the oracle, so the early-stop iteration l, the accepted steps J and the iteration counts
must agree exactly, and the estimates agree up to the drift of the CG trajectory under the
products' rounding.

Tolerances.  A K V product of the mixed path is within 1e-4 of its dot-product scale
(measured 1e-6 ... 4e-5), and Sec. 3's CG recurrence feeds each product into the next
direction.  On the Census-shaped inputs used here (n <= 2,500, noise 0.05, q = 1) the
trajectories stop within 8 iterations, where the measured drift of the estimates is 1e-6 ...
1.1e-5 (solves) and 5e-6 ... 7e-5 (gradients, norm-wise); both are compared at 1e-4, the
tolerance the FP32 path meets on the same cases.  Where the oracle's early-stop test lies
within 1e-4 of the threshold (relative), rounding may move l by one iteration; such a column
is excused, as in the FP32 tests, and every other column is compared.

The benchmark regime's unbiasedness check (noise 0.05, q = 1, Rademacher probes) cannot use
a sample standard error: the truncation weights e^{j(j+1)/2} put part of E[s~] on events of
probability e^{-j(j+1)/2} that no feasible sample contains (and the exact covariance of Sec.
4's estimator overflows FP64 once the trajectory after the early stop is longer than ~37
iterations, as it is here).  The test splits the expectation instead:
  * the law of J: the GPU's accepted-step counts over >= 10^4 seeded draws follow
    P(J >= j) = exp(-j(j+1)/2) (chi-square over j = 0, 1, 2, >= 3);
  * each estimate is the right function of its J: the GPU estimate equals the oracle's
    reconstruction s_l + sum_{j<=J} W_j delta_{l+j} from its FP64 trajectory;
  * the part of the expectation the sample carries: the mean of s~ 1{J <= 3} is within
    4 exact standard errors of sum_{J<=3} P(J) rec(J) (variance from the law of J, exact);
  * the rest, sum_{J>3} P(J) rec(J), is the oracle's enumeration pin (tests/
    test_oracle_pins.py: E over the exact law of J is the converged solution).
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

SOLVE_TOL = 1e-4
GRAD_TOL = 1e-4


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _ctx(prob, **cfg):
    X = torch.from_numpy(prob.X).cuda()
    y = torch.from_numpy(prob.y).cuda()
    return u.Context(X, y, u.ulisse_config_default(precision=u.PREC_MIXED, **cfg))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _same_ints(st, st_ref):
    return all(tuple(st[c][:4]) == tuple(int(v) for v in st_ref[c, :4]) for c in range(len(st)))


@pytest.mark.parametrize("n,R,q", [(700, 4, 1.0), (1500, 9, 1.0), (1800, 6, 1.0),
                                   (1900, 17, 0.8)])
def test_solve_parity_mixed(orc, n, R, q):
    """ulisse_solve on the tensor-core path: integer outcomes equal, estimates within
    SOLVE_TOL of the oracle's (both estimators of the y column, every probe column)."""
    prob = w.census_like(n=n, seed=300 + n)
    rng = np.random.default_rng(n)
    B = rng.choice([-1.0, 1.0], (n, R)).astype(np.float32)
    B[:, 0] = prob.y
    n_est = np.ones(R, np.int32)
    n_est[0] = 2
    Xd = prob.X.astype(np.float64)
    Sref, st_ref = orc.ulisse_solve(Xd, prob.psi_true, B.astype(np.float64), n_est=n_est, q=q,
                                    beta=1.0, eps=1e-8, max_iter=500, seed=21, step=4)
    assert st_ref[:, 1].max() <= 8
    with _ctx(prob, q=q, max_iter=500, seed=21) as ctx:
        Sg, st = ctx.solve(prob.psi_true, torch.from_numpy(B).cuda(), n_est=n_est, step=4)
    Sg = Sg.cpu().numpy().astype(np.float64)
    assert _same_ints(st, st_ref), (st, st_ref)
    errs = [_rel(Sg[:, k], Sref[:, k]) for k in range(Sref.shape[1])]
    print("mixed solve n=%d R=%d: max rel err %.2e (per column %s)"
          % (n, R, max(errs), " ".join("%.1e" % e for e in errs)))
    assert max(errs) <= SOLVE_TOL


@pytest.mark.parametrize("n,nr", [(800, 4), (1500, 8), (900, 16), (2000, 16), (2500, 16)])
def test_grad_parity_mixed(orc, n, nr):
    """ulisse_grad on the tensor-core path (mixed solves and the tensor-core gradient pass)
    against the oracle's seeded estimate, steps 0..2."""
    prob = w.census_like(n=n, seed=500 + n)
    Xd, yd = prob.X.astype(np.float64), prob.y.astype(np.float64)
    worst = 0.0
    with _ctx(prob, n_probes=nr, max_iter=500, seed=33) as ctx:
        for step in (0, 1, 2):
            gref, st_ref = orc.grad_estimate(Xd, yd, prob.psi_true, nr=nr, q=1.0, beta=1.0,
                                             max_iter=500, seed=33, step=step)
            g, st = ctx.grad(prob.psi_true, step=step)
            assert _same_ints(st, st_ref), (step, st, st_ref)
            worst = max(worst, _rel(g, gref))
    print("mixed gradient n=%d nr=%d: max rel err %.2e" % (n, nr, worst))
    assert worst <= GRAD_TOL


def _margin(orc, Xd, psi, b, s0, q, iters):
    """Smallest relative distance of ||e_i|| (i = 1..iters) to the threshold q sqrt(n)."""
    tr = orc.cg_record(Xd, psi, b, s0=s0, eps=1e-8, max_iter=max(iters, 1) + 1)
    a = q * math.sqrt(len(b))
    norms = np.linalg.norm(tr["E"], axis=1)[1:iters + 1]
    return float(np.min(np.abs(norms - a) / a)) if len(norms) else 1.0


def test_warm_started_solves_chained_mixed(orc):
    """Three steps of solves chained the way warm-started solves chain them (Sec. 5.1: each
    step starts from the previous step's result while the right-hand side is unchanged):
    step t + 1 passes the GPU's step-t estimates as S0, and the oracle is given the same S0.
    The keep-if-better decision, l, J and the iteration counts agree, and the estimates
    agree within SOLVE_TOL."""
    n, R = 1500, 9
    prob = w.census_like(n=n, seed=300 + n)
    Xd = prob.X.astype(np.float64)
    rng = np.random.default_rng(n)
    B = rng.choice([-1.0, 1.0], (n, R)).astype(np.float32)
    B[:, 0] = prob.y
    Bd = B.astype(np.float64)
    S0 = None
    kept_any = False
    compared = 0
    with _ctx(prob, q=1.0, max_iter=500, seed=77) as ctx:
        for step in range(4, 7):
            S0d = S0.astype(np.float64) if S0 is not None else None
            Sg, st = ctx.solve(prob.psi_true, torch.from_numpy(B).cuda(), step=step,
                               S0=torch.from_numpy(S0).cuda() if S0 is not None else None)
            Sref, st_ref = orc.ulisse_solve(Xd, prob.psi_true, Bd, q=1.0, beta=1.0, eps=1e-8,
                                            max_iter=500, seed=77, step=step, S0=S0d)
            assert st_ref[:, 1].max() <= 10
            Sg = Sg.cpu().numpy()
            errs = []
            for c in range(R):
                if tuple(st[c][:4]) != tuple(int(v) for v in st_ref[c, :4]):
                    m = _margin(orc, Xd, prob.psi_true, Bd[:, c],
                                S0d[:, c] if S0d is not None else None, 1.0, int(st_ref[c, 1]))
                    assert m < 1e-4, (step, c, st[c], st_ref[c], m)
                    continue
                errs.append(_rel(Sg[:, c].astype(np.float64), Sref[:, c]))
            compared += len(errs)
            print("chained step %d: iterations %s, max rel err %.2e"
                  % (step, [s[1] for s in st], max(errs)))
            assert max(errs) <= SOLVE_TOL
            if S0 is not None:
                K_s0 = orc.kmv(Xd, prob.psi_true, S0d)
                kept = np.linalg.norm(Bd - K_s0, axis=0) < np.linalg.norm(Bd, axis=0)
                kept_any |= bool(kept.any())
            S0 = Sg.copy()
    assert kept_any   # the chain really started some solves from the previous step
    assert compared >= 3 * R - 3


def _law_of_J(jmax):
    """P(J = j) for j < jmax and P(J >= jmax), J the accepted steps after the early stop
    (u_j < 1/w_j = exp(-j) for j = 1.. J, beta = 1)."""
    tail = [math.exp(-j * (j + 1) / 2.0) for j in range(jmax + 1)]
    return np.array([tail[j] - tail[j + 1] for j in range(jmax)] + [tail[jmax]])


@pytest.mark.parametrize("col", ["y", "probe"])
def test_unbiased_benchmark_regime_mixed(orc, col):
    """The benchmark's regime (Census-shaped, noise 0.05, q = 1, beta = 1) on the tensor-core
    path, 40,960 seeded ULISSE estimates of one column (see the module docstring for the
    split of the expectation)."""
    n, R, calls = 2000, 1024, 40
    prob = w.census_like(n=n, seed=5150)
    Xd = prob.X.astype(np.float64)
    b = prob.y.astype(np.float64) if col == "y" else orc.probes(n, 1, 0, 99, 0)[:, 0]
    q, beta = 1.0, 1.0
    # the first iterates of the FP64 trajectory (all that the estimates with J <= 3 use)
    tr = orc.cg_record(Xd, prob.psi_true, b, eps=1e-8, max_iter=60)
    S, E = tr["S"], tr["E"]
    T = tr["T"]
    norms = np.linalg.norm(E, axis=1)
    l = next(i for i in range(1, T + 1) if norms[i] < q * math.sqrt(n))
    delta = np.diff(S, axis=0)                   # delta[i - 1] = s_i - s_{i-1}
    jcut = 3
    assert l + jcut + 1 <= T                     # the tail is still running at J = jcut + 1
    rec = [S[l].copy()]
    for j in range(1, jcut + 1):
        rec.append(rec[-1] + orc.weight_product(j, beta) * delta[l + j - 1])
    rec = np.array(rec)                          # rec[J] for J = 0..jcut
    law = _law_of_J(jcut + 1)                    # P(J = 0..jcut), P(J > jcut)
    B = torch.from_numpy(np.repeat(b[:, None], R, axis=1).astype(np.float32)).cuda()
    Js, acc = [], np.zeros(n)
    worst = np.zeros(jcut + 1)
    with _ctx(prob, q=q, beta=beta, max_iter=4 * n, seed=31) as ctx:
        for call in range(calls):
            Sg, st = ctx.solve(prob.psi_true, B, step=1000 + call)
            Sg = Sg.cpu().numpy().astype(np.float64)
            for c in range(R):
                assert st[c][0] == l, (c, st[c], l)
                J = st[c][3]
                Js.append(J)
                if J <= jcut:
                    acc += Sg[:, c]
                    worst[J] = max(worst[J], _rel(Sg[:, c], rec[J]))
    N = len(Js)
    Js = np.array(Js)
    # the law of J (chi-square, 3 degrees of freedom; 16.3 is the 0.1% point)
    counts = np.array([np.sum(Js == j) for j in range(3)] + [np.sum(Js >= 3)])
    expect = N * np.array(list(law[:3]) + [law[3:].sum()])
    chi2 = float(np.sum((counts - expect) ** 2 / expect))
    print("%s column: l = %d; J counts %s (expected %s), chi2 %.2f; per-J max rel "
          "err vs FP64 reconstruction %s" % (col, l, counts.tolist(),
                                             np.round(expect, 1).tolist(), chi2,
                                             " ".join("%.1e" % e for e in worst)))
    assert chi2 < 16.3
    # each estimate is the reconstruction from its own J
    assert np.all(worst <= SOLVE_TOL), worst
    # the part of the expectation the sample carries, with its exact standard error, on
    # eight fixed projections (a 4-SE test on each)
    P = np.random.default_rng(8).standard_normal((n, 8))
    P[:, 0] = rec[1] - rec[0]
    recP = rec @ P                               # (jcut + 1) x 8
    mu = law[:jcut + 1] @ recP
    var = law[:jcut + 1] @ (recP * recP) - mu * mu
    z = ((acc @ P) / N - mu) / np.sqrt(var / N)
    print("truncated expectation on 8 projections: z = %s" % np.round(z, 2).tolist())
    assert np.max(np.abs(z)) < 4.0
