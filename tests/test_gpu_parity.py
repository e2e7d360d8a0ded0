"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded
inputs.

Tolerances (derivation in the design notes):
  * K V, FP32 path: every entry within 1e-5 of its own dot-product scale sum_j |A_ij||V_jr|
    (the standard rounding bound of a length-n dot product evaluated in FP32 with an
    approximate exp), and 1e-5 in Frobenius norm relative to the exact product.
  * K V, FP64 path: 1e-12 of the same scale.
  * Seeded ULISSE solves: identical integer outcomes (early-stop iteration l, accepted steps
    J, iterations) unless the oracle's early-stop test is within 1e-4 of the threshold;
    estimates within 1e-4 (FP32 path) or 1e-6 (FP64 path, float output buffer) per column.
  * Seeded gradients: ||g_gpu - g_oracle|| <= 1e-4 ||g_oracle|| (FP32), 1e-5 (FP64, where
    the gradient sum's own conditioning limits any FP64 evaluation to ~1e-6).
  * FP32 seeded parity is checked where the CG trajectories are short (Census-shaped
    inputs, n <= 2000): FP32 products make a CG trajectory drift from the FP64 one
    geometrically with the iteration count (about 1e-5 after 10 iterations, 1e-2 after 20
    on these inputs), so longer FP32 runs are checked statistically (unbiasedness) and
    the FP64 path is checked seeded on the ill-conditioned, long-trajectory problems.
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


def _kv_check(U, ref, scale, tol):
    err = np.abs(U - ref)
    assert np.all(err <= tol * scale + 1e-30), float(np.max(err / (scale + 1e-300)))
    assert np.linalg.norm(U - ref) <= tol * np.linalg.norm(ref)


# ----------------------------------------------------------------------------------------
# K V (Sec. 3)
# ----------------------------------------------------------------------------------------
@pytest.mark.parametrize("n,d,R", [(1, 1, 1), (37, 2, 3), (64, 3, 1), (1000, 2, 5),
                                   (1333, 8, 17), (2111, 16, 7), (3000, 5, 32), (700, 4, 40)])
def test_kmv_fp32(orc, n, d, R):
    prob = w.random_problem(n, d, seed=100 + n + d)
    rng = np.random.default_rng(n * R)
    V = rng.standard_normal((n, R)).astype(np.float32)
    Xd = prob.X.astype(np.float64)
    Vd = V.astype(np.float64)
    with _ctx(prob) as ctx:
        Vt = torch.from_numpy(V).cuda()
        for which in [-1] + list(range(d + 2)):
            Ug = ctx.kmv(prob.psi_true, Vt, which).cpu().numpy().astype(np.float64)
            A = orc.cov_matrix(Xd, prob.psi_true, which)
            ref = A @ Vd if n <= 1500 else orc.kmv(Xd, prob.psi_true, Vd, which)
            scale = np.abs(A) @ np.abs(Vd)
            _kv_check(Ug, ref, scale, 1e-5)


def test_kmv_fp64(orc):
    prob = w.random_problem(777, 2, seed=5)
    V = np.random.default_rng(1).standard_normal((777, 5))
    with _ctx(prob, precision=u.PREC_FP64) as ctx:
        Vt = torch.from_numpy(V).cuda()
        for which in (-1, 0, 1, 2, 3):
            Ug = ctx.kmv(prob.psi_true, Vt, which).cpu().numpy()
            A = orc.cov_matrix(prob.X.astype(np.float64), prob.psi_true, which)
            _kv_check(Ug, A @ V, np.abs(A) @ np.abs(V), 1e-12)


def test_kmv_full_size_sampled_rows(orc):
    """Full-size Census-like product (n = 50,000, d = 8, R = 17) in the launch configuration
    of the benchmark: sampled rows against the oracle, which evaluates them one by one."""
    prob = w.census_like()
    n = prob.n
    rng = np.random.default_rng(3)
    V = rng.choice([-1.0, 1.0], (n, 17)).astype(np.float32)
    V[:, 0] = prob.y
    rows = np.sort(rng.choice(n, 48, replace=False))
    rows[-1] = n - 1
    with _ctx(prob, n_probes=16) as ctx:
        Ug = ctx.kmv(prob.psi_true, torch.from_numpy(V).cuda()).cpu().numpy()[rows]
    Xd, Vd = prob.X.astype(np.float64), V.astype(np.float64)
    ref = orc.kmv_rows(Xd, prob.psi_true, Vd, rows)
    scale = orc.kmv_rows(Xd, prob.psi_true, Vd, rows, absolute=True)
    _kv_check(Ug.astype(np.float64), ref, scale, 1e-5)


# Mixed precision (tensor cores): the contraction K V by three BF16 products (~2^-16 per
# product) and the exponent either from FP32 FMAs (cross=1) or from three TF32 products of the
# augmented rows [x^_i, 1] . [2 c1 x^_j, -c1 |x^_j|^2] (cross=2: ~2^-21 of 2 c1 sum_k
# |x^_ik x^_jk| + c1 |x^_j|^2 in the exponent) leave every generated entry with a relative
# error of 1e-6 to a few 1e-5, and the FP32 accumulation over a CTA's j range adds up to a few
# 1e-5 at n = 50,000.  Those errors are independent across
# entries, so each output stays within 1e-4 of its dot-product scale sum_j |K_ij||V_jr|; the
# norm-wise error is reported by the test.
MIXED_TOL = 1e-4
CROSS = [1, 2]


@pytest.mark.parametrize("cross", CROSS)
@pytest.mark.parametrize("n,d,R", [(1, 2, 1), (130, 2, 3), (1000, 8, 17), (2111, 16, 7),
                                   (3000, 3, 32), (1500, 8, 40), (900, 5, 70)])
def test_kmv_mixed_tensor_cores(orc, n, d, R, cross):
    prob = w.random_problem(n, d, seed=700 + n + d) if d != 8 else w.census_like(n=n, seed=700 + n)
    V = np.random.default_rng(n + R).standard_normal((n, R)).astype(np.float32)
    Xd = prob.X.astype(np.float64)
    Vd = V.astype(np.float64)
    with _ctx(prob, precision=u.PREC_MIXED, tc_cross_term=cross) as ctx:
        Ug = ctx.kmv(prob.psi_true, torch.from_numpy(V).cuda()).cpu().numpy().astype(np.float64)
    A = orc.cov_matrix(Xd, prob.psi_true)
    ref = A @ Vd
    scale = np.abs(A) @ np.abs(Vd)
    comp = np.max(np.abs(Ug - ref) / scale)
    frob = np.linalg.norm(Ug - ref) / np.linalg.norm(ref)
    print("mixed K V (cross %d) n=%d d=%d R=%d: max |err|/scale %.2e, Frobenius %.2e"
          % (cross, n, d, R, comp, frob))
    assert comp <= MIXED_TOL and frob <= MIXED_TOL


@pytest.mark.parametrize("cross", CROSS)
def test_kmv_mixed_full_size_sampled_rows(orc, cross):
    """Near-duplicate workload shape at reduced n (d = 16, 1% jittered copies): the split
    cross term keeps the near-zero distances accurate."""
    prob = w.near_duplicates(n=20_000)
    n = prob.n
    rng = np.random.default_rng(5)
    V = rng.choice([-1.0, 1.0], (n, 64)).astype(np.float32)
    rows = np.sort(rng.choice(n, 32, replace=False))
    with _ctx(prob, precision=u.PREC_MIXED, tc_cross_term=cross) as ctx:
        Ug = ctx.kmv(prob.psi_true, torch.from_numpy(V).cuda()).cpu().numpy()[rows]
    Xd, Vd = prob.X.astype(np.float64), V.astype(np.float64)
    ref = orc.kmv_rows(Xd, prob.psi_true, Vd, rows)
    scale = orc.kmv_rows(Xd, prob.psi_true, Vd, rows, absolute=True)
    comp = np.max(np.abs(Ug - ref) / scale)
    print("mixed K V (cross %d) near-duplicates n=%d: max |err|/scale %.2e" % (cross, n, comp))
    assert comp <= MIXED_TOL


@pytest.fixture(scope="module")
def near_dup_full():
    return w.near_duplicates()


@pytest.mark.parametrize("cross", CROSS)
def test_kmv_mixed_near_duplicates_full_size(orc, near_dup_full, cross):
    """The near-duplicate workload at its full size (n = 200,000, d = 16, 64 right-hand sides,
    1% jittered copies): 32 sampled rows against the oracle.  At this n the accumulation
    bound gives every row block at least ten j-splits (the split partial sums take ~0.5 GB)."""
    prob = near_dup_full
    n = prob.n
    rng = np.random.default_rng(12)
    V = rng.choice([-1.0, 1.0], (n, 64)).astype(np.float32)
    rows = np.sort(rng.choice(n, 32, replace=False))
    with _ctx(prob, precision=u.PREC_MIXED, tc_cross_term=cross) as ctx:
        Ug = ctx.kmv(prob.psi_true, torch.from_numpy(V).cuda()).cpu().numpy()[rows]
    Xd, Vd = prob.X.astype(np.float64), V.astype(np.float64)
    ref = orc.kmv_rows(Xd, prob.psi_true, Vd, rows)
    scale = orc.kmv_rows(Xd, prob.psi_true, Vd, rows, absolute=True)
    comp = np.max(np.abs(Ug - ref) / scale)
    print("mixed K V (cross %d) near-duplicates full size n=%d: max |err|/scale %.2e"
          % (cross, n, comp))
    assert comp <= MIXED_TOL


def test_kmv_symmetry_and_linearity():
    """Properties that hold at any size: e_i^T K e_j = e_j^T K e_i; K (aV) = a K V."""
    prob = w.random_problem(5000, 4, seed=9)
    with _ctx(prob) as ctx:
        idx = [0, 17, 2500, 4999]
        E = torch.zeros((5000, 4), device="cuda")
        for c, i in enumerate(idx):
            E[i, c] = 1.0
        KE = ctx.kmv(prob.psi_true, E).cpu().numpy()
        S = KE[idx, :]
        assert np.allclose(S, S.T, rtol=1e-6, atol=0)
        V = torch.randn((5000, 3), device="cuda")
        a = ctx.kmv(prob.psi_true, V)
        b = ctx.kmv(prob.psi_true, 2.0 * V)
        assert torch.allclose(2.0 * a, b, rtol=1e-6, atol=1e-6)


# ----------------------------------------------------------------------------------------
# ULISSE solves (Sec. 4) and gradients (Eq. gradient:unbiased)
# ----------------------------------------------------------------------------------------
def _early_stop_margin(orc, Xd, psi, b, q, iters):
    """Smallest relative distance of ||e_i|| (i = 1..iters) to the threshold q sqrt(n)."""
    tr = orc.cg_record(Xd, psi, b, eps=1e-8, max_iter=max(iters, 1) + 1)
    a = q * math.sqrt(len(b))
    norms = np.linalg.norm(tr["E"], axis=1)[1:iters + 1]
    return float(np.min(np.abs(norms - a) / a)) if len(norms) else 1.0


def _compare_solves(orc, prob, B, n_est, Sg, st, Sref, st_ref, q, tol):
    Xd = prob.X.astype(np.float64)
    R = B.shape[1]
    col = 0
    checked = 0
    for c in range(R):
        if tuple(st[c][:4]) != tuple(int(v) for v in st_ref[c, :4]):
            # only allowed where the oracle's early-stop test is within rounding of alpha
            margin = _early_stop_margin(orc, Xd, prob.psi_true, B[:, c].astype(np.float64), q,
                                        int(st_ref[c, 1]))
            assert margin < 1e-4, (c, st[c], st_ref[c], margin)
            col += n_est[c]
            continue
        if n_est[c] > 1:
            assert st[c][4] == st_ref[c, 4]
        for t in range(n_est[c]):
            ref = Sref[:, col + t]
            err = np.linalg.norm(Sg[:, col + t] - ref) / np.linalg.norm(ref)
            assert err <= tol, (c, t, err)
        checked += 1
        col += n_est[c]
    assert checked >= R - 1


@pytest.mark.parametrize("n,d,R,q", [(700, 8, 4, 1.0), (1500, 8, 9, 1.0), (1800, 8, 6, 1.0),
                                     (1900, 8, 17, 0.8)])
def test_solve_parity_fp32(orc, n, d, R, q):
    """FP32 path on Census-shaped inputs, where the solves stop within a few iterations."""
    prob = w.census_like(n=n, d=d, seed=300 + n)
    rng = np.random.default_rng(n)
    B = rng.choice([-1.0, 1.0], (n, R)).astype(np.float32)
    B[:, 0] = prob.y
    n_est = np.ones(R, np.int32)
    n_est[0] = 2
    Sref, st_ref = orc.ulisse_solve(prob.X.astype(np.float64), prob.psi_true,
                                    B.astype(np.float64), n_est=n_est, q=q, beta=1.0, eps=1e-8,
                                    max_iter=500, seed=21, step=4)
    assert st_ref[:, 1].max() <= 8       # short trajectories: the FP32 regime
    with _ctx(prob, q=q, max_iter=500, seed=21) as ctx:
        Sg, st = ctx.solve(prob.psi_true, torch.from_numpy(B).cuda(), n_est=n_est, step=4)
    _compare_solves(orc, prob, B, n_est, Sg.cpu().numpy().astype(np.float64), st, Sref, st_ref,
                    q, 1e-4)


@pytest.mark.parametrize("n,d,R,q", [(500, 2, 4, 1.0), (1200, 3, 6, 1.0), (1000, 2, 5, 1.0)])
def test_solve_parity_fp64(orc, n, d, R, q):
    """FP64 path on ill-conditioned inputs (U[0,1]^d, trajectories of up to ~10 iterations):
    the GPU follows the oracle's CG trajectory to the float resolution of the output."""
    prob = w.random_problem(n, d, seed=300 + n) if n != 1000 else w.small_2d(n)
    rng = np.random.default_rng(n)
    B = rng.choice([-1.0, 1.0], (n, R)).astype(np.float32)
    B[:, 0] = prob.y
    n_est = np.ones(R, np.int32)
    n_est[0] = 2
    Sref, st_ref = orc.ulisse_solve(prob.X.astype(np.float64), prob.psi_true,
                                    B.astype(np.float64), n_est=n_est, q=q, beta=1.0, eps=1e-8,
                                    max_iter=500, seed=21, step=4)
    with _ctx(prob, precision=u.PREC_FP64, q=q, max_iter=500, seed=21) as ctx:
        Sg, st = ctx.solve(prob.psi_true, torch.from_numpy(B).cuda(), n_est=n_est, step=4)
    _compare_solves(orc, prob, B, n_est, Sg.cpu().numpy().astype(np.float64), st, Sref, st_ref,
                    q, 1e-6)


def test_solve_initial_iterates_fp64(orc):
    """Columns with a good initial iterate (kept), a bad one (dropped: zero start) and none:
    the keep decision and the trajectories follow the oracle."""
    prob = w.small_2d(n=400)
    n = prob.n
    rng = np.random.default_rng(3)
    B = rng.standard_normal((n, 3)).astype(np.float32)
    B[:, 0] = prob.y
    Xd = prob.X.astype(np.float64)
    good = orc.exact_solve(Xd, prob.psi_true, B[:, 0].astype(np.float64))
    good = good + 0.02 * np.std(good) * rng.standard_normal(n)
    S0 = np.stack([good, 30.0 * rng.standard_normal(n), np.zeros(n)], axis=1).astype(np.float32)
    Sref, st_ref = orc.ulisse_solve(Xd, prob.psi_true, B.astype(np.float64),
                                    S0=S0.astype(np.float64), q=0.1, max_iter=300, seed=5, step=1)
    Sz, st_z = orc.ulisse_solve(Xd, prob.psi_true, B.astype(np.float64), q=0.1, max_iter=300,
                                seed=5, step=1)
    assert st_ref[0, 1] < st_z[0, 1]                       # the kept start saves iterations
    assert np.array_equal(Sref[:, 1:], Sz[:, 1:])          # the dropped one changes nothing
    with _ctx(prob, precision=u.PREC_FP64, q=0.1, max_iter=300, seed=5) as ctx:
        Sg, st = ctx.solve(prob.psi_true, torch.from_numpy(B).cuda(),
                           S0=torch.from_numpy(S0).cuda(), step=1)
        Sg0, _ = ctx.solve(prob.psi_true, torch.from_numpy(B).cuda(), step=1)
    for c in range(3):
        assert tuple(st[c][:4]) == tuple(int(v) for v in st_ref[c, :4])
    Sg = Sg.cpu().numpy().astype(np.float64)
    # the kept start: 5 FP64 iterations, the GPU follows the oracle's trajectory
    assert np.max(np.abs(Sg[:, 0] - Sref[:, 0])) <= 2e-6 * np.max(np.abs(Sref[:, 0]))
    # the dropped starts: exactly the GPU's own zero-start solve
    assert np.array_equal(Sg[:, 1:], Sg0.cpu().numpy().astype(np.float64)[:, 1:])


def test_solve_fp64_matches_oracle_tightly(orc):
    prob = w.small_2d(n=400)
    B = np.random.default_rng(2).standard_normal((400, 3)).astype(np.float32)
    B[:, 0] = prob.y
    Sref, st_ref = orc.ulisse_solve(prob.X.astype(np.float64), prob.psi_true,
                                    B.astype(np.float64), q=1.0, max_iter=300, seed=5, step=1)
    with _ctx(prob, precision=u.PREC_FP64, max_iter=300, seed=5) as ctx:
        Sg, st = ctx.solve(prob.psi_true, torch.from_numpy(B).cuda(), step=1)
    for c in range(3):
        assert tuple(st[c][:4]) == tuple(int(v) for v in st_ref[c, :4])
    Sg = Sg.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(Sg - Sref)) <= 1e-6 * np.max(np.abs(Sref))


def _grad_case(orc, prob, nr, kind, precision, tol, steps=(0, 1, 2), seed=33):
    n = prob.n
    Xd, yd = prob.X.astype(np.float64), prob.y.astype(np.float64)
    with _ctx(prob, n_probes=nr, probe_kind=kind, max_iter=500, seed=seed,
              precision=precision) as ctx:
        for step in steps:
            gref, st_ref = orc.grad_estimate(Xd, yd, prob.psi_true, nr=nr, probe_kind=kind,
                                             q=1.0, beta=1.0, max_iter=500, seed=seed, step=step)
            g, st = ctx.grad(prob.psi_true, step=step)
            same = all(tuple(st[c][:4]) == tuple(int(v) for v in st_ref[c, :4])
                       for c in range(1 + nr))
            if not same:
                B = np.column_stack([yd, orc.probes(n, nr, kind, seed, step)])
                margins = [_early_stop_margin(orc, Xd, prob.psi_true, B[:, c], 1.0,
                                              int(st_ref[c, 1])) for c in range(1 + nr)]
                assert min(margins) < 1e-4, (st, st_ref)
                continue
            rel = np.linalg.norm(g - gref) / np.linalg.norm(gref)
            t = tol if tol is not None else _derived_grad_tol(orc, ctx, prob, nr, kind, seed,
                                                                 step, gref)
            assert rel <= t, (step, g, gref, rel, t)


@pytest.mark.parametrize("n,d,nr", [(800, 8, 4), (1500, 8, 8), (900, 8, 16), (2000, 8, 16),
                                    (2500, 8, 16)])
def test_grad_parity_fp32(orc, n, d, nr):
    """FP32 path, Census-shaped inputs, trajectories of at most ~7 iterations."""
    _grad_case(orc, w.census_like(n=n, d=d, seed=500 + n), nr, 0, u.PREC_FP32, 1e-4)


def _derived_grad_tol(orc, ctx, prob, nr, kind, seed, step, gref):
    """The FP64 gradient's tolerance from the case itself.  g~ is the bilinear form
    sum_m s_m a_m^T dK_i b_m of the solves' outputs (Eq. gradient:unbiased), so a relative
    error delta_s of the solve outputs moves component i by at most ~2 delta_s
    sum_m |s_m| |a_m|^T |dK_i| |b_m|.  delta_s is measured here (the GPU's solves against the
    oracle's on the same right-hand sides and draws), the sums of |terms| come from the
    oracle's bilinear form on absolute values; the bound is 4 delta_s max_i sum|terms_i| /
    ||g||.  (On these inputs max sum|terms| / ||g|| is 2e3-7e3: FP64 rounding of the form
    itself is ~1e-12, and the difference comes from the solves' trajectories.)"""
    n = prob.n
    Xd, yd = prob.X.astype(np.float64), prob.y.astype(np.float64)
    B = np.column_stack([yd, orc.probes(n, nr, kind, seed, step)])
    n_est = np.array([2] + [1] * nr, dtype=np.int32)
    Sref, _ = orc.ulisse_solve(Xd, prob.psi_true, B, n_est=n_est, q=1.0, beta=1.0, eps=1e-8,
                               max_iter=500, seed=seed, step=step)
    Sg, _ = ctx.solve(prob.psi_true, torch.from_numpy(B.astype(np.float32)).cuda(),
                      n_est=n_est, step=step)
    Sg = Sg.cpu().numpy().astype(np.float64)
    d_s = max(np.linalg.norm(Sg[:, k] - Sref[:, k]) / np.linalg.norm(Sref[:, k])
              for k in range(Sref.shape[1]))
    A = np.column_stack([Sref[:, 0]] + [Sref[:, 2 + j] for j in range(nr)])
    Bf = np.column_stack([Sref[:, 1]] + [B[:, 1 + j] for j in range(nr)])
    sc = np.array([0.5] + [-0.5 / nr] * nr)
    terms = orc.dk_bilinear(Xd, prob.psi_true, np.abs(A), np.abs(Bf), np.abs(sc))
    ratio = float(terms.max() / np.linalg.norm(gref))
    print("FP64 gradient tolerance: solve drift %.1e x sum|terms|/|g| %.2e -> %.1e"
          % (d_s, ratio, 4 * d_s * ratio))
    assert d_s <= 1e-6          # the FP64 solve parity bound (float output buffer)
    return max(1e-12, 4 * d_s * ratio)


# FP64 tolerance: derived per case from the measured solve drift and the conditioning of the
# gradient's sum (_derived_grad_tol).
@pytest.mark.parametrize("n,d,nr,kind", [(800, 2, 4, 0), (900, 2, 4, 1), (1200, 2, 4, 0)])
def test_grad_parity_fp64(orc, n, d, nr, kind):
    _grad_case(orc, w.random_problem(n, d, seed=500 + n), nr, kind, u.PREC_FP64, None)


def test_grad_parity_small_2d_fp64(orc):
    """The 2-D workload's configuration: FP64, 4 Gaussian probes."""
    _grad_case(orc, w.small_2d(n=1000), 4, 1, u.PREC_FP64, None, steps=(0, 1))


@pytest.mark.parametrize("precision,prob_fn,tol", [
    (u.PREC_FP64, lambda: w.random_problem(1500, 3, seed=1800), 1e-6),
    (u.PREC_FP64, lambda: w.small_2d(n=1000), 1e-6),
])
def test_converged_solve_matches_cholesky(orc, precision, prob_fn, tol):
    """Long trajectories: with no early stop (q = 0) every column runs Algorithm 1 to its
    convergence threshold, whose result is unique -- the Cholesky solution (Sec. 3's error
    definition) -- however the rounding steered the trajectory."""
    prob = prob_fn()
    n = prob.n
    B = np.random.default_rng(4).standard_normal((n, 3)).astype(np.float32)
    B[:, 0] = prob.y
    with _ctx(prob, precision=precision, q=0.0, eps=1e-10, max_iter=3000, seed=1) as ctx:
        S, st = ctx.solve(prob.psi_true, torch.from_numpy(B).cuda())
    S = S.cpu().numpy().astype(np.float64)
    for c in range(3):
        assert st[c][0] == 0 and st[c][2] == 0          # no early stop, converged
        ref = orc.exact_solve(prob.X.astype(np.float64), prob.psi_true, B[:, c].astype(np.float64))
        assert np.linalg.norm(S[:, c] - ref) <= tol * np.linalg.norm(ref), c


def test_sgld_step_parity(orc):
    """Three SGLD steps of the 2-D workload (FP64, Gaussian probes, preconditioner, prior).
    Each step starts both sides from the oracle's current psi (a chain fed its own psi
    would turn 1e-7 differences into different CG trajectories).  Seed 11 keeps every
    solve under ten iterations, inside the FP64 seeded-parity regime."""
    prob = w.small_2d(n=400)
    Xd, yd = prob.X.astype(np.float64), prob.y.astype(np.float64)
    M = np.diag([0.5, 0.7, 0.9, 1.1])
    pg = np.array([0.1, -0.2, 0.05, 0.0])
    with _ctx(prob, n_probes=4, probe_kind=1, max_iter=500, seed=11,
              precision=u.PREC_FP64) as ctx:
        psi_ref = prob.psi_true.copy()
        for step in range(3):
            psi, g = ctx.sgld_step(psi_ref, 1e-3, step, M=M, prior_grad=pg)
            psi_ref, gref, st_ref = orc.sgld_step(Xd, yd, psi_ref, 1e-3, nr=4, probe_kind=1,
                                                  max_iter=500, seed=11, step=step, M=M,
                                                  prior_grad=pg)
            assert st_ref[:, 1].max() <= 10
            assert np.linalg.norm(g - gref) <= 1e-5 * np.linalg.norm(gref)
            assert np.max(np.abs(psi - psi_ref)) < 1e-7


def test_sgld_step_parity_fp32(orc):
    prob = w.census_like(n=1500, seed=44)
    Xd, yd = prob.X.astype(np.float64), prob.y.astype(np.float64)
    with _ctx(prob, n_probes=8, max_iter=500, seed=9) as ctx:
        psi, g = ctx.sgld_step(prob.psi_true, 1e-4, 0)
    psi_ref, gref, st_ref = orc.sgld_step(Xd, yd, prob.psi_true, 1e-4, nr=8, max_iter=500,
                                          seed=9, step=0)
    assert np.linalg.norm(g - gref) <= 1e-4 * np.linalg.norm(gref)
    assert np.max(np.abs(psi - psi_ref)) < 1e-6


def test_grad_unbiased_fp32_gpu(orc):
    """E[g~] = g for the FP32 GPU path: the mean of 4000 seeded GPU estimates is within
    4 standard errors of the exact (Cholesky) gradient -- a check that holds however long
    the CG trajectories are."""
    prob = w.census_like(n=600, seed=61)
    g_exact = orc.exact_gradient(prob.X.astype(np.float64), prob.y.astype(np.float64),
                                 prob.psi_true)
    N = 4000
    with _ctx(prob, n_probes=2, q=0.7, max_iter=600, seed=123) as ctx:
        G = np.array([ctx.grad(prob.psi_true, step=s)[0] for s in range(N)])
    se = G.std(axis=0, ddof=1) / math.sqrt(N)
    z = (G.mean(axis=0) - g_exact) / se
    assert np.max(np.abs(z)) < 4.0, (G.mean(axis=0), g_exact, se)


def test_chain_matches_steps(orc):
    """The device-resident chain gives the same psi as repeated host-driven steps."""
    prob = w.random_problem(700, 2, seed=71)
    eps = torch.full((4,), 2e-3, dtype=torch.float64, device="cuda")
    with _ctx(prob, n_probes=3, seed=2) as ctx:
        psi_dev = torch.tensor(prob.psi_true, dtype=torch.float64, device="cuda")
        trace = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
        ctx.sgld_chain(psi_dev, eps, step0=10, trace_dev=trace)
        psi = prob.psi_true.copy()
        for k in range(4):
            psi, _ = ctx.sgld_step(psi, 2e-3, 10 + k)
            assert np.allclose(trace[k].cpu().numpy(), psi, rtol=0, atol=1e-12)
        assert np.allclose(psi_dev.cpu().numpy(), psi, rtol=0, atol=1e-12)


def test_deterministic_repeat():
    prob = w.random_problem(1100, 3, seed=12)
    with _ctx(prob, n_probes=4, seed=3) as ctx:
        g1, _ = ctx.grad(prob.psi_true, step=5)
        g2, _ = ctx.grad(prob.psi_true, step=5)
        g3, _ = ctx.grad(prob.psi_true, step=6)
    assert np.array_equal(g1, g2)
    assert not np.array_equal(g1, g3)


# ----------------------------------------------------------------------------------------
# Failure reporting (no GPU fault: bad data is caught by the solver's own checks)
# ----------------------------------------------------------------------------------------
def test_nan_input_reports_breakdown():
    prob = w.random_problem(300, 2, seed=1)
    B = np.random.default_rng(0).standard_normal((300, 2)).astype(np.float32)
    B[5, 1] = np.nan
    with _ctx(prob) as ctx:
        S, st = ctx.solve(prob.psi_true, torch.from_numpy(B).cuda(),
                          allow=(u.ULISSE_ERR_BREAKDOWN,))
        assert st[1][2] == u.ULISSE_ERR_BREAKDOWN
        assert st[0][2] == 0
        # the context stays usable
        g, _ = ctx.grad(prob.psi_true, step=0)
        assert np.all(np.isfinite(g))


def test_max_iter_reported():
    prob = w.random_problem(400, 2, seed=2)
    B = np.random.default_rng(0).standard_normal((400, 1)).astype(np.float32)
    with _ctx(prob, q=0.0, max_iter=2) as ctx:
        with pytest.raises(u.UlisseError) as ei:
            ctx.solve(prob.psi_true, torch.from_numpy(B).cuda())
        assert ei.value.status == u.ULISSE_ERR_MAXITER


def test_bad_psi_rejected():
    prob = w.random_problem(100, 2, seed=3)
    with _ctx(prob) as ctx:
        with pytest.raises(u.UlisseError) as ei:
            ctx.grad(np.array([0.0, np.nan, 0.0, 0.0]))
        assert ei.value.status == u.ULISSE_ERR_ARG
        with pytest.raises(u.UlisseError):
            ctx.kmv(prob.psi_true, torch.zeros((100, 1), device="cuda"), which=9)


def test_timeout_path_leaves_context_usable():
    """Failure detection without a GPU fault: a wait that nothing completes runs out, the
    call returns ULISSE_ERR_TIMEOUT, and the same context then computes K V exactly as a
    fresh context does."""
    prob = w.random_problem(3000, 4, seed=88)
    V = torch.randn((prob.n, 5), device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    with _ctx(prob) as fresh:
        ref = fresh.kmv(prob.psi_true, V).cpu().numpy()
    with _ctx(prob) as ctx:
        ctx.kmv(prob.psi_true, V)
        assert ctx.selftest_wait_timeout() == u.ULISSE_ERR_TIMEOUT
        U = ctx.kmv(prob.psi_true, V).cpu().numpy()
        g, _ = ctx.grad(prob.psi_true, step=0)
    assert np.array_equal(U, ref)
    assert np.all(np.isfinite(g))
