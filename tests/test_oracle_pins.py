"""Pins for the FP64 oracle: checks against things other than the oracle itself.

Each test ties an oracle function to a closed form, an invariant, a library routine, brute
force on a tiny input or a value the paper prints, so that a plausible slip (a dropped term,
a wrong sign or index, a transposed operand, a wrong weight) fails at least one of them.

  function              pinned by
  --------------------  ------------------------------------------------------------------
  philox4x64_10         numpy.random.Philox (independent implementation), exact words
  u01 / probes          range, exact +-1 values, moments within 4 SE, E[r r^T] = I
  cov_matrix            closed forms (n=1, coincident points, distance l), scipy cdist,
                        symmetry, positive definiteness (eigvalsh >= lambda)
  cov_matrix(which)     central finite differences of K in psi; dK/dlog lambda = lambda I;
                        dK/dlog sigma^2 = K - lambda I
  kmv / dkmv_all /      dense matrix product with numpy on tiny and ragged sizes
  kmv_rows
  exact_gradient        central finite differences of the log marginal likelihood
  dk_bilinear           unit-vector factors give the hand-written entries of dK/dpsi_i; exact
                        solves and identity columns as factors give the exact gradient
  log_marginal_lik.     scipy.stats.multivariate_normal.logpdf
  cg_record             Cholesky solution (Sec. 3 error definition), conjugacy and residual
                        orthogonality, n=1 in one step, K ~ c I in one step
  draw_J                P(J >= j) = exp(-beta j (j+1)/2) within 4 SE; expected tail length
                        vs the paper's printed 1.4 at beta = 1 (tests/golden)
  ulisse_solve          reconstruction from the recorded CG trajectory; exact expectation by
                        enumerating J equals the converged CG solution; mean of 10^4 seeded
                        estimates within 4 SE (exact covariance) of the Cholesky solution;
                        a worse initial iterate gives the zero-start result bit for bit, a
                        kept one is reconstructed from its own trajectory
  grad_estimate         mean of 10^4 seeded estimates within 4 SE of the exact gradient;
                        Hutchinson identity by enumerating all sign vectors
  chol / sgld_update    numpy.linalg.cholesky; closed-form update with the drawn noise;
                        stationary moments of a Gaussian target
  cross_signal          sub-block of cov_matrix (signal part) for a subset of the inputs
  mlp.residual_matrices y_I - M c equals the rows I of y - K s_0 with dense K
  mlp.forward           a two-unit network evaluated by hand (tanh ln a = (a^2-1)/(a^2+1))
  mlp.loss_and_grad     central finite differences of the loss in every parameter block;
                        the loss at a hand-built exact fit is 0, the ridge term alone
  mlp.pooled_constant   the loss gradient in b3 vanishes there (W3 = 0), and any other
                        constant has a larger loss
  pcg.pcg_record        Cholesky solution (exact and inexact inner solves); d_i^T K d_j = 0
                        and e_i^T z_j = 0; delta -> 0 solves in one step, delta -> infinity
                        gives the C oracle's plain CG iterates; flexible beta = standard beta
                        with exact inner solves
  pcg.inner_cg          the stopping rule ||r|| <= tau ||e|| at the returned count, not before
  pcg.ulisse_pcg_solve  reconstruction from the outer trajectory; E over the exact law of J is
                        the Cholesky solution
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_X(n, d, seed, scale=1.0):
    return np.random.default_rng(seed).uniform(0.0, scale, (n, d))


# ----------------------------------------------------------------------------------------
# Random numbers
# ----------------------------------------------------------------------------------------
@pytest.mark.parametrize("ctr,key", [
    ((1, 0, 0, 0), (0, 0)),
    ((6, 7, 9, 11), (123, 456)),
    ((2**64 - 1, 2**63, 12345, 2**40 + 3), (2**64 - 1, 20150122)),
    ((977, 3, 20150123, 2 | (1 << 8)), (20150123, 0)),
])
def test_philox_matches_numpy(orc, ctr, key):
    # numpy's Philox pre-increments its counter: its first block is philox(counter + 1).
    c = list(ctr)
    c[0] = (c[0] - 1) % 2**64
    if ctr[0] == 0:
        pytest.skip("borrow case not needed")
    ref = np.random.Philox(counter=np.array(c, dtype=np.uint64),
                          key=np.array(key, dtype=np.uint64)).random_raw(4)
    got = orc.philox4x64_10(ctr, key)
    assert [int(x) for x in got] == [int(x) for x in ref]


def test_u01_range_and_moments(orc):
    words = np.random.Philox(key=[7, 9]).random_raw(200_000)
    u = np.array([orc.u01(int(w)) for w in words[:20000]])
    assert u.min() >= 0.0 and u.max() < 1.0
    n = len(u)
    assert abs(u.mean() - 0.5) < 4 * math.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 4 * math.sqrt(1 / 180 / n)
    # exact dyadic values: top 53 bits scaled by 2^-53
    assert orc.u01(0) == 0.0
    assert orc.u01(2**64 - 1) == (2**53 - 1) / 2**53


def test_probes_rademacher(orc):
    n, nr = 257, 3
    r = orc.probes(n, nr, 0, seed=11, epoch=5)
    assert r.shape == (n, nr)
    assert set(np.unique(r)) == {-1.0, 1.0}
    # E[r r^T] = I (Sec. 2.1): average outer products over many epochs of a short probe.
    m, reps = 6, 4000
    acc = np.zeros((m, m))
    for e in range(reps):
        v = orc.probes(m, 1, 0, seed=3, epoch=e)[:, 0]
        acc += np.outer(v, v)
    acc /= reps
    assert np.allclose(np.diag(acc), 1.0)
    off = acc[~np.eye(m, dtype=bool)]
    assert np.max(np.abs(off)) < 4.5 / math.sqrt(reps)
    # different epochs / columns / seeds give different probes
    assert not np.array_equal(orc.probes(n, 1, 0, 11, 5), orc.probes(n, 1, 0, 11, 6))
    assert not np.array_equal(r[:, 0], r[:, 1])


def test_probes_gaussian_moments(orc):
    z = orc.probes(50_000, 2, 1, seed=5, epoch=0).ravel()
    n = z.size
    assert abs(z.mean()) < 4 / math.sqrt(n)
    assert abs(z.var() - 1) < 4 * math.sqrt(2 / n)
    kurt = np.mean(z**4)
    assert abs(kurt - 3) < 4 * math.sqrt(96 / n)


# ----------------------------------------------------------------------------------------
# Covariance (Eq. covariance:rbf, ARD reading)
# ----------------------------------------------------------------------------------------
def test_cov_closed_forms(orc):
    psi = np.log([0.7, 1.3, 2.0, 0.25])   # l1, l2, sigma^2, lambda
    K = orc.cov_matrix(np.array([[0.3, -0.2]]), psi)
    assert K.shape == (1, 1) and abs(K[0, 0] - (2.0 + 0.25)) < 1e-15
    # coincident points: off-diagonal = sigma^2
    K = orc.cov_matrix(np.array([[0.1, 0.2], [0.1, 0.2]]), psi)
    assert abs(K[0, 1] - 2.0) < 1e-15 and abs(K[0, 0] - 2.25) < 1e-15
    # points one lengthscale apart along dim 0: sigma^2 e^{-1/2}
    K = orc.cov_matrix(np.array([[0.0, 0.0], [0.7, 0.0]]), psi)
    assert abs(K[0, 1] - 2.0 * math.exp(-0.5)) < 1e-14
    # along dim 1 by 2 l2: sigma^2 e^{-2}
    K = orc.cov_matrix(np.array([[0.0, 0.0], [0.0, 2.6]]), psi)
    assert abs(K[1, 0] - 2.0 * math.exp(-2.0)) < 1e-14


def test_cov_vs_scipy_cdist(orc):
    from scipy.spatial.distance import cdist
    X = _rand_X(37, 3, 1)
    psi = np.log([0.3, 0.5, 0.9, 1.7, 0.05])
    ls = np.exp(psi[:3])
    ref = 1.7 * np.exp(-0.5 * cdist(X / ls, X / ls, "sqeuclidean")) + 0.05 * np.eye(37)
    K = orc.cov_matrix(X, psi)
    assert np.max(np.abs(K - ref)) < 1e-14
    assert np.array_equal(K, K.T)
    assert np.linalg.eigvalsh(K).min() >= 0.05 * (1 - 1e-9)


@pytest.mark.parametrize("which", [0, 1, 2, 3, 4])
def test_dK_vs_finite_differences(orc, which):
    X = _rand_X(9, 3, 2)
    psi = np.log([0.4, 0.8, 0.6, 1.3, 0.2])
    h = 1e-5
    pp, pm = psi.copy(), psi.copy()
    pp[which] += h
    pm[which] -= h
    fd = (orc.cov_matrix(X, pp) - orc.cov_matrix(X, pm)) / (2 * h)
    dK = orc.cov_matrix(X, psi, which=which)
    assert np.max(np.abs(fd - dK)) < 1e-8


def test_dK_closed_forms(orc):
    X = _rand_X(11, 2, 3)
    psi = np.log([0.4, 0.8, 1.6, 0.3])
    K = orc.cov_matrix(X, psi)
    assert np.allclose(orc.cov_matrix(X, psi, which=3), 0.3 * np.eye(11), rtol=0, atol=1e-15)
    assert np.allclose(orc.cov_matrix(X, psi, which=2), K - 0.3 * np.eye(11), rtol=0, atol=1e-15)
    for q in range(2):
        assert np.all(np.diag(orc.cov_matrix(X, psi, which=q)) == 0.0)


@pytest.mark.parametrize("n,d,R", [(1, 1, 1), (5, 2, 3), (67, 3, 4), (130, 8, 2), (40, 2, 1100)])
def test_kmv_vs_dense(orc, n, d, R):
    X = _rand_X(n, d, 4 + n)
    psi = np.concatenate([np.log(np.full(d, 0.5)), [np.log(1.2), np.log(0.1)]])
    V = np.random.default_rng(n).standard_normal((n, R))
    for which in [-1] + list(range(d + 2)):
        dense = orc.cov_matrix(X, psi, which) @ V
        got = orc.kmv(X, psi, V, which)
        assert np.max(np.abs(got - dense)) <= 1e-12 * max(1.0, np.max(np.abs(dense)))
    allp = orc.dkmv_all(X, psi, V)
    for q in range(d + 2):
        dense = orc.cov_matrix(X, psi, q) @ V
        assert np.max(np.abs(allp[q] - dense)) <= 1e-12 * max(1.0, np.max(np.abs(dense)))


def test_kmv_rows_vs_dense(orc):
    n, d, R = 83, 3, 3
    X = _rand_X(n, d, 40)
    psi = np.log([0.4, 0.6, 0.5, 1.1, 0.2])
    V = np.random.default_rng(40).standard_normal((n, R))
    rows = [0, 5, 41, 82]
    for which in (-1, 1, 3, 4):
        A = orc.cov_matrix(X, psi, which)
        assert np.max(np.abs(orc.kmv_rows(X, psi, V, rows, which) - (A @ V)[rows])) < 1e-12
        absu = orc.kmv_rows(X, psi, V, rows, which, absolute=True)
        assert np.max(np.abs(absu - (np.abs(A) @ np.abs(V))[rows])) < 1e-12
    allr = orc.dkmv_all_rows(X, psi, V, rows)
    for q in range(d + 2):
        A = orc.cov_matrix(X, psi, q)
        assert np.max(np.abs(allr[q] - (A @ V)[rows])) < 1e-12


# ----------------------------------------------------------------------------------------
# Exact path (Sec. 2)
# ----------------------------------------------------------------------------------------
def test_log_marginal_likelihood_vs_scipy(orc):
    from scipy.stats import multivariate_normal
    X = _rand_X(40, 2, 5)
    psi = np.log([0.3, 0.6, 1.1, 0.2])
    y = np.random.default_rng(5).standard_normal(40)
    K = orc.cov_matrix(X, psi)
    ref = multivariate_normal(mean=np.zeros(40), cov=K).logpdf(y)
    assert abs(orc.log_marginal_likelihood(X, y, psi) - ref) < 1e-9 * abs(ref)


def test_exact_gradient_vs_fd_of_log_marginal_likelihood(orc):
    X = _rand_X(60, 3, 6)
    psi = np.log([0.35, 0.5, 0.8, 1.4, 0.15])
    y = np.random.default_rng(6).standard_normal(60)
    g = orc.exact_gradient(X, y, psi)
    h = 1e-5
    fd = np.zeros_like(psi)
    for i in range(len(psi)):
        pp, pm = psi.copy(), psi.copy()
        pp[i] += h
        pm[i] -= h
        fd[i] = (orc.log_marginal_likelihood(X, y, pp) - orc.log_marginal_likelihood(X, y, pm)) / (2 * h)
    assert np.max(np.abs(g - fd)) < 1e-6 * max(1.0, np.max(np.abs(g)))


def test_dk_bilinear_unit_vectors(orc):
    """a = e_p, b = e_q: the (p, q) entry of every derivative matrix, written out by hand:
    sigma^2 exp(-1/2 sum_k r_k^2) r_k^2 (r_k = (x_pk - x_qk) / l_k) for log l_k, the signal
    covariance for log sigma^2, lambda [p == q] for log lambda."""
    X = _rand_X(9, 3, 21)
    l = np.array([0.4, 0.7, 1.3])
    sig2, lam = 1.7, 0.2
    psi = np.log(np.concatenate([l, [sig2, lam]]))
    for p_, q_ in [(0, 0), (1, 5), (5, 1), (8, 2), (3, 3)]:
        A = np.zeros((9, 1))
        B = np.zeros((9, 1))
        A[p_, 0] = 1.0
        B[q_, 0] = 1.0
        out = orc.dk_bilinear(X, psi, A, B, scale=[1.0])
        r = (X[p_] - X[q_]) / l
        ks = sig2 * math.exp(-0.5 * float(np.sum(r * r)))
        want = np.concatenate([ks * r * r, [ks, lam if p_ == q_ else 0.0]])
        assert np.allclose(out, want, rtol=1e-13, atol=1e-15)
    # scale and the sum over m: two unit pairs with weights
    A = np.zeros((9, 2))
    B = np.zeros((9, 2))
    A[1, 0] = B[5, 0] = 1.0
    A[2, 1] = B[2, 1] = 1.0
    out = orc.dk_bilinear(X, psi, A, B, scale=[2.0, -0.5])
    one = orc.dk_bilinear(X, psi, A[:, :1], B[:, :1])
    two = orc.dk_bilinear(X, psi, A[:, 1:], B[:, 1:])
    assert np.allclose(out, 2.0 * one - 0.5 * two, rtol=1e-13, atol=1e-15)


def test_dk_bilinear_gives_the_exact_gradient(orc):
    """With a_0 = b_0 = K^{-1} y (weight 1/2) and a_k = K^{-1} e_k, b_k = e_k (weight -1/2) the
    forms are 1/2 y^T K^-1 dK K^-1 y - 1/2 tr(K^-1 dK): the exact gradient, itself pinned by
    finite differences of the log marginal likelihood."""
    n = 40
    X = _rand_X(n, 2, 22)
    psi = np.log([0.3, 0.5, 1.1, 0.2])
    y = np.random.default_rng(22).standard_normal(n)
    K = orc.cov_matrix(X, psi)
    Kinv = np.linalg.inv(K)
    alpha = Kinv @ y
    A = np.column_stack([alpha, Kinv])
    B = np.column_stack([alpha, np.eye(n)])
    scale = np.concatenate([[0.5], np.full(n, -0.5)])
    out = orc.dk_bilinear(X, psi, A, B, scale)
    g = orc.exact_gradient(X, y, psi)
    assert np.allclose(out, g, rtol=1e-9, atol=1e-10 * np.max(np.abs(g)))


# ----------------------------------------------------------------------------------------
# CG (Algorithm 1)
# ----------------------------------------------------------------------------------------
def test_cg_converges_to_cholesky(orc):
    X = _rand_X(80, 2, 7)
    psi = np.log([0.3, 0.3, 1.0, 0.1])
    b = np.random.default_rng(7).standard_normal(80)
    tr = orc.cg_record(X, psi, b, eps=1e-10)
    exact = orc.exact_solve(X, psi, b)
    assert np.linalg.norm(tr["S"][-1] - exact) < 1e-7 * np.linalg.norm(exact)
    assert np.linalg.norm(tr["E"][-1]) < 1e-10


def test_cg_invariants(orc):
    X = _rand_X(50, 2, 8)
    psi = np.log([0.5, 0.5, 1.0, 0.5])     # well conditioned: orthogonality holds to rounding
    b = np.random.default_rng(8).standard_normal(50)
    tr = orc.cg_record(X, psi, b, eps=1e-12)
    K = orc.cov_matrix(X, psi)
    k = min(6, tr["T"])
    Dm, Em = tr["D"][:k], tr["E"][:k]
    G = Dm @ K @ Dm.T
    off = G - np.diag(np.diag(G))
    assert np.max(np.abs(off)) < 1e-9 * np.max(np.diag(G))
    H = Em @ Em.T
    offe = H - np.diag(np.diag(H))
    assert np.max(np.abs(offe)) < 1e-9 * np.max(np.diag(H))
    # residual recurrence equals the true residual b - K s
    for i in range(k):
        assert np.linalg.norm(tr["E"][i] - (b - K @ tr["S"][i])) < 1e-10 * np.linalg.norm(b)


def test_cg_single_step_cases(orc):
    # n = 1: one step gives b / K
    X = np.array([[0.2, 0.4]])
    psi = np.log([0.5, 0.5, 2.0, 0.5])
    tr = orc.cg_record(X, psi, np.array([3.0]))
    assert tr["T"] == 1 and abs(tr["S"][-1][0] - 3.0 / 2.5) < 1e-15
    # far-apart points: K = (sigma^2 + lambda) I up to e^{-huge}; one step
    X = np.arange(10, dtype=float)[:, None] * 100.0
    psi = np.log([0.1, 1.5, 0.5])
    b = np.random.default_rng(9).standard_normal(10)
    tr = orc.cg_record(X, psi, b)
    assert tr["T"] == 1 and np.allclose(tr["S"][-1], b / 2.0, rtol=1e-15, atol=0)


# ----------------------------------------------------------------------------------------
# ULISSE (Sec. 4)
# ----------------------------------------------------------------------------------------
def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split("=", 1)
            vals[k.strip()] = float(v)
    return vals


def test_expected_tail_length_matches_paper(orc):
    g = _read_golden("ulisse_tail_length.txt")
    # the paper's rounded value for beta = 1
    assert abs(orc.expected_tail_steps(1.0) - g["expected_tail_steps_beta1"]) < g["tolerance"]
    # and the closed form of the same sum: sum_j exp(-beta j (j+1) / 2)
    cf = sum(math.exp(-j * (j + 1) / 2) for j in range(60))
    assert abs(orc.expected_tail_steps(1.0) - cf) < 1e-12


@pytest.mark.parametrize("beta", [1.0, 0.3])
def test_J_distribution(orc, beta):
    N = 20000
    Js = np.array([orc.draw_J(99, step, colid=5, est=0, beta=beta) for step in range(N)])
    for j in range(1, 5):
        p = math.exp(-beta * j * (j + 1) / 2)
        emp = np.mean(Js >= j)
        assert abs(emp - p) < 4 * math.sqrt(p * (1 - p) / N) + 1e-12
    # estimators 0 and 1 of the same column draw independently
    J0 = [orc.draw_J(1, s, 0, 0, beta) for s in range(3000)]
    J1 = [orc.draw_J(1, s, 0, 1, beta) for s in range(3000)]
    assert abs(np.corrcoef(J0, J1)[0, 1]) < 4 / math.sqrt(3000)


def _trajectory(orc, X, psi, b, eps):
    tr = orc.cg_record(X, psi, b, eps=eps)
    S = tr["S"]
    delta = np.diff(S, axis=0)           # delta_i = s_i - s_{i-1}, i = 1..T
    norms = np.linalg.norm(tr["E"], axis=1)
    return tr, S, delta, norms


def test_ulisse_reconstruction_from_trajectory(orc):
    n = 60
    X = _rand_X(n, 2, 10)
    psi = np.log([0.25, 0.25, 1.0, 0.05])
    b = np.random.default_rng(10).choice([-1.0, 1.0], n)
    q, beta, eps = 0.3, 1.0, 1e-10
    tr, S, delta, norms = _trajectory(orc, X, psi, b, eps)
    alpha = q * math.sqrt(n)
    l = next(i for i in range(1, tr["T"] + 1) if norms[i] < alpha)
    R = 200
    B = np.repeat(b[:, None], R, axis=1)
    S_est, st = orc.ulisse_solve(X, psi, B, colid=np.arange(R), q=q, beta=beta, eps=eps,
                                 seed=4, step=17)
    for c in range(R):
        J = int(st[c, 3])
        assert st[c, 0] == l
        ref = S[l].copy()
        for j in range(1, J + 1):
            if l + j > tr["T"]:
                break
            ref += orc.weight_product(j, beta) * delta[l + j - 1]
        assert np.linalg.norm(S_est[:, c] - ref) < 1e-9 * np.linalg.norm(ref)
        assert st[c, 1] == min(l + J, tr["T"])


def test_ulisse_expectation_by_enumeration(orc):
    """E[s~] over the exact law of J equals the converged CG solution s_T."""
    n = 40
    X = _rand_X(n, 2, 11)
    psi = np.log([0.3, 0.3, 1.0, 0.3])
    b = np.random.default_rng(11).standard_normal(n)
    q, beta = 0.5, 1.0
    tr, S, delta, norms = _trajectory(orc, X, psi, b, 1e-11)
    T = tr["T"]
    l = next(i for i in range(1, T + 1) if norms[i] < q * math.sqrt(n))
    # every J in 0..T-l has a representable probability, so the enumeration is complete
    assert T - l <= 30, (T, l)
    mean = np.zeros(n)
    for J in range(0, T - l + 1):
        pJ = math.exp(-beta * J * (J + 1) / 2) - (math.exp(-beta * (J + 1) * (J + 2) / 2)
                                                  if J < T - l else 0.0)
        est = S[l].copy()
        for j in range(1, J + 1):
            est += orc.weight_product(j, beta) * delta[l + j - 1]
        mean += pJ * est
    assert np.linalg.norm(mean - S[T]) < 1e-9 * np.linalg.norm(S[T])
    exact = orc.exact_solve(X, psi, b)
    assert np.linalg.norm(mean - exact) < 1e-7 * np.linalg.norm(exact)


def test_ulisse_unbiased_statistical(orc):
    """Mean of 10^4 seeded ULISSE estimates within 4 SE of the Cholesky solution, with the
    SE from the exact covariance Cov(s~) = sum_{j,k} (W_min(j,k) - 1) delta_j delta_k^T."""
    n = 48
    X = _rand_X(n, 2, 12)
    psi = np.log([0.3, 0.3, 1.0, 0.05])
    b = np.random.default_rng(12).choice([-1.0, 1.0], n)
    q, beta, eps = 0.5, 1.0, 1e-11
    tr, S, delta, norms = _trajectory(orc, X, psi, b, eps)
    T = tr["T"]
    l = next(i for i in range(1, T + 1) if norms[i] < q * math.sqrt(n))
    N = 10000
    B = np.repeat(b[:, None], N, axis=1)
    S_est, st = orc.ulisse_solve(X, psi, B, colid=np.arange(N), q=q, beta=beta, eps=eps,
                                 seed=2024, step=3)
    var = np.zeros(n)
    for j in range(1, T - l + 1):
        for k in range(1, T - l + 1):
            W = orc.weight_product(min(j, k), beta)
            var += (W - 1.0) * delta[l + j - 1] * delta[l + k - 1]
    se = np.sqrt(var / N)
    exact = orc.exact_solve(X, psi, b)
    z = (S_est.mean(axis=1) - exact) / np.maximum(se, 1e-300)
    assert np.max(np.abs(z)) < 4.0
    # the estimator is not degenerate: it really varies
    assert np.max(np.std(S_est, axis=1)) > 0
    # plain CG would need T iterations; ULISSE's mean cost is l + E[J]
    assert st[:, 1].mean() < T


def test_ulisse_initial_iterate_rule(orc):
    """An initial iterate s_0 is kept only when ||b - K s_0|| < ||b||.  A worse one gives
    exactly the zero-start estimates; a kept one starts CG (Algorithm 1) from s_0, and the
    expectation over the law of J, enumerated exactly, is still the solution of K s = b."""
    n = 40
    X = _rand_X(n, 2, 13)
    psi = np.log([0.3, 0.3, 1.0, 0.3])
    b = np.random.default_rng(13).standard_normal(n)
    q, beta, eps = 0.5, 1.0, 1e-11
    exact = orc.exact_solve(X, psi, b)
    R = 64
    B = np.repeat(b[:, None], R, axis=1)
    kw = dict(colid=np.arange(R), q=q, beta=beta, eps=eps, seed=6, step=2)
    S_zero, st_zero = orc.ulisse_solve(X, psi, B, **kw)
    bad = 50.0 * np.random.default_rng(14).standard_normal((n, R))
    S_bad, st_bad = orc.ulisse_solve(X, psi, B, S0=bad, **kw)
    assert np.array_equal(S_bad, S_zero) and np.array_equal(st_bad, st_zero)

    s0 = exact + 0.05 * np.linalg.norm(exact) / math.sqrt(n) * \
        np.random.default_rng(15).standard_normal(n)
    K = orc.cov_matrix(X, psi)
    assert np.linalg.norm(b - K @ s0) < np.linalg.norm(b)
    tr = orc.cg_record(X, psi, b, s0=s0, eps=eps)
    S, T = tr["S"], tr["T"]
    delta = np.diff(S, axis=0)
    norms = np.linalg.norm(tr["E"], axis=1)
    l = next(i for i in range(1, T + 1) if norms[i] < q * math.sqrt(n))
    S_est, st = orc.ulisse_solve(X, psi, B, S0=np.repeat(s0[:, None], R, axis=1), **kw)
    for c in range(R):
        J = int(st[c, 3])
        assert st[c, 0] == l
        ref = S[l].copy()
        for j in range(1, min(J, T - l) + 1):
            ref += orc.weight_product(j, beta) * delta[l + j - 1]
        assert np.linalg.norm(S_est[:, c] - ref) < 1e-9 * np.linalg.norm(ref)
    mean = np.zeros(n)
    for J in range(0, T - l + 1):
        pJ = math.exp(-beta * J * (J + 1) / 2) - (math.exp(-beta * (J + 1) * (J + 2) / 2)
                                                  if J < T - l else 0.0)
        est = S[l].copy()
        for j in range(1, J + 1):
            est += orc.weight_product(j, beta) * delta[l + j - 1]
        mean += pJ * est
    assert np.linalg.norm(mean - exact) < 1e-7 * np.linalg.norm(exact)


def test_hutchinson_identity_exhaustive(orc):
    """Sec. 2.1: E[r^T A r] = Tr(A) for +-1 probes, checked by enumerating all 2^n vectors."""
    n = 10
    X = _rand_X(n, 2, 13)
    psi = np.log([0.4, 0.4, 1.0, 0.1])
    K = orc.cov_matrix(X, psi)
    A = np.linalg.solve(K, orc.cov_matrix(X, psi, which=0))
    tot = 0.0
    for m in range(2**n):
        r = np.array([1.0 if (m >> i) & 1 else -1.0 for i in range(n)])
        tot += r @ A @ r
    assert abs(tot / 2**n - np.trace(A)) < 1e-10 * max(1.0, abs(np.trace(A)))
    assert abs(np.trace(A) - orc.exact_trace_term(X, psi, 0)) < 1e-10 * max(1.0, abs(np.trace(A)))


@pytest.mark.slow
def test_grad_estimate_unbiased(orc):
    """E[g~] = g (Eq. gradient:unbiased vs Eq. gradient:exact): mean of 10^4 seeded
    estimates within 4 standard errors of the Cholesky gradient."""
    n = 64
    rng = np.random.default_rng(14)
    X = rng.uniform(0, 1, (n, 2))
    psi = np.log([0.3, 0.4, 1.0, 0.1])
    y = np.linalg.cholesky(orc.cov_matrix(X, psi)) @ rng.standard_normal(n)
    g = orc.exact_gradient(X, y, psi)
    N = 10000
    G = np.array([orc.grad_estimate(X, y, psi, nr=2, q=0.5, beta=1.0, eps=1e-11, seed=77,
                                    step=s)[0] for s in range(N)])
    se = G.std(axis=0, ddof=1) / math.sqrt(N)
    z = (G.mean(axis=0) - g) / se
    assert np.max(np.abs(z)) < 4.0, (G.mean(axis=0), g, se)


def test_grad_estimate_without_truncation_is_hutchinson(orc):
    """With q -> 0 (no early stop) every solve is the converged CG solution, so g~ is the
    plain Hutchinson estimate; with the probes fixed it is a closed form in K."""
    n = 30
    rng = np.random.default_rng(15)
    X = rng.uniform(0, 1, (n, 2))
    psi = np.log([0.5, 0.5, 1.0, 0.2])
    y = rng.standard_normal(n)
    nr = 3
    g, st = orc.grad_estimate(X, y, psi, nr=nr, q=0.0, eps=1e-12, seed=5, step=9)
    r = orc.probes(n, nr, 0, 5, 9)
    K = orc.cov_matrix(X, psi)
    a = np.linalg.solve(K, y)
    for i in range(4):
        dK = orc.cov_matrix(X, psi, which=i)
        tr = sum(np.linalg.solve(K, r[:, j]) @ dK @ r[:, j] for j in range(nr)) / nr
        ref = -0.5 * tr + 0.5 * a @ dK @ a
        assert abs(g[i] - ref) < 1e-8 * max(1.0, abs(ref))
    assert np.all(st[:, 0] == 0)        # early stop never reached


# ----------------------------------------------------------------------------------------
# SGLD (Sec. 2.1)
# ----------------------------------------------------------------------------------------
def test_chol_vs_numpy(orc):
    A = np.random.default_rng(16).standard_normal((7, 7))
    M = A @ A.T + 7 * np.eye(7)
    assert np.allclose(orc.chol(M), np.linalg.cholesky(M), rtol=0, atol=1e-13)
    with pytest.raises(np.linalg.LinAlgError):
        orc.chol(-np.eye(3))


def test_sgld_update_closed_form(orc):
    p = 5
    rng = np.random.default_rng(17)
    psi = rng.standard_normal(p)
    g = rng.standard_normal(p)
    A = rng.standard_normal((p, p))
    M = A @ A.T + np.eye(p)
    pg = rng.standard_normal(p)
    eps_t = 3e-3
    xi = orc.sgld_noise(8, 21, p)
    out = orc.sgld_update(psi, g, eps_t, M=M, prior_grad=pg, seed=8, step=21)
    ref = psi + 0.5 * eps_t * M @ (g + pg) + math.sqrt(eps_t) * np.linalg.cholesky(M) @ xi
    assert np.allclose(out, ref, rtol=0, atol=1e-14)
    out = orc.sgld_update(psi, g, eps_t, seed=8, step=21)
    assert np.allclose(out, psi + 0.5 * eps_t * g + math.sqrt(eps_t) * xi, rtol=0, atol=1e-14)


def test_sgld_noise_moments(orc):
    Z = np.array([orc.sgld_noise(3, s, 4) for s in range(20000)])
    N = Z.shape[0]
    assert np.max(np.abs(Z.mean(axis=0))) < 4 / math.sqrt(N)
    C = np.cov(Z.T)
    assert np.max(np.abs(np.diag(C) - 1)) < 4 * math.sqrt(2 / N)
    assert np.max(np.abs(C - np.diag(np.diag(C)))) < 4 / math.sqrt(N)


def test_sgld_stationary_gaussian(orc):
    """With the exact gradient of a Gaussian log density, small-step SGLD leaves
    N(mu, Sigma) (approximately) invariant: the chain's mean and covariance match."""
    mu = np.array([0.5, -1.0])
    Sigma = np.array([[1.0, 0.6], [0.6, 2.0]])
    P = np.linalg.inv(Sigma)
    M = Sigma.copy()                      # preconditioner = posterior covariance
    eps_t = 0.02
    psi = mu.copy()
    N = 60000
    out = np.empty((N, 2))
    for t in range(N):
        g = -P @ (psi - mu)
        psi = orc.sgld_update(psi, g, eps_t, M=M, seed=12, step=t)
        out[t] = psi
    burn = out[1000:]
    # effective sample size: with M = Sigma the chain is an AR(1) with rho = 1 - eps/2
    rho = 1 - eps_t / 2
    ess = len(burn) * (1 - rho) / (1 + rho)
    se_mean = np.sqrt(np.diag(Sigma) / ess)
    assert np.all(np.abs(burn.mean(axis=0) - mu) < 4 * se_mean)
    C = np.cov(burn.T)
    # discretisation bias of the Euler step is O(eps); allow 4 SE + 2 eps relative
    for i in range(2):
        se_var = Sigma[i, i] * math.sqrt(2 / ess)
        assert abs(C[i, i] - Sigma[i, i]) < 4 * se_var + 2 * eps_t * Sigma[i, i]


# ----------------------------------------------------------------------------------------
# Learned warm start (oracle/mlp.py)
# ----------------------------------------------------------------------------------------
def test_cross_signal_is_covariance_block(orc):
    X = _rand_X(30, 3, 50)
    psi = np.log([0.4, 0.7, 0.5, 1.3, 0.2])
    K = orc.cov_matrix(X, psi) - 0.2 * np.eye(30)
    idx = [3, 7, 21, 29]
    C = orc.cross_signal(X, X[idx], psi)
    assert np.max(np.abs(C - K[:, idx])) < 1e-14


def _mlp_case(seed=0, p=4, hidden=7, A=5, m=6, T=3, n=12):
    from oracle import mlp
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, (n, p - 2))
    y = rng.standard_normal(n)
    Z = X[rng.choice(n, A, replace=False)]
    Rows = rng.integers(0, n, (T, m))
    Psi = np.log([0.4, 0.5, 1.0, 0.1]) + 0.1 * rng.standard_normal((T, p))
    w = 0.3 * rng.standard_normal(sum(int(np.prod(s)) for s in mlp.shapes(p, hidden, A)))
    mu = Psi.mean(axis=0)
    sd = Psi.std(axis=0) + 1e-3
    return mlp, w, Psi, Rows, X, y, Z, mu, sd, hidden


def test_mlp_residual_matrices_are_initial_residual_rows(orc):
    """y_I - M c is the initial residual y - K s_0 of Algorithm 1 at s_0 = K_s(X, Z) c, on
    the rows I (dense K from cov_matrix)."""
    mlp, w, Psi, Rows, X, y, Z, mu, sd, hidden = _mlp_case(seed=3)
    M = mlp.residual_matrices(X, Rows, Z, Psi)
    c = np.random.default_rng(4).standard_normal(Z.shape[0])
    for t, psi in enumerate(Psi):
        K = orc.cov_matrix(X, psi)
        s0 = orc.cross_signal(X, Z, psi) @ c
        ref = (y - K @ s0)[Rows[t]]
        assert np.allclose(y[Rows[t]] - M[t] @ c, ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))


def test_mlp_gradient_vs_finite_differences(orc):
    mlp, w, Psi, Rows, X, y, Z, mu, sd, hidden = _mlp_case()
    M = mlp.residual_matrices(X, Rows, Z, Psi)
    ridge = 0.01
    loss, g = mlp.loss_and_grad(w, Psi, Rows, X, y, Z, mu, sd, hidden, ridge)
    h = 1e-6
    rng = np.random.default_rng(1)
    idx = rng.choice(len(w), 40, replace=False)
    # every parameter block is represented
    sizes = np.cumsum([int(np.prod(s)) for s in mlp.shapes(4, hidden, 5)])
    idx = np.unique(np.concatenate([idx, sizes - 1]))
    for k in idx:
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        fd = (mlp.loss_and_grad(wp, Psi, Rows, X, y, Z, mu, sd, hidden, ridge, M=M)[0] -
              mlp.loss_and_grad(wm, Psi, Rows, X, y, Z, mu, sd, hidden, ridge, M=M)[0]) / (2 * h)
        assert abs(fd - g[k]) < 1e-7 * max(1.0, abs(fd)), (k, fd, g[k])


def test_mlp_exact_fit_has_zero_loss(orc):
    """With W3 = 0 the network outputs c = b3; data y = K K_s(X, Z) b3 at the pair's
    parameters has a zero initial residual, so the loss (ridge 0) and its gradient vanish."""
    mlp, w, Psi, Rows, X, _, Z, mu, sd, hidden = _mlp_case(seed=2, T=1)
    W1, b1, W2, b2, W3, b3 = mlp.unflatten(w, 4, hidden, 5)
    w0 = mlp.flatten([W1, b1, W2, b2, np.zeros_like(W3), b3])
    y = orc.cov_matrix(X, Psi[0]) @ (orc.cross_signal(X, Z, Psi[0]) @ b3)
    loss, g = mlp.loss_and_grad(w0, Psi, Rows, X, y, Z, mu, sd, hidden, 0.0)
    assert loss < 1e-26 and np.max(np.abs(g)) < 1e-12
    # the ridge term alone: rho ||b3||^2
    loss_r, _ = mlp.loss_and_grad(w0, Psi, Rows, X, y, Z, mu, sd, hidden, 0.5)
    assert abs(loss_r - 0.5 * np.sum(b3 * b3)) < 1e-12


def test_mlp_pooled_constant_is_the_loss_minimiser(orc):
    mlp, w, Psi, Rows, X, y, Z, mu, sd, hidden = _mlp_case(seed=5, T=4, m=9)
    ridge = 0.05
    M = mlp.residual_matrices(X, Rows, Z, Psi)
    c = mlp.pooled_constant(M, y[Rows], ridge)
    W1, b1, W2, b2, W3, b3 = mlp.unflatten(w, 4, hidden, 5)
    w0 = mlp.flatten([W1, b1, W2, b2, np.zeros_like(W3), c])
    loss, g = mlp.loss_and_grad(w0, Psi, Rows, X, y, Z, mu, sd, hidden, ridge, M=M)
    gb3 = g[-5:]
    assert np.max(np.abs(gb3)) < 1e-12 * max(1.0, np.max(np.abs(c)))
    rng = np.random.default_rng(6)
    for _ in range(5):
        w1 = mlp.flatten([W1, b1, W2, b2, np.zeros_like(W3), c + 0.01 * rng.standard_normal(5)])
        assert mlp.loss_and_grad(w1, Psi, Rows, X, y, Z, mu, sd, hidden, ridge, M=M)[0] > loss


def test_mlp_forward_hand_evaluated():
    """mlp.forward on a network small enough to evaluate by hand.  With p = 2, H = 2, A = 2,
    mu = (3, -1), sd = (2, 4) and psi = (5, -1) the standardised input is z = (1, 0).  W1's
    first row (ln 2, ln 3) and b1 = 0 give h1 = (tanh ln 2, tanh ln 3) = (3/5, 4/5) (tanh ln a
    = (a^2 - 1)/(a^2 + 1)); W1's second row (5, 7) is multiplied by z_2 = 0.  W2 = I and
    b2 = (ln 2 - 3/5, ln 3 - 4/5) give h2 = (3/5, 4/5) again.  W3 = [[2, 1/2], [-1, 1]] and
    b3 = (1/4, -1) give c = (6/5 - 4/5 + 1/4, 3/10 + 4/5 - 1) = (0.65, 0.1).  Dropping the
    standardisation (z = psi), a tanh, or transposing W1 or W3 changes c."""
    from oracle import mlp
    ln2, ln3 = math.log(2.0), math.log(3.0)
    W1 = np.array([[ln2, ln3], [5.0, 7.0]])
    b1 = np.zeros(2)
    W2 = np.eye(2)
    b2 = np.array([ln2 - 0.6, ln3 - 0.8])
    W3 = np.array([[2.0, 0.5], [-1.0, 1.0]])
    b3 = np.array([0.25, -1.0])
    w = mlp.flatten([W1, b1, W2, b2, W3, b3])
    mu, sd = np.array([3.0, -1.0]), np.array([2.0, 4.0])
    C, (Z, H1, H2) = mlp.forward(w, np.array([[5.0, -1.0]]), mu, sd, 2, 2, 2)
    assert np.allclose(Z, [[1.0, 0.0]], rtol=0, atol=1e-15)
    assert np.allclose(H1, [[0.6, 0.8]], rtol=0, atol=1e-15)
    assert np.allclose(H2, [[0.6, 0.8]], rtol=0, atol=1e-15)
    assert np.allclose(C, [[0.65, 0.1]], rtol=0, atol=1e-14)
    # a second input, z = (0, 1): h1 = tanh(W1[1]) = (tanh 5, tanh 7)
    C2, (_, H1b, H2b) = mlp.forward(w, np.array([[3.0, 3.0]]), mu, sd, 2, 2, 2)
    t5, t7 = math.tanh(5.0), math.tanh(7.0)
    assert np.allclose(H1b, [[t5, t7]], rtol=0, atol=1e-15)
    h2 = np.tanh(np.array([t5 + ln2 - 0.6, t7 + ln3 - 0.8]))
    assert np.allclose(C2[0], [2 * h2[0] - h2[1] + 0.25, 0.5 * h2[0] + h2[1] - 1.0],
                       rtol=0, atol=1e-14)


# ----------------------------------------------------------------------------------------
# Preconditioned CG, J = K + delta I (oracle/pcg.py; Sec. 3 "Preconditioned CG", Sec. 4)
# ----------------------------------------------------------------------------------------
def _pcg_problem(n=60, seed=21, noise=0.05):
    X = _rand_X(n, 2, seed)
    psi = np.log([0.25, 0.35, 1.0, noise])
    b = np.random.default_rng(seed).standard_normal(n)
    return X, psi, b


def test_pcg_converges_to_cholesky(orc):
    """Exact and inexact inner solves both reach the Cholesky solution (Sec. 3's error)."""
    from oracle import pcg
    X, psi, b = _pcg_problem()
    exact = orc.exact_solve(X, psi, b)
    for kw in (dict(exact_inner=True), dict(tau=1e-3, inner_max=200), dict(tau=1e-1, inner_max=30)):
        tr = pcg.pcg_record(X, psi, b, delta=0.3, eps=1e-10, **kw)
        assert np.linalg.norm(tr["S"][-1] - exact) < 1e-7 * np.linalg.norm(exact), kw


def test_pcg_invariants_with_exact_inner_solves(orc):
    """With a fixed preconditioner the directions are K-conjugate and the residuals are
    J^{-1}-orthogonal: d_i^T K d_j = 0 and e_i^T z_j = 0 for i != j (Golub & Van Loan)."""
    from oracle import pcg
    X, psi, b = _pcg_problem(n=40)
    K = orc.cov_matrix(X, psi)
    tr = pcg.pcg_record(X, psi, b, delta=0.5, eps=1e-11, exact_inner=True, max_iter=8)
    D, E, Z = tr["D"], tr["E"], tr["Z"]
    m = min(len(D), 6)
    G = D[:m] @ K @ D[:m].T
    off = G - np.diag(np.diag(G))
    assert np.max(np.abs(off)) < 1e-8 * np.max(np.abs(np.diag(G)))
    H = E[:m] @ Z[:m].T
    offh = H - np.diag(np.diag(H))
    assert np.max(np.abs(offh)) < 1e-8 * np.max(np.abs(np.diag(H)))


def test_pcg_limits(orc):
    """delta -> 0 with exact inner solves: J = K and one outer iteration gives K^{-1} b.
    delta -> infinity: J^{-1} -> I / delta, and PCG with a multiple of the identity is plain
    CG -- the outer iterates equal the C oracle's Algorithm 1 (cg_record)."""
    from oracle import pcg
    X, psi, b = _pcg_problem(n=50)
    exact = orc.exact_solve(X, psi, b)
    tr = pcg.pcg_record(X, psi, b, delta=0.0, eps=1e-9, exact_inner=True, max_iter=3)
    assert np.linalg.norm(tr["S"][1] - exact) < 1e-9 * np.linalg.norm(exact)
    tr = pcg.pcg_record(X, psi, b, delta=1e12, eps=1e-12, exact_inner=True, max_iter=8)
    ref = orc.cg_record(X, psi, b, eps=1e-12, max_iter=8)
    for i in range(1, 9):
        assert np.linalg.norm(tr["S"][i] - ref["S"][i]) < 1e-7 * np.linalg.norm(ref["S"][i]), i


def test_pcg_flexible_beta_equals_standard_with_exact_solves(orc):
    """With exact inner solves e_{i+1}^T z_i = 0, so the flexible beta equals
    e_{i+1}^T z_{i+1} / e_i^T z_i."""
    from oracle import pcg
    X, psi, b = _pcg_problem(n=45)
    tr = pcg.pcg_record(X, psi, b, delta=0.2, eps=1e-11, exact_inner=True, max_iter=6)
    E, Z = tr["E"], tr["Z"]
    for i in range(len(Z) - 1):
        std = float(E[i + 1] @ Z[i + 1]) / float(E[i] @ Z[i])
        assert abs(tr["beta"][i] - std) < 1e-9 * max(1.0, abs(std)), i


def test_pcg_inner_cg_stopping_rule(orc):
    """The inner CG stops at the first iteration with ||r|| <= tau ||e||: at that count the
    residual of J z = e is below the threshold, one iteration earlier it is not."""
    from oracle import pcg
    X, psi, b = _pcg_problem(n=50)
    Jm = orc.cov_matrix(X, psi) + 0.2 * np.eye(50)
    for tau in (1e-1, 1e-2, 1e-4):
        x, k = pcg.inner_cg(Jm, b, tau, 500)
        assert np.linalg.norm(b - Jm @ x) <= tau * np.linalg.norm(b) * (1 + 1e-9)
        if k > 1:
            x1, _ = pcg.inner_cg(Jm, b, tau, k - 1)
            assert np.linalg.norm(b - Jm @ x1) > tau * np.linalg.norm(b) * (1 - 1e-9)


def test_ulisse_on_pcg_expectation_by_enumeration(orc):
    """Sec. 4 applies to the outer PCG iteration: the estimates are the reconstruction from
    the outer trajectory, and E over the exact law of J is the converged solution, which is
    the Cholesky solution."""
    from oracle import pcg
    X, psi, b = _pcg_problem(n=40, noise=0.2)
    q, beta = 0.3, 1.0
    tr = pcg.pcg_record(X, psi, b, delta=0.4, tau=1e-3, inner_max=200, eps=1e-11)
    S, T = tr["S"], tr["T"]
    norms = np.linalg.norm(tr["E"], axis=1)
    l = next(i for i in range(1, T + 1) if norms[i] < q * math.sqrt(40))
    assert T - l <= 30
    mean = np.zeros(40)
    for J in range(0, T - l + 1):
        pJ = math.exp(-beta * J * (J + 1) / 2) - (math.exp(-beta * (J + 1) * (J + 2) / 2)
                                                  if J < T - l else 0.0)
        est = S[l].copy()
        for j in range(1, J + 1):
            est += pcg.weight(j, beta) * (S[l + j] - S[l + j - 1])
        mean += pJ * est
    exact = orc.exact_solve(X, psi, b)
    assert np.linalg.norm(mean - exact) < 1e-7 * np.linalg.norm(exact)
    # the solver's estimates are those reconstructions with the drawn J
    Bm = np.repeat(b[:, None], 16, axis=1)
    Sest, st, _ = pcg.ulisse_pcg_solve(X, psi, Bm, delta=0.4, tau=1e-3, inner_max=200, q=q,
                                       beta=beta, eps=1e-11, seed=9, step=2)
    for c in range(16):
        J = int(st[c, 3])
        ref = S[l].copy()
        for j in range(1, min(J, T - l) + 1):
            ref += pcg.weight(j, beta) * (S[l + j] - S[l + j - 1])
        assert st[c, 0] == l and st[c, 1] == min(l + J, T)
        assert np.linalg.norm(Sest[:, c] - ref) < 1e-12 * np.linalg.norm(ref)


# ----------------------------------------------------------------------------------------
# Posterior predictive (oracle.predict; Sec. 2, Eq. monte:carlo:integration)
# ----------------------------------------------------------------------------------------
def test_predict_single_training_point(orc):
    """n = 1: mean = k_s(x*, x1) y1 / (sigma^2 + lambda), var = sigma^2 + lambda -
    k_s(x*, x1)^2 / (sigma^2 + lambda), k_s = sigma^2 exp(-1/2 sum (x* - x1)^2 / l^2)."""
    psi = np.log([0.5, 2.0, 1.5, 0.2])
    X = np.array([[0.3, -0.4]])
    y = np.array([1.7])
    Xs = np.array([[0.1, 0.6], [0.3, -0.4]])
    mean, var = orc.predict(X, y, psi, Xs)
    s2, lam = 1.5, 0.2
    for j in range(2):
        k = s2 * math.exp(-0.5 * ((Xs[j, 0] - 0.3) ** 2 / 0.25 + (Xs[j, 1] + 0.4) ** 2 / 4.0))
        assert abs(mean[j] - k * 1.7 / (s2 + lam)) < 1e-14
        assert abs(var[j] - (s2 + lam - k * k / (s2 + lam))) < 1e-14


def test_predict_matches_sklearn(orc):
    """An independent implementation: scikit-learn's Gaussian-process regressor with the same
    fixed covariance (ConstantKernel sigma^2 x RBF(l) + WhiteKernel(lambda), no optimisation)
    gives the same predictive mean and, with the noise kernel at the test input, the same
    variance of a new label."""
    gp = pytest.importorskip("sklearn.gaussian_process")
    kern = pytest.importorskip("sklearn.gaussian_process.kernels")
    rng = np.random.default_rng(31)
    X = rng.uniform(0, 1, (60, 3))
    y = np.sin(4 * X[:, 0]) + 0.3 * rng.standard_normal(60)
    psi = np.log([0.3, 0.5, 0.8, 1.3, 0.05])
    Xs = rng.uniform(0, 1, (25, 3))
    k = (kern.ConstantKernel(1.3, "fixed") * kern.RBF([0.3, 0.5, 0.8], "fixed")
         + kern.WhiteKernel(0.05, "fixed"))
    reg = gp.GaussianProcessRegressor(kernel=k, optimizer=None, alpha=0.0, normalize_y=False)
    reg.fit(X, y)
    m_ref, sd_ref = reg.predict(Xs, return_std=True)
    mean, var = orc.predict(X, y, psi, Xs)
    assert np.max(np.abs(mean - m_ref)) < 1e-8 * max(1.0, np.max(np.abs(m_ref)))
    assert np.max(np.abs(var - sd_ref ** 2)) < 1e-8


def test_predict_at_training_inputs(orc):
    """At a training input the mean is the smoothed value (K_s K^{-1} y)_i and the latent
    variance (var - lambda) is the posterior variance diag(K_s - K_s K^{-1} K_s)_i -- the
    textbook smoother, formed here from the dense matrices with numpy."""
    X = _rand_X(40, 2, 32)
    psi = np.log([0.3, 0.4, 1.0, 0.1])
    y = np.random.default_rng(32).standard_normal(40)
    K = orc.cov_matrix(X, psi)
    Ks = K - 0.1 * np.eye(40)
    mean, var = orc.predict(X, y, psi, X[[3, 17]])
    sm = Ks @ np.linalg.solve(K, y)
    pv = np.diag(Ks - Ks @ np.linalg.solve(K, Ks))
    assert np.allclose(mean, sm[[3, 17]], rtol=0, atol=1e-12)
    assert np.allclose(var - 0.1, pv[[3, 17]], rtol=0, atol=1e-12)
