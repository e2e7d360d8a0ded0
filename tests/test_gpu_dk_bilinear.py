"""The fused gradient pass on its own (ulisse_dk_bilinear, Eq. gradient:unbiased, Sec. 4.1):
every component of out_i = sum_m s_m a_m^T (dK/dpsi_i) b_m against the FP64 oracle.

The derivative matrices have no negative entries, so the natural error scale of component i
is scale_i = sum_m |s_m| |a_m|^T dK_i |b_m| (the same form with |A|, |B|, |s|); the components
themselves can be far smaller than their scale when the factors have mixed signs, as the
gradient's do.  Bounds:
  * FP32 (SIMT, FP32 tile sums, FP64 across tiles): 1e-5 of the scale;
  * mixed (tensor cores: W = A B^T and the sums P [x, x^2, 1] by three BF16 products each, FP32
    accumulation, the x^2 S - 2 x G + H combination in FP64): 1e-4 of the scale;
  * FP64: 1e-10 of the scale.
At the census-like size (n = 50,000, d = 8, M = 17) the oracle's O(n^2 M p) sum takes minutes,
so the mixed pass is checked there against sum_m s_m a_m . (dK_i b_m) built from the FP32
derivative products of ulisse_kmv (themselves parity-tested against the oracle at 1e-5)."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU runs deselect this module
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1501_05427_gb300 import ulisse as u  # noqa: E402
from paper_1501_05427_gb300 import workloads as w  # noqa: E402

TOL = {u.PREC_FP32: 1e-5, u.PREC_MIXED: 1e-4, u.PREC_FP64: 1e-10}


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _ctx(prob, precision):
    X = torch.from_numpy(prob.X).cuda()
    y = torch.from_numpy(prob.y).cuda()
    return u.Context(X, y, u.ulisse_config_default(precision=precision))


def _factors(n, M, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, M)).astype(np.float32)
    B = rng.standard_normal((n, M)).astype(np.float32)
    s = rng.choice([0.5, -0.25, -1.0 / 32.0], M)
    return A, B, s


def _rel(err, scale, prob):
    """err / scale per component.  A lengthscale scale vanishes only when every pair of
    points coincides in that coordinate (n = 1): there the mixed pass's x^2 S - 2 x G + H
    expansion leaves rounding of the size of its terms, scale_sigma x max_j x^_jk^2."""
    d = prob.d
    xh2 = np.max((prob.X.astype(np.float64) / np.exp(prob.psi_true[:d])) ** 2, axis=0)
    floor = np.concatenate([scale[d] * xh2, [0.0, 0.0]])
    den = np.where(scale > 0, scale, floor)
    return np.where(den > 0, err / np.where(den > 0, den, 1.0), err)


def _check(orc, prob, M, precision, seed):
    A, B, s = _factors(prob.n, M, seed)
    Xd = prob.X.astype(np.float64)
    ref = orc.dk_bilinear(Xd, prob.psi_true, A.astype(np.float64), B.astype(np.float64), s)
    scale = orc.dk_bilinear(Xd, prob.psi_true, np.abs(A).astype(np.float64),
                            np.abs(B).astype(np.float64), np.abs(s))
    with _ctx(prob, precision) as ctx:
        out = ctx.dk_bilinear(prob.psi_true, torch.from_numpy(A).cuda(),
                              torch.from_numpy(B).cuda(), s)
    rel = _rel(np.abs(out - ref), scale, prob)
    print("dk_bilinear %s n=%d d=%d M=%d: max |err|/scale %.2e, max |err|/|out| %.2e"
          % ({0: "fp32", 1: "mixed", 2: "fp64"}[precision], prob.n, prob.d, M, rel.max(),
             np.max(np.abs(out - ref) / np.maximum(np.abs(ref), 1e-300))))
    assert np.all(np.isfinite(out))
    assert rel.max() <= TOL[precision]


# M covers every slot count of the tensor-core pass: 2M <= 16, 32, 48, 64 and 128
CASES = [(1, 2, 1), (130, 2, 3), (1000, 8, 17), (2111, 5, 9), (700, 16, 33), (900, 4, 64),
         (3000, 3, 16), (1500, 8, 28)]


def _prob(n, d):
    return w.census_like(n=n, seed=900 + n) if d == 8 else w.random_problem(n, d, seed=900 + n + d)


@pytest.mark.parametrize("n,d,M", CASES)
def test_dk_bilinear_fp32(orc, n, d, M):
    _check(orc, _prob(n, d), M, u.PREC_FP32, seed=n + M)


@pytest.mark.parametrize("n,d,M", CASES)
def test_dk_bilinear_mixed_tensor_cores(orc, n, d, M):
    _check(orc, _prob(n, d), M, u.PREC_MIXED, seed=n + M)


@pytest.mark.parametrize("n,d,M", [(1, 2, 1), (130, 2, 3), (777, 8, 17)])
def test_dk_bilinear_fp64(orc, n, d, M):
    _check(orc, _prob(n, d), M, u.PREC_FP64, seed=n + M)


def test_dk_bilinear_gives_the_exact_gradient(orc):
    """Exact solves and identity columns as factors: the forms are the exact gradient
    1/2 y^T K^-1 dK K^-1 y - 1/2 tr(K^-1 dK) (n = 60, M = 61 <= 64), in every precision."""
    prob = w.random_problem(60, 2, seed=31)
    Xd = prob.X.astype(np.float64)
    K = orc.cov_matrix(Xd, prob.psi_true)
    Kinv = np.linalg.inv(K)
    alpha = Kinv @ prob.y.astype(np.float64)
    A = np.column_stack([alpha, Kinv]).astype(np.float32)
    B = np.column_stack([alpha, np.eye(60)]).astype(np.float32)
    s = np.concatenate([[0.5], np.full(60, -0.5)])
    g = orc.exact_gradient(Xd, prob.y.astype(np.float64), prob.psi_true)
    # the float32 factors are the exact solve rounded: compare with the oracle on them too
    ref = orc.dk_bilinear(Xd, prob.psi_true, A.astype(np.float64), B.astype(np.float64), s)
    scale = orc.dk_bilinear(Xd, prob.psi_true, np.abs(A).astype(np.float64),
                            np.abs(B).astype(np.float64), np.abs(s))
    assert np.allclose(ref, g, rtol=1e-4, atol=1e-5 * np.max(np.abs(g)))
    for prec in (u.PREC_FP32, u.PREC_MIXED, u.PREC_FP64):
        with _ctx(prob, prec) as ctx:
            out = ctx.dk_bilinear(prob.psi_true, torch.from_numpy(A).cuda(),
                                  torch.from_numpy(B).cuda(), s)
        assert np.max(np.abs(out - ref) / scale) <= TOL[prec]


def test_dk_bilinear_full_size_mixed():
    """census_like at full size: the tensor-core pass against the FP32 derivative products
    (ulisse_kmv, which = i), and both timed."""
    prob = w.census_like()
    n, M = prob.n, 17
    A, B, s = _factors(n, M, seed=5)
    At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    Ad = At.double()
    with _ctx(prob, u.PREC_FP32) as c32:
        ref = np.zeros(prob.d + 2)
        for i in range(prob.d + 2):
            U = c32.kmv(prob.psi_true, Bt, which=i).double()
            ref[i] = float((Ad * U).sum(dim=0).cpu().numpy() @ s)
        scale = c32.dk_bilinear(prob.psi_true, At.abs(), Bt.abs(), np.abs(s))
        out32 = c32.dk_bilinear(prob.psi_true, At, Bt, s)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            c32.dk_bilinear(prob.psi_true, At, Bt, s)
        t32 = (time.perf_counter() - t0) / 3
    with _ctx(prob, u.PREC_MIXED) as cm:
        outm = cm.dk_bilinear(prob.psi_true, At, Bt, s)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            cm.dk_bilinear(prob.psi_true, At, Bt, s)
        tm = (time.perf_counter() - t0) / 3
    rel_m = np.abs(outm - ref) / scale
    rel_32 = np.abs(out32 - ref) / scale
    print("dk_bilinear n=%d M=%d: mixed max |err|/scale %.2e (fp32 pass %.2e); call time "
          "fp32 %.2f ms, mixed %.2f ms (incl. copies of A and B)"
          % (n, M, rel_m.max(), rel_32.max(), 1e3 * t32, 1e3 * tm))
    assert rel_32.max() <= 1e-5
    assert rel_m.max() <= TOL[u.PREC_MIXED]


def test_dk_bilinear_argument_errors():
    prob = w.random_problem(100, 3, seed=4)
    with _ctx(prob, u.PREC_FP32) as ctx:
        A = torch.zeros((100, 65), device="cuda")
        with pytest.raises(u.UlisseError):
            ctx.dk_bilinear(prob.psi_true, A, A)
        A = torch.zeros((100, 2), device="cuda")
        with pytest.raises(u.UlisseError):
            ctx.dk_bilinear(np.array([0.0, np.inf, 0.0, 0.0, 0.0]), A, A)
        with pytest.raises(u.UlisseError):
            ctx.dk_bilinear(prob.psi_true, A, A, scale=[1.0, np.nan])


@pytest.mark.parametrize("precision", [u.PREC_FP32, u.PREC_MIXED])
def test_grad_is_solve_plus_bilinear_form(precision):
    """ulisse_grad = the ULISSE solves of [y, probes] (Sec. 4, two estimators for y) followed
    by the bilinear forms 1/2 a1^T dK a2 - 1/(2 N_r) sum_j z_j^T dK r_j (Eq. gradient:unbiased)
    -- bit for bit, with the same step (same probes and truncation draws).  Pins the
    gradient's factor maps and scales on the FP32-storage paths (an FP64 context returns its
    estimates rounded to float, so there the two differ by that rounding)."""
    import oracle
    oracle.build()
    prob = w.census_like(n=3000, seed=4242)
    psi = prob.psi_true + 0.2
    nr, n = 8, prob.n
    X = torch.from_numpy(prob.X).cuda()
    y = torch.from_numpy(prob.y).cuda()
    cfg = u.ulisse_config_default(n_probes=nr, precision=precision, seed=91)
    with u.Context(X, y, cfg) as c:
        for step in (0, 3):
            g_api, _ = c.grad(psi, step=step)
            R = oracle.probes(n, nr, 0, 91, step).astype(np.float32)
            Bm = np.column_stack([prob.y, R]).astype(np.float32)
            S, _ = c.solve(psi, torch.from_numpy(Bm).cuda(), n_est=[2] + [1] * nr, step=step)
            S = S.cpu().numpy()
            A = np.column_stack([S[:, 0], S[:, 2:]]).astype(np.float32)
            B = np.column_stack([S[:, 1], R]).astype(np.float32)
            s = np.array([0.5] + [-0.5 / nr] * nr)
            g_man = c.dk_bilinear(psi, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), s)
            assert np.array_equal(g_api, g_man)
