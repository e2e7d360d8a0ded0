"""Large inputs: n = 2^20 + 1 points (a ragged last tile; n^2 ~ 1.1e12 generated entries per
product, far beyond 32-bit counts).  K V of the FP32 and mixed paths on sampled rows against
the oracle (which evaluates those rows one by one), at the paths' tolerances: every entry
within 1e-5 (FP32) or 1e-4 (mixed) of its dot-product scale sum_j |K_ij| |V_jr|.  At n = 2^19 + 1
the tensor-core gradient pass is checked against the derivative products of the SIMT path
(a property that holds at any size)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU runs deselect this module
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1501_05427_gb300 import ulisse as u  # noqa: E402
from paper_1501_05427_gb300 import workloads as w  # noqa: E402

N = (1 << 20) + 1


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="module")
def prob():
    return w.random_problem(N, 8, seed=77, lengthscale=0.8, dist="normal")


@pytest.mark.parametrize("precision,tol", [(u.PREC_FP32, 1e-5), (u.PREC_MIXED, 1e-4)])
def test_large_n_kmv_sampled_rows(orc, prob, precision, tol):
    rng = np.random.default_rng(3)
    R = 5
    V = rng.standard_normal((N, R)).astype(np.float32)
    X = torch.from_numpy(prob.X).cuda()
    y = torch.from_numpy(prob.y).cuda()
    with u.Context(X, y, u.ulisse_config_default(precision=precision, n_probes=4)) as ctx:
        U = ctx.kmv(prob.psi_true, torch.from_numpy(V).cuda()).cpu().numpy()
    rows = np.unique(np.r_[0, 1, N - 2, N - 1, rng.choice(N, 12, replace=False)])
    Xd, Vd = prob.X.astype(np.float64), V.astype(np.float64)
    ref = orc.kmv_rows(Xd, prob.psi_true, Vd, rows)
    scale = orc.kmv_rows(Xd, prob.psi_true, Vd, rows, absolute=True)
    err = np.abs(U[rows].astype(np.float64) - ref)
    print("n = %d, precision %d: worst entry error / scale %.2e"
          % (N, precision, float(np.max(err / scale))))
    assert np.all(err <= tol * scale)


def test_large_n_gradient_pass_matches_derivative_products():
    """The tensor-core gradient pass (each unordered pair once, 2M factor slots) against the
    derivative products of the SIMT path at n = 2^19 + 1: for random A, B,
        out_i = sum_m a_m^T dK/dpsi_i b_m   must equal   sum_m a_m . (dK/dpsi_i b_m),
    every dK/dpsi_i here being entrywise non-negative (sigma^2 and lengthscale derivatives of
    the squared exponential, lambda I), so |a|^T dK |b| bounds the sum's rounding; tolerance
    1e-4 of that scale (the mixed path's bound)."""
    n = (1 << 19) + 1
    p = w.random_problem(n, 8, seed=78, lengthscale=0.8, dist="normal")
    rng = np.random.default_rng(4)
    M = 2
    A = rng.standard_normal((n, M)).astype(np.float32)
    B = rng.standard_normal((n, M)).astype(np.float32)
    X = torch.from_numpy(p.X).cuda()
    y = torch.from_numpy(p.y).cuda()
    At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    Ab, Bb = torch.from_numpy(np.abs(A)).cuda(), torch.from_numpy(np.abs(B)).cuda()
    with u.Context(X, y, u.ulisse_config_default(precision=u.PREC_MIXED, n_probes=4)) as ctx:
        out = ctx.dk_bilinear(p.psi_true, At, Bt)
        ref, scale = [], []
        for i in range(p.d + 2):
            KB = ctx.kmv(p.psi_true, Bt, which=i).double()
            KBa = ctx.kmv(p.psi_true, Bb, which=i).double()
            ref.append(float(torch.sum(At.double() * KB)))
            scale.append(float(torch.sum(Ab.double() * KBa)))
    ref, scale = np.array(ref), np.array(scale)
    r = np.abs(out - ref) / scale
    print("n = %d gradient pass vs derivative products: worst error / scale %.2e" % (n, r.max()))
    assert np.all(r <= 1e-4), (out, ref, scale)
