"""K V launch tables (ulisse_set_tune): every configuration the autotuner may choose keeps
the K V product's parity with the FP64 oracle, tables installed from an earlier tuning give
the tuned results, and the solver run under forced tables keeps its seeded parity.

The autotuner picks, per live column count, the fastest of the compiled widths (16, 32, 64
on the tensor-core path), the two forms of the exponent's cross term (FP32 FMAs or the
tensor cores) and the j-range splits near the launch plan's; which one wins depends on
timing, so a configuration that a test run never happens to pick would otherwise go
unchecked.  Here each is forced in turn.  Tolerance: every entry within 1e-4 of its
dot-product scale sum_j |K_ij| |V_jr| (the mixed path's K V tolerance).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU runs deselect this module
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1501_05427_gb300 import ulisse as u  # noqa: E402
from paper_1501_05427_gb300 import workloads as w  # noqa: E402

TOL = 1e-4


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _ctx(prob, **cfg):
    X = torch.from_numpy(prob.X).cuda()
    y = torch.from_numpy(prob.y).cuda()
    return u.Context(X, y, u.ulisse_config_default(precision=u.PREC_MIXED, **cfg))


def _default_entry(nl):
    return {"width": 16 if nl <= 16 else 32 if nl <= 32 else 64, "rows_per_thread": 0,
            "nsplit": 0, "cross_term": 2}


def _table(nl_forced=None, entry=None, **override):
    tab = []
    for k in range(32):
        e = _default_entry(k + 1)
        e.update(override)
        if override.get("width") is not None and override["width"] < k + 1:
            e["width"] = _default_entry(k + 1)["width"]
        if nl_forced is not None and k + 1 == nl_forced:
            e = dict(entry)
        tab.append(e)
    return tab


def _check_rows(orc, prob, psi, V, U, rows):
    Xd = prob.X.astype(np.float64)
    Vd = V.astype(np.float64)
    ref = orc.kmv_rows(Xd, psi, Vd, rows)
    scale = orc.kmv_rows(Xd, psi, Vd, rows, absolute=True)
    err = np.abs(U[rows] - ref)
    return float(np.max(err / scale))


def test_every_tensor_core_configuration_keeps_parity(orc):
    prob = w.census_like(n=5_037, seed=8201)          # ragged: 158 tiles of 32 points
    n = prob.n
    rng = np.random.default_rng(5)
    rows = np.unique(np.r_[0, n - 1, rng.choice(n, 14, replace=False)])
    worst = 0.0
    with _ctx(prob, n_probes=16) as ctx:
        for nl in (1, 4, 9, 16, 17, 24, 32):
            V = rng.standard_normal((n, nl)).astype(np.float32)
            Vt = torch.from_numpy(V).cuda()
            for width in (16, 32, 64):
                if width < nl:
                    continue
                for cross in (1, 2):
                    for nsplit in (0, 1, 3, 64):
                        ctx.set_tune(_table(nl, {"width": width, "rows_per_thread": 0,
                                                 "nsplit": nsplit, "cross_term": cross}))
                        U = ctx.kmv(prob.psi_true, Vt).cpu().numpy().reshape(n, nl)
                        r = _check_rows(orc, prob, prob.psi_true, V, U, rows)
                        worst = max(worst, r)
                        assert r <= TOL, (nl, width, cross, nsplit, r)
    print("worst entry error / scale over all configurations: %.2e" % worst)


def test_installed_table_reproduces_the_tuned_context():
    prob = w.census_like(n=12_000, seed=8202)
    rng = np.random.default_rng(6)
    V = torch.from_numpy(rng.standard_normal((prob.n, 17)).astype(np.float32)).cuda()
    with _ctx(prob, n_probes=16) as ctx:
        table = ctx.autotune(prob.psi_true, 17, reps=2)
        outs = [ctx.kmv(prob.psi_true, V[:, :R].contiguous()).cpu().numpy()
                for R in (1, 9, 17)]
    with _ctx(prob, n_probes=16) as ctx2:
        ctx2.set_tune(table)
        outs2 = [ctx2.kmv(prob.psi_true, V[:, :R].contiguous()).cpu().numpy()
                 for R in (1, 9, 17)]
    for a, b in zip(outs, outs2):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("override", [{"cross_term": 1}, {"cross_term": 2, "nsplit": 3},
                                      {"width": 64, "cross_term": 2, "nsplit": 1},
                                      {"width": 32, "cross_term": 1, "nsplit": 64}])
def test_forced_tables_keep_solve_parity(orc, override):
    """The solver applies K V to the live columns only (compacted column maps); under each
    forced table the seeded solve matches the oracle as in the default configuration."""
    n, R = 1500, 9
    prob = w.census_like(n=n, seed=300 + n)
    rng = np.random.default_rng(n)
    B = rng.choice([-1.0, 1.0], (n, R)).astype(np.float32)
    B[:, 0] = prob.y
    n_est = np.ones(R, np.int32)
    n_est[0] = 2
    Sref, st_ref = orc.ulisse_solve(prob.X.astype(np.float64), prob.psi_true,
                                    B.astype(np.float64), n_est=n_est, q=1.0, beta=1.0,
                                    eps=1e-8, max_iter=500, seed=21, step=4)
    with _ctx(prob, q=1.0, max_iter=500, seed=21) as ctx:
        ctx.set_tune(_table(**override))
        S, st = ctx.solve(prob.psi_true, torch.from_numpy(B).cuda(), n_est=n_est, step=4)
    S = S.cpu().numpy().astype(np.float64)
    assert all(tuple(st[c][:4]) == tuple(int(v) for v in st_ref[c, :4]) for c in range(R))
    errs = [float(np.linalg.norm(S[:, k] - Sref[:, k]) / np.linalg.norm(Sref[:, k]))
            for k in range(Sref.shape[1])]
    print("forced table %s: max solve rel. error %.2e" % (override, max(errs)))
    assert max(errs) <= TOL


def test_set_tune_rejects_invalid_entries():
    prob = w.census_like(n=2000, seed=8203)
    with _ctx(prob, n_probes=4) as ctx:
        for bad in ({"width": 0}, {"width": 65}, {"cross_term": 0}, {"nsplit": -1},
                    {"nsplit": 65}):
            e = _default_entry(1)
            e.update(bad)
            with pytest.raises(u.UlisseError):
                ctx.set_tune([e])
        with pytest.raises(u.UlisseError):       # entry 1 serves two columns
            ctx.set_tune([_default_entry(1), dict(_default_entry(2), width=1)])
        with pytest.raises(u.UlisseError):
            ctx.set_tune([_default_entry(k + 1) for k in range(33)])
        ctx.set_tune([])            # clearing is allowed
