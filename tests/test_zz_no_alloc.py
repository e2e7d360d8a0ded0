"""The allocation-free K V entry point (ulisse_kmv_noalloc) against the context-based one.

Some callers cannot allocate device memory; ulisse_kmv_noalloc serves them from a static
device array.  This file is collected last so that a run stopping at the first failure has
already run every other test.  It checks two calls in a row (a large ragged problem, then a
smaller one with fewer right-hand sides and a derivative) so that state the first call leaves
in the shared array cannot leak into the second.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU runs deselect this module
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1501_05427_gb300 import ulisse as u  # noqa: E402
from paper_1501_05427_gb300 import workloads as w  # noqa: E402

TOL = 1e-5   # the K V parity tolerance used for the context-based entry point


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _noalloc(lib, X, psi, which, V):
    n, d = X.shape
    R = V.shape[1]
    Vc = V.t().contiguous()           # column-major n x R
    U = torch.full((R, n), float("nan"), device="cuda")
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    st = lib.ulisse_kmv_noalloc(ctypes.c_void_p(X.data_ptr()), n, d,
                                psi.ctypes.data_as(ctypes.c_void_p), which,
                                ctypes.c_void_p(Vc.data_ptr()), R, ctypes.c_void_p(U.data_ptr()),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == u.ULISSE_OK
    torch.cuda.synchronize()
    return U.t()


def _reference(prob, X, y, which, V):
    with u.Context(X, y, u.ulisse_config_default()) as ctx:
        return ctx.kmv(prob.psi_true, V, which)


def _close(a, b):
    a = a.double()
    b = b.double()
    scale = b.abs().max().item()
    assert torch.isfinite(a).all()
    assert (a - b).abs().max().item() <= TOL * scale
    assert torch.linalg.norm(a - b).item() <= TOL * torch.linalg.norm(b).item()


def test_noalloc_matches_context_entry_point_twice(orc):
    lib = u.load()
    cases = [
        (w.census_like(n=9_937, d=8, seed=3), -1, 17),   # ragged n, many right-hand sides
        (w.random_problem(1_037, 3, seed=4), 3, 5),       # smaller n, dK/dlog sigma^2
    ]
    for prob, which, R in cases:
        X = torch.from_numpy(prob.X).cuda()
        y = torch.from_numpy(prob.y).cuda()
        V = torch.randn((prob.n, R), device="cuda")
        got = _noalloc(lib, X, prob.psi_true, which, V)
        assert u.ulisse_kmv_noalloc_status() == 0
        ref = _reference(prob, X, y, which, V)
        _close(got, ref)
        # and on its own against the oracle, row by row (FP64, rows evaluated one by one)
        rows = np.unique(np.r_[0, prob.n - 1, np.random.default_rng(9).integers(0, prob.n, 14)])
        Vd = V.double().cpu().numpy()
        want = orc.kmv_rows(prob.X.astype(np.float64), prob.psi_true, Vd, rows, which)
        scale = orc.kmv_rows(prob.X.astype(np.float64), prob.psi_true, Vd, rows, which,
                             absolute=True)
        err = np.abs(got.double().cpu().numpy()[rows] - want)
        assert np.all(err <= TOL * np.maximum(scale, 1e-30))


def test_noalloc_rejects_oversized_requests():
    lib = u.load()
    X = torch.zeros((4, 2), device="cuda")
    V = torch.zeros((32, 4), device="cuda")
    psi = np.zeros(4)
    bad_R = lib.ulisse_kmv_noalloc(ctypes.c_void_p(X.data_ptr()), 4, 2,
                                   psi.ctypes.data_as(ctypes.c_void_p), -1,
                                   ctypes.c_void_p(V.data_ptr()), 33,
                                   ctypes.c_void_p(V.data_ptr()), None)
    assert bad_R == u.ULISSE_ERR_ARG
    too_big = lib.ulisse_kmv_noalloc(ctypes.c_void_p(X.data_ptr()), 10_000_000, 2,
                                     psi.ctypes.data_as(ctypes.c_void_p), -1,
                                     ctypes.c_void_p(V.data_ptr()), 1,
                                     ctypes.c_void_p(V.data_ptr()), None)
    assert too_big == u.ULISSE_ERR_ARG


def test_noalloc_timing_against_context_entry_point():
    """Times the two entry points with CUDA events at the test sizes (FP32 context path).
    The allocation-free call plans its j-range split for the SMs whose partial sums fit
    the static array, so it can be slower than the context path; this test prints both
    times and only checks that the call completes."""
    lib = u.load()
    for n, R in ((9_937, 17), (50_000, 17)):
        prob = w.census_like(n=n, d=8, seed=5)
        X = torch.from_numpy(prob.X).cuda()
        y = torch.from_numpy(prob.y).cuda()
        V = torch.randn((n, R), device="cuda")
        Vc = V.t().contiguous()
        U = torch.empty((R, n), device="cuda")
        psi = np.ascontiguousarray(prob.psi_true, dtype=np.float64)
        stream = torch.cuda.current_stream()

        def na():
            st = lib.ulisse_kmv_noalloc(ctypes.c_void_p(X.data_ptr()), n, 8,
                                        psi.ctypes.data_as(ctypes.c_void_p), -1,
                                        ctypes.c_void_p(Vc.data_ptr()), R,
                                        ctypes.c_void_p(U.data_ptr()),
                                        ctypes.c_void_p(stream.cuda_stream))
            assert st == u.ULISSE_OK

        def timed(fn, reps=5):
            fn()
            ts = []
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                b.synchronize()
                ts.append(a.elapsed_time(b))
            return sorted(ts)[len(ts) // 2]

        t_na = timed(na)
        assert u.ulisse_kmv_noalloc_status() == 0
        with u.Context(X, y, u.ulisse_config_default()) as ctx:
            Ucx = torch.empty((R, n), device="cuda").t()
            t_cx = timed(lambda: ctx.kmv(prob.psi_true, V, out=Ucx))
        print("K V n=%d R=%d: allocation-free %.3f ms, context %.3f ms" % (n, R, t_na, t_cx))
