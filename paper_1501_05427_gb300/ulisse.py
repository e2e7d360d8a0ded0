"""Thin Python binding of libulisse (include/ulisse.h).

Argument marshalling only: every step of the method runs in the library's CUDA kernels.
PyTorch provides device memory and the stream.  Blocks of vectors are passed as (n, R)
tensors stored column-major (``t.T.is_contiguous()``); other layouts are copied once into
that layout.  The library is loaded from ``paper_1501_05427_gb300/_build/libulisse.so``;
if it is missing, ``load()`` raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libulisse.so")

ULISSE_OK = 0
ULISSE_ERR_ARG = 1
ULISSE_ERR_CUDA = 2
ULISSE_ERR_BREAKDOWN = 3
ULISSE_ERR_MAXITER = 4
ULISSE_ERR_NOMEM = 5
ULISSE_ERR_TIMEOUT = 6

PREC_FP32, PREC_MIXED, PREC_FP64 = 0, 1, 2
PROBE_RADEMACHER, PROBE_GAUSSIAN = 0, 1

EXPORTED = [
    "ulisse_config_default", "ulisse_create", "ulisse_create_host", "ulisse_kmv",
    "ulisse_kmv_f64", "ulisse_solve", "ulisse_grad", "ulisse_sgld_step", "ulisse_sgld_chain",
    "ulisse_counters", "ulisse_profile_enable", "ulisse_profile_read", "ulisse_last_error",
    "ulisse_destroy", "ulisse_kmv_noalloc", "ulisse_kmv_noalloc_status", "ulisse_ws_init", "ulisse_ws_set", "ulisse_ws_train",
    "ulisse_ws_loss_grad", "ulisse_ws_export", "ulisse_ws_x0", "ulisse_create_batched",
    "ulisse_batch_size", "ulisse_batch_kmv", "ulisse_batch_grad", "ulisse_batch_sgld_step",
    "ulisse_set_graph", "ulisse_autotune", "ulisse_set_tune", "ulisse_batch_sgld_chain", "ulisse_dk_bilinear",
    "ulisse_selftest_wait_timeout", "ulisse_measure_ex2_rate", "ulisse_predict",
]


class ulisse_config(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("n_probes", ctypes.c_int),
        ("probe_kind", ctypes.c_int),
        ("probe_refresh", ctypes.c_int),
        ("warm_start_probes", ctypes.c_int),
        ("q", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("max_iter", ctypes.c_int),
        ("seed", ctypes.c_ulonglong),
        ("kmv_rows_per_thread", ctypes.c_int),
        ("tc_cross_term", ctypes.c_int),
        ("pcg_delta", ctypes.c_double),
        ("pcg_inner_tol", ctypes.c_double),
        ("pcg_inner_max", ctypes.c_int),
    ]


class ulisse_col_stats(ctypes.Structure):
    _fields_ = [("l", ctypes.c_int), ("iterations", ctypes.c_int), ("outcome", ctypes.c_int),
                ("J0", ctypes.c_int), ("J1", ctypes.c_int)]


class ulisse_profile(ctypes.Structure):
    _fields_ = [("kmv_launches", ctypes.c_longlong), ("kmv_ms", ctypes.c_double),
                ("kmv_flop", ctypes.c_double), ("grad_launches", ctypes.c_longlong),
                ("grad_ms", ctypes.c_double), ("grad_flop", ctypes.c_double)]


class ulisse_ws_config(ctypes.Structure):
    _fields_ = [("n_anchors", ctypes.c_int), ("hidden", ctypes.c_int), ("n_rows", ctypes.c_int),
                ("max_pairs", ctypes.c_int), ("seed", ctypes.c_ulonglong),
                ("ridge", ctypes.c_double)]


class ulisse_ws_state(ctypes.Structure):
    _fields_ = [("weights", ctypes.c_void_p), ("anchors", ctypes.c_void_p),
                ("pair_rows", ctypes.c_void_p), ("mu", ctypes.c_void_p), ("sd", ctypes.c_void_p),
                ("pair_psi", ctypes.c_void_p), ("n_pairs", ctypes.c_int),
                ("n_params", ctypes.c_longlong)]


class ulisse_tune_entry(ctypes.Structure):
    _fields_ = [("live_cols", ctypes.c_int), ("width", ctypes.c_int),
                ("rows_per_thread", ctypes.c_int), ("nsplit", ctypes.c_int),
                ("ms", ctypes.c_float), ("ms_default", ctypes.c_float),
                ("cross_term", ctypes.c_int)]


class UlisseError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("ulisse status %d: %s" % (status, msg))
        self.status = status


_lib = None


def load():
    """Load libulisse.so (built by ``paper_1501_05427_gb300.build``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libulisse.so not built: run __graft_entry__.build() "
                           "(or python -m paper_1501_05427_gb300.build)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, LL, U64 = (ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong,
                        ctypes.c_ulonglong)
    PP = ctypes.POINTER(ctypes.c_void_p)
    cfgp = ctypes.POINTER(ulisse_config)
    sp = ctypes.POINTER(ulisse_col_stats)
    lib.ulisse_config_default.argtypes = [cfgp]
    lib.ulisse_config_default.restype = None
    lib.ulisse_create.argtypes = [PP, P, P, LL, I, cfgp, P]
    lib.ulisse_create_host.argtypes = [PP, P, P, LL, I, cfgp, P]
    lib.ulisse_kmv.argtypes = [P, P, I, P, I, P]
    lib.ulisse_kmv_f64.argtypes = [P, P, I, P, I, P]
    lib.ulisse_solve.argtypes = [P, P, P, I, P, P, P, U64, sp]
    lib.ulisse_grad.argtypes = [P, P, U64, P, sp]
    lib.ulisse_dk_bilinear.argtypes = [P, P, P, P, I, P, P]
    lib.ulisse_selftest_wait_timeout.argtypes = [P]
    lib.ulisse_measure_ex2_rate.argtypes = [P, I, ctypes.POINTER(D), ctypes.POINTER(D)]
    lib.ulisse_predict.argtypes = [P, P, P, LL, U64, P, P]
    lib.ulisse_sgld_step.argtypes = [P, P, D, P, P, U64, P]
    lib.ulisse_sgld_chain.argtypes = [P, P, P, I, P, P, U64, P]
    lib.ulisse_counters.argtypes = [P, ctypes.POINTER(LL), ctypes.POINTER(D), ctypes.POINTER(LL)]
    lib.ulisse_profile_enable.argtypes = [P, I]
    lib.ulisse_profile_read.argtypes = [P, ctypes.POINTER(ulisse_profile), I]
    lib.ulisse_kmv_noalloc.argtypes = [P, LL, I, P, I, P, I, P, P]
    lib.ulisse_kmv_noalloc_status.argtypes = [P, ctypes.POINTER(ctypes.c_int)]
    lib.ulisse_ws_init.argtypes = [P, ctypes.POINTER(ulisse_ws_config)]
    lib.ulisse_ws_set.argtypes = [P, I, I]
    lib.ulisse_ws_train.argtypes = [P, I, I, D, ctypes.POINTER(D)]
    lib.ulisse_ws_loss_grad.argtypes = [P, ctypes.POINTER(D), P]
    lib.ulisse_ws_export.argtypes = [P, ctypes.POINTER(ulisse_ws_state)]
    lib.ulisse_ws_x0.argtypes = [P, P, I, P]
    lib.ulisse_create_batched.argtypes = [PP, I, P, P, P, P, cfgp, P]
    lib.ulisse_batch_size.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I)]
    lib.ulisse_batch_kmv.argtypes = [P, P, P, I, P]
    lib.ulisse_batch_grad.argtypes = [P, P, U64, P, sp]
    lib.ulisse_batch_sgld_step.argtypes = [P, P, D, U64, P]
    lib.ulisse_batch_sgld_chain.argtypes = [P, P, P, I, U64, P]
    lib.ulisse_set_graph.argtypes = [P, I]
    lib.ulisse_autotune.argtypes = [P, P, I, I, ctypes.POINTER(ulisse_tune_entry)]
    lib.ulisse_set_tune.argtypes = [P, ctypes.POINTER(ulisse_tune_entry), I]
    lib.ulisse_last_error.argtypes = [P]
    lib.ulisse_last_error.restype = ctypes.c_char_p
    lib.ulisse_destroy.argtypes = [P]
    lib.ulisse_destroy.restype = None
    for name in EXPORTED:
        f = getattr(lib, name)
        if name not in ("ulisse_config_default", "ulisse_last_error", "ulisse_destroy"):
            f.restype = ctypes.c_int
    _lib = lib
    return lib


def ulisse_config_default(**overrides) -> ulisse_config:
    cfg = ulisse_config()
    load().ulisse_config_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def _f64_host(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.size == n
    return a


def _hptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _colmajor(t):
    """(n,) or (n, R) CUDA tensor -> (n, R) column-major tensor (copy only if needed)."""
    if t.dim() == 1:
        t = t[:, None]
    if not t.t().is_contiguous():
        t = t.t().contiguous().t()
    return t


class Context:
    """One GP regression problem on the current CUDA device (ulisse_create)."""

    def __init__(self, X, y, cfg: ulisse_config | None = None, stream=None, host=False):
        import torch
        self._lib = load()
        cfg = cfg or ulisse_config_default()
        self.cfg = cfg
        if host:
            Xh = np.ascontiguousarray(X, dtype=np.float32)
            yh = np.ascontiguousarray(y, dtype=np.float32)
            n, d = Xh.shape
            self._keep = (Xh, yh)
            xp, yp = _hptr(Xh), _hptr(yh)
        else:
            X = X.contiguous().float()
            y = y.contiguous().float()
            n, d = X.shape
            self._keep = (X, y)
            xp, yp = ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(y.data_ptr())
        self.n, self.d, self.p = n, d, d + 2
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        fn = self._lib.ulisse_create_host if host else self._lib.ulisse_create
        st = fn(ctypes.byref(h), xp, yp, n, d, ctypes.byref(cfg),
                ctypes.c_void_p(self.stream.cuda_stream))
        if st != ULISSE_OK:
            raise UlisseError(st, self._lib.ulisse_last_error(None).decode())
        self._h = h

    # -- helpers ---------------------------------------------------------------------
    def _check(self, st, allow=()):
        if st != ULISSE_OK and st not in allow:
            raise UlisseError(st, self._lib.ulisse_last_error(self._h).decode())
        return st

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ulisse_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- API ---------------------------------------------------------------------------
    def kmv(self, psi, V, which=-1, out=None):
        """U = K V (which=-1) or dK/dpsi_which V.  V: (n,) or (n, R) CUDA tensor."""
        import torch
        f64 = V.dtype == torch.float64
        Vc = _colmajor(V)
        R = Vc.shape[1]
        if out is None:
            out = torch.empty((R, self.n), dtype=V.dtype, device=V.device).t()
        psi = _f64_host(psi, self.p)
        fn = self._lib.ulisse_kmv_f64 if f64 else self._lib.ulisse_kmv
        self._check(fn(self._h, _hptr(psi), which, ctypes.c_void_p(Vc.data_ptr()), R,
                       ctypes.c_void_p(out.data_ptr())))
        return out[:, 0] if V.dim() == 1 else out

    def solve(self, psi, B, n_est=None, S0=None, step=0, allow=()):
        """ULISSE estimates of K^{-1} B.  Returns (S_est (n, sum n_est), stats list)."""
        import torch
        Bc = _colmajor(B.float())
        R = Bc.shape[1]
        ne = np.ascontiguousarray(n_est if n_est is not None else np.ones(R), dtype=np.int32)
        tot = int(ne.sum())
        S_est = torch.empty((tot, self.n), dtype=torch.float32, device=B.device).t()
        S0c = _colmajor(S0.float()) if S0 is not None else None
        stats = (ulisse_col_stats * R)()
        psi = _f64_host(psi, self.p)
        st = self._lib.ulisse_solve(self._h, _hptr(psi), ctypes.c_void_p(Bc.data_ptr()), R,
                                    _hptr(ne), ctypes.c_void_p(S0c.data_ptr()) if S0c is not None
                                    else None, ctypes.c_void_p(S_est.data_ptr()), step, stats)
        self._check(st, allow)
        return S_est, [(s.l, s.iterations, s.outcome, s.J0, s.J1) for s in stats]

    def grad(self, psi, step=0, allow=()):
        """Unbiased gradient estimate (host numpy, p) and per-column stats."""
        psi = _f64_host(psi, self.p)
        g = np.zeros(self.p)
        R = 1 + self.cfg.n_probes
        stats = (ulisse_col_stats * R)()
        st = self._lib.ulisse_grad(self._h, _hptr(psi), step, _hptr(g), stats)
        self._check(st, allow)
        return g, [(s.l, s.iterations, s.outcome, s.J0, s.J1) for s in stats]

    def dk_bilinear(self, psi, A, B, scale=None):
        """out_i = sum_m scale_m a_m^T dK/dpsi_i b_m for every parameter (host numpy, p).
        A, B: (n, M) CUDA tensors."""
        Ac = _colmajor(A.float())
        Bc = _colmajor(B.float())
        if Ac.shape != Bc.shape or Ac.shape[0] != self.n:
            raise ValueError("A and B must both be (n, M)")
        M = Ac.shape[1]
        sc = np.ascontiguousarray(scale, dtype=np.float64) if scale is not None else None
        if sc is not None and sc.shape != (M,):
            raise ValueError("scale must have M entries")
        psi = _f64_host(psi, self.p)
        out = np.zeros(self.p)
        self._check(self._lib.ulisse_dk_bilinear(self._h, _hptr(psi), ctypes.c_void_p(Ac.data_ptr()),
                                                 ctypes.c_void_p(Bc.data_ptr()), M, _hptr(sc),
                                                 _hptr(out)))
        return out

    def predict(self, psi, Xs, step=0, var=True, allow=()):
        """Posterior predictive at psi for the test inputs Xs ((m, d) CUDA tensor): returns
        (mean, var) as CUDA tensors of m floats (var None when not requested)."""
        import torch
        Xs = Xs.contiguous().float()
        m = Xs.shape[0]
        if Xs.dim() != 2 or Xs.shape[1] != self.d:
            raise ValueError("Xs must be (m, d)")
        mean = torch.empty(m, dtype=torch.float32, device=Xs.device)
        v = torch.empty(m, dtype=torch.float32, device=Xs.device) if var else None
        psi = _f64_host(psi, self.p)
        self._check(self._lib.ulisse_predict(self._h, _hptr(psi), ctypes.c_void_p(Xs.data_ptr()), m,
                                             step, ctypes.c_void_p(mean.data_ptr()),
                                             ctypes.c_void_p(v.data_ptr()) if var else None),
                    allow)
        return mean, v

    def sgld_step(self, psi, eps_t, step, M=None, prior_grad=None, allow=()):
        """One SGLD step; returns (psi_new, g) as numpy arrays."""
        psi = np.array(psi, dtype=np.float64, copy=True)
        g = np.zeros(self.p)
        Mh = np.ascontiguousarray(M, dtype=np.float64) if M is not None else None
        ph = _f64_host(prior_grad, self.p) if prior_grad is not None else None
        st = self._lib.ulisse_sgld_step(self._h, _hptr(psi), float(eps_t), _hptr(Mh), _hptr(ph),
                                        step, _hptr(g))
        self._check(st, allow)
        return psi, g

    def sgld_chain(self, psi_dev, eps_dev, step0=0, M=None, prior_grad=None, trace_dev=None,
                   allow=()):
        """len(eps_dev) SGLD steps with psi resident on the device (in place)."""
        Mh = np.ascontiguousarray(M, dtype=np.float64) if M is not None else None
        ph = _f64_host(prior_grad, self.p) if prior_grad is not None else None
        st = self._lib.ulisse_sgld_chain(
            self._h, ctypes.c_void_p(psi_dev.data_ptr()), ctypes.c_void_p(eps_dev.data_ptr()),
            int(eps_dev.numel()), _hptr(Mh), _hptr(ph), step0,
            ctypes.c_void_p(trace_dev.data_ptr()) if trace_dev is not None else None)
        self._check(st, allow)
        return psi_dev

    # -- learned warm start --------------------------------------------------------------
    def ws_init(self, n_anchors=512, hidden=256, n_rows=1024, max_pairs=256, seed=0,
                ridge=1e-2):
        cfg = ulisse_ws_config(n_anchors, hidden, n_rows, max_pairs, seed, ridge)
        self._check(self._lib.ulisse_ws_init(self._h, ctypes.byref(cfg)))
        self.ws_cfg = cfg

    def ws_set(self, record=False, use=False):
        self._check(self._lib.ulisse_ws_set(self._h, int(bool(record)), int(bool(use))))

    def ws_train(self, steps, batch=64, lr=1e-3):
        loss = ctypes.c_double()
        self._check(self._lib.ulisse_ws_train(self._h, steps, batch, lr, ctypes.byref(loss)))
        return loss.value

    def ws_loss_grad(self):
        st = self.ws_export()
        g = np.zeros(st["n_params"], dtype=np.float32)
        loss = ctypes.c_double()
        self._check(self._lib.ulisse_ws_loss_grad(self._h, ctypes.byref(loss), _hptr(g)))
        return loss.value, g

    def ws_export(self):
        cfg = self.ws_cfg
        p, H, A, m, P = self.p, cfg.hidden, cfg.n_anchors, cfg.n_rows, cfg.max_pairs
        npar = p * H + H + H * H + H + H * A + A
        out = dict(weights=np.zeros(npar, np.float32), anchors=np.zeros(A, np.int32),
                   pair_rows=np.zeros((P, m), np.int32), mu=np.zeros(p, np.float32),
                   sd=np.zeros(p, np.float32), pair_psi=np.zeros((P, p), np.float32))
        st = ulisse_ws_state(*[_hptr(out[k]) for k in ("weights", "anchors", "pair_rows", "mu",
                                                       "sd", "pair_psi")], 0, 0)
        self._check(self._lib.ulisse_ws_export(self._h, ctypes.byref(st)))
        out["n_pairs"] = st.n_pairs
        out["n_params"] = st.n_params
        return out

    def ws_x0(self, psi, bf16=False):
        import torch
        x0 = torch.empty(self.n, dtype=torch.float32, device="cuda")
        psi = _f64_host(psi, self.p)
        self._check(self._lib.ulisse_ws_x0(self._h, _hptr(psi), int(bool(bf16)),
                                           ctypes.c_void_p(x0.data_ptr())))
        return x0

    def autotune(self, psi, max_cols=None, reps=3):
        """Tune the K V launch configuration for 1..max_cols live columns; returns the table
        as a list of dicts."""
        max_cols = max_cols or (1 + self.cfg.n_probes)
        out = (ulisse_tune_entry * max_cols)()
        psi = _f64_host(psi, self.p)
        self._check(self._lib.ulisse_autotune(self._h, _hptr(psi), max_cols, reps, out))
        return [{k: getattr(e, k) for k, _ in ulisse_tune_entry._fields_} for e in out]

    def set_tune(self, table):
        """Install a K V launch table (a list of dicts as autotune returns, entry k for k + 1
        columns); an empty list clears it."""
        arr = (ulisse_tune_entry * max(1, len(table)))()
        for k, e in enumerate(table):
            arr[k] = ulisse_tune_entry(k + 1, e["width"], e["rows_per_thread"], e["nsplit"],
                                       e.get("ms", 0.0), e.get("ms_default", 0.0),
                                       e["cross_term"])
        self._check(self._lib.ulisse_set_tune(self._h, arr, len(table)))

    def selftest_wait_timeout(self):
        """Run the failure-path self-test; returns the status code (ULISSE_ERR_TIMEOUT)."""
        return self._lib.ulisse_selftest_wait_timeout(self._h)

    def set_graph(self, enable=True):
        """sgld_chain: one CUDA-graph launch per step (True) or the host loop (False)."""
        self._check(self._lib.ulisse_set_graph(self._h, int(bool(enable))))

    def counters(self):
        """(K V rounds, generated entries x right-hand sides, kernel launches) so far."""
        a = ctypes.c_longlong()
        b = ctypes.c_double()
        c = ctypes.c_longlong()
        self._lib.ulisse_counters(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
        return a.value, b.value, c.value

    def profile_enable(self, enable=True):
        self._check(self._lib.ulisse_profile_enable(self._h, 1 if enable else 0))

    def profile_read(self, reset=False):
        """Event-timed totals of the K V and gradient kernels since enabling (a dict)."""
        pr = ulisse_profile()
        self._check(self._lib.ulisse_profile_read(self._h, ctypes.byref(pr), 1 if reset else 0))
        return {k: getattr(pr, k) for k, _ in ulisse_profile._fields_}


# Same names as the C ABI, for callers that prefer functions over the class.
def ulisse_create(X, y, cfg=None, stream=None):
    return Context(X, y, cfg, stream)


def ulisse_create_host(X, y, cfg=None, stream=None):
    return Context(X, y, cfg, stream, host=True)


def ulisse_kmv(ctx: Context, psi, which, V):
    return ctx.kmv(psi, V, which)


ulisse_kmv_f64 = ulisse_kmv


def ulisse_solve(ctx: Context, psi, B, n_est=None, S0=None, step=0):
    return ctx.solve(psi, B, n_est, S0, step)


def ulisse_grad(ctx: Context, psi, step=0):
    return ctx.grad(psi, step)


def ulisse_dk_bilinear(ctx: Context, psi, A, B, scale=None):
    return ctx.dk_bilinear(psi, A, B, scale)


def ulisse_sgld_step(ctx: Context, psi, eps_t, step, M=None, prior_grad=None):
    return ctx.sgld_step(psi, eps_t, step, M, prior_grad)


def ulisse_sgld_chain(ctx: Context, psi_dev, eps_dev, step0=0, M=None, prior_grad=None,
                      trace_dev=None):
    return ctx.sgld_chain(psi_dev, eps_dev, step0, M, prior_grad, trace_dev)


def ulisse_counters(ctx: Context):
    return ctx.counters()


def ulisse_profile_enable(ctx: Context, enable=True):
    ctx.profile_enable(enable)


def ulisse_profile_read(ctx: Context, reset=False):
    return ctx.profile_read(reset)


class BatchContext:
    """Many independent GP problems advanced together (ulisse_create_batched).

    Parameters and gradients are packed: problem b's d_b + 2 values follow problem b-1's.
    Problem b draws from the random streams of seed cfg.seed + b."""

    def __init__(self, Xs, ys, cfg: ulisse_config | None = None, stream=None):
        import torch
        self._lib = load()
        cfg = cfg or ulisse_config_default()
        self.cfg = cfg
        self._keep = [(X.contiguous().float(), y.contiguous().float()) for X, y in zip(Xs, ys)]
        B = len(self._keep)
        self.ns = [int(X.shape[0]) for X, _ in self._keep]
        self.ds = [int(X.shape[1]) for X, _ in self._keep]
        self.ps = [d + 2 for d in self.ds]
        self.p_off = np.concatenate([[0], np.cumsum(self.ps)[:-1]]).astype(int)
        self.n_params = int(sum(self.ps))
        n_arr = np.array(self.ns, dtype=np.int64)
        d_arr = np.array(self.ds, dtype=np.int32)
        xp = (ctypes.c_void_p * B)(*[X.data_ptr() for X, _ in self._keep])
        yp = (ctypes.c_void_p * B)(*[y.data_ptr() for _, y in self._keep])
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        st = self._lib.ulisse_create_batched(ctypes.byref(h), B, _hptr(n_arr), _hptr(d_arr),
                                             ctypes.cast(xp, ctypes.c_void_p),
                                             ctypes.cast(yp, ctypes.c_void_p), ctypes.byref(cfg),
                                             ctypes.c_void_p(self.stream.cuda_stream))
        if st != ULISSE_OK:
            raise UlisseError(st, self._lib.ulisse_last_error(None).decode())
        self._h = h
        self.n_problems = B

    _check = Context._check
    close = Context.close
    __del__ = Context.__del__
    __enter__ = Context.__enter__
    __exit__ = Context.__exit__

    def split(self, packed):
        """Packed vector -> list of per-problem arrays."""
        return [np.asarray(packed)[o:o + p] for o, p in zip(self.p_off, self.ps)]

    def kmv(self, psi, Vs):
        """U_b = K_b V_b for all problems.  Vs: list of (n_b, R) CUDA tensors (same R)."""
        import torch
        Vc = [_colmajor(V.float()) for V in Vs]
        R = Vc[0].shape[1]
        Us = [torch.empty((R, n), dtype=torch.float32, device=V.device).t()
              for V, n in zip(Vc, self.ns)]
        vp = (ctypes.c_void_p * self.n_problems)(*[V.data_ptr() for V in Vc])
        up = (ctypes.c_void_p * self.n_problems)(*[U.data_ptr() for U in Us])
        psi = _f64_host(psi, self.n_params)
        self._check(self._lib.ulisse_batch_kmv(self._h, _hptr(psi), ctypes.cast(vp, ctypes.c_void_p),
                                               R, ctypes.cast(up, ctypes.c_void_p)))
        return Us

    def grad(self, psi, step=0, allow=()):
        """Packed gradient estimates (host numpy) and per-problem column stats."""
        psi = _f64_host(psi, self.n_params)
        g = np.zeros(self.n_params)
        R = 1 + self.cfg.n_probes
        stats = (ulisse_col_stats * (R * self.n_problems))()
        self._check(self._lib.ulisse_batch_grad(self._h, _hptr(psi), step, _hptr(g), stats), allow)
        st = [(s.l, s.iterations, s.outcome, s.J0, s.J1) for s in stats]
        return g, [st[b * R:(b + 1) * R] for b in range(self.n_problems)]

    def sgld_step(self, psi, eps_t, step, allow=()):
        """One SGLD step of every problem; returns (psi_new, g), packed."""
        psi = np.array(psi, dtype=np.float64, copy=True)
        assert psi.size == self.n_params
        g = np.zeros(self.n_params)
        self._check(self._lib.ulisse_batch_sgld_step(self._h, _hptr(psi), eps_t, step, _hptr(g)),
                    allow)
        return psi, g

    counters = Context.counters
    set_graph = Context.set_graph

    def sgld_chain_status(self, psi_dev, eps_dev, step0=0, trace_dev=None):
        """As sgld_chain; returns the status instead of raising on ULISSE_ERR_MAXITER."""
        return self.sgld_chain(psi_dev, eps_dev, step0, trace_dev, allow=(ULISSE_ERR_MAXITER,),
                               status=True)

    def sgld_chain(self, psi_dev, eps_dev, step0=0, trace_dev=None, allow=(), status=False):
        """len(eps_dev) batched SGLD steps with the packed psi resident on the device."""
        st = self._lib.ulisse_batch_sgld_chain(
            self._h, ctypes.c_void_p(psi_dev.data_ptr()), ctypes.c_void_p(eps_dev.data_ptr()),
            int(eps_dev.numel()), step0,
            ctypes.c_void_p(trace_dev.data_ptr()) if trace_dev is not None else None)
        self._check(st, allow)
        return st if status else psi_dev


def ulisse_kmv_noalloc(X, psi, V, which=-1, out=None, stream=None):
    """U = K V (or dK/dpsi_which V) through the allocation-free entry point: X (n, d) and
    V (n, R <= 32) CUDA float tensors; the library allocates nothing for this call."""
    import torch
    lib = load()
    X = X.contiguous().float()
    n, d = X.shape
    Vc = _colmajor(V.float())
    R = Vc.shape[1]
    if out is None:
        out = torch.empty((R, n), dtype=torch.float32, device=V.device).t()
    psi = _f64_host(psi, d + 2)
    stream = stream if stream is not None else torch.cuda.current_stream(V.device)
    st = lib.ulisse_kmv_noalloc(ctypes.c_void_p(X.data_ptr()), n, d, _hptr(psi), which,
                                ctypes.c_void_p(Vc.data_ptr()), R,
                                ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(stream.cuda_stream))
    if st != ULISSE_OK:
        raise UlisseError(st, "ulisse_kmv_noalloc rejected the call")
    return out[:, 0] if V.dim() == 1 else out


def ulisse_kmv_noalloc_status(stream=None):
    """Status word of the last ulisse_kmv_noalloc call's device work (0: every bounded wait
    ended); synchronises `stream`.  Raises UlisseError on a timeout or a CUDA error."""
    import torch
    lib = load()
    stream = stream if stream is not None else torch.cuda.current_stream()
    word = ctypes.c_int(-1)
    st = lib.ulisse_kmv_noalloc_status(ctypes.c_void_p(stream.cuda_stream), ctypes.byref(word))
    if st != ULISSE_OK:
        raise UlisseError(st, "ulisse_kmv_noalloc: status word %d" % word.value)
    return word.value


def ulisse_measure_ex2_rate(stream=None, reps=5):
    """Exponentials per second of the current device (best of `reps` timed launches) and
    the duration of that launch in ms."""
    import torch
    stream = stream if stream is not None else torch.cuda.current_stream()
    rate, ms = ctypes.c_double(), ctypes.c_double()
    st = load().ulisse_measure_ex2_rate(ctypes.c_void_p(stream.cuda_stream), int(reps),
                                        ctypes.byref(rate), ctypes.byref(ms))
    if st != ULISSE_OK:
        raise UlisseError(st, "ulisse_measure_ex2_rate failed")
    return rate.value, ms.value


def ulisse_ws_init(ctx: Context, **kw):
    ctx.ws_init(**kw)


def ulisse_ws_set(ctx: Context, record=False, use=False):
    ctx.ws_set(record, use)


def ulisse_ws_train(ctx: Context, steps, batch=64, lr=1e-3):
    return ctx.ws_train(steps, batch, lr)


def ulisse_ws_loss_grad(ctx: Context):
    return ctx.ws_loss_grad()


def ulisse_ws_export(ctx: Context):
    return ctx.ws_export()


def ulisse_ws_x0(ctx: Context, psi, bf16=False):
    return ctx.ws_x0(psi, bf16)


def ulisse_destroy(ctx: Context):
    ctx.close()


def ulisse_create_batched(Xs, ys, cfg: ulisse_config | None = None, stream=None) -> BatchContext:
    return BatchContext(Xs, ys, cfg, stream)


def ulisse_batch_size(ctx: BatchContext):
    n = ctypes.c_int()
    p = ctypes.c_int()
    ctx._check(ctx._lib.ulisse_batch_size(ctx._h, ctypes.byref(n), ctypes.byref(p)))
    return n.value, p.value


def ulisse_batch_kmv(ctx: BatchContext, psi, Vs):
    return ctx.kmv(psi, Vs)


def ulisse_batch_grad(ctx: BatchContext, psi, step=0):
    return ctx.grad(psi, step)


def ulisse_batch_sgld_step(ctx: BatchContext, psi, eps_t, step):
    return ctx.sgld_step(psi, eps_t, step)


def ulisse_set_graph(ctx: Context, enable=True):
    ctx.set_graph(enable)


def ulisse_autotune(ctx: Context, psi, max_cols=None, reps=3):
    return ctx.autotune(psi, max_cols, reps)


def ulisse_batch_sgld_chain(ctx: BatchContext, psi_dev, eps_dev, step0=0, trace_dev=None):
    return ctx.sgld_chain(psi_dev, eps_dev, step0, trace_dev)
