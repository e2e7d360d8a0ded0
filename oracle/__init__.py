"""FP64 CPU oracle for SGLD + ULISSE (Filippone & Engler, ICML 2015).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow reference the CUDA library is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the library itself never does, and it shares no code with the
library.  The O(n^2) loops live in ``ulisse_oracle.c`` (plain C, double precision); the exact
small-n path (dense Cholesky, log marginal likelihood, exact gradient) is written here with
numpy, using ``numpy.linalg.cholesky`` / triangular solves as library steps.

Parameter vector: psi = (log l_1..log l_d, log sigma^2, log lambda), p = d + 2.

Preconditioned CG with J = K + delta I (Sec. 3) and ULISSE on its outer iteration is in
``oracle/pcg.py`` (numpy on the dense K).

Pinning status of each function (what other than itself checks it) is listed in
``tests/test_oracle_pins.py``; every function here is pinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "ulisse_oracle.c")
_lock = threading.Lock()
_lib = None

PURPOSE_PROBE = 1
PURPOSE_ULISSE = 2
PURPOSE_SGLD = 3


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, OpenMP, no fast-math).  Returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            L = ctypes.c_long
            I = ctypes.c_int
            D = ctypes.c_double
            U64 = ctypes.c_uint64
            lib.orc_philox4x64_10.argtypes = [P, P, P]
            lib.orc_u01.argtypes = [U64]
            lib.orc_u01.restype = D
            lib.orc_cov_matrix.argtypes = [P, L, I, P, I, P]
            lib.orc_kmv.argtypes = [P, L, I, P, I, P, I, P]
            lib.orc_dkmv_all.argtypes = [P, L, I, P, P, I, P]
            lib.orc_kmv_rows.argtypes = [P, L, I, P, I, P, I, P, L, P]
            lib.orc_kmv_rows_abs.argtypes = [P, L, I, P, I, P, I, P, L, P]
            lib.orc_dkmv_all_rows.argtypes = [P, L, I, P, P, I, P, L, P]
            lib.orc_cross_signal.argtypes = [P, L, P, L, I, P, P]
            lib.orc_probes.argtypes = [L, I, I, U64, U64, P]
            lib.orc_draw_J.argtypes = [U64, U64, U64, I, D, I]
            lib.orc_draw_J.restype = I
            lib.orc_cg_record.argtypes = [P, L, I, P, P, P, D, I, P, P, P, P, P]
            lib.orc_cg_record.restype = I
            lib.orc_ulisse_solve.argtypes = [P, L, I, P, P, I, P, P, P, D, D, D, I, U64, U64, P, P]
            lib.orc_grad_estimate.argtypes = [P, P, L, I, P, I, I, I, D, D, D, I, U64, U64, P, P]
            lib.orc_chol.argtypes = [I, P, P]
            lib.orc_chol.restype = I
            lib.orc_sgld_noise.argtypes = [U64, U64, I, P]
            lib.orc_sgld_update.argtypes = [I, P, P, P, P, D, U64, U64, P]
            lib.orc_sgld_update.restype = I
            lib.orc_sgld_step.argtypes = [P, P, L, I, P, I, I, I, D, D, D, I, U64, U64, D, P, P, P, P, P]
            lib.orc_sgld_step.restype = I
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _colmajor(V, n):
    """(n,) or (n, R) array -> contiguous column-major float64 buffer and R."""
    V = np.asarray(V, dtype=np.float64)
    if V.ndim == 1:
        V = V[:, None]
    assert V.shape[0] == n
    return np.ascontiguousarray(V.T), V.shape[1]


# ----------------------------------------------------------------------------------------
# Random numbers
# ----------------------------------------------------------------------------------------
def philox4x64_10(ctr, key):
    """Philox4x64-10 block: four 64-bit counter words and two key words -> four words."""
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    _load().orc_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def u01(word: int) -> float:
    return _load().orc_u01(int(word))


def probes(n, nr, kind, seed, epoch):
    """Hutchinson probes (Sec. 2.1): n x nr, +-1 (kind 0) or N(0,1) (kind 1)."""
    out = np.zeros((nr, n))
    _load().orc_probes(n, nr, kind, seed, epoch, _ptr(out))
    return out.T.copy()


def draw_J(seed, step, colid, est, beta, jcap=1000):
    """Number of accepted ULISSE steps j >= 1 after the early stop (Sec. 4)."""
    return _load().orc_draw_J(seed, step, colid, est, beta, jcap)


def sgld_noise(seed, step, p):
    out = np.zeros(p)
    _load().orc_sgld_noise(seed, step, p, _ptr(out))
    return out


# ----------------------------------------------------------------------------------------
# Covariance and matrix-free products (Eq. covariance:rbf, Sec. 3)
# ----------------------------------------------------------------------------------------
def cov_matrix(X, psi, which=-1):
    """Dense K (which=-1) or dK/dpsi_which, computed entry by entry (small n)."""
    X = _f64(X)
    n, d = X.shape
    psi = _f64(psi)
    assert psi.shape == (d + 2,)
    K = np.zeros((n, n))
    _load().orc_cov_matrix(_ptr(X), n, d, _ptr(psi), which, _ptr(K))
    return K


def kmv(X, psi, V, which=-1):
    """U = K V (which=-1) or dK/dpsi_which V without storing K.  V: (n,) or (n, R)."""
    X = _f64(X)
    n, d = X.shape
    psi = _f64(psi)
    Vc, R = _colmajor(V, n)
    U = np.zeros((R, n))
    _load().orc_kmv(_ptr(X), n, d, _ptr(psi), which, _ptr(Vc), R, _ptr(U))
    out = U.T.copy()
    return out[:, 0] if np.asarray(V).ndim == 1 else out


def kmv_rows(X, psi, V, rows, which=-1, absolute=False):
    """Rows `rows` of K V (or dK/dpsi_which V); absolute=True gives sum_j |A_ij| |V_jr|."""
    X = _f64(X)
    n, d = X.shape
    psi = _f64(psi)
    Vc, R = _colmajor(V, n)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    U = np.zeros((R, len(rows)))
    fn = _load().orc_kmv_rows_abs if absolute else _load().orc_kmv_rows
    fn(_ptr(X), n, d, _ptr(psi), which, _ptr(Vc), R, _ptr(rows), len(rows), _ptr(U))
    return U.T.copy()


def dkmv_all_rows(X, psi, V, rows):
    """Rows `rows` of all p derivative products, returned as (p, len(rows), R)."""
    X = _f64(X)
    n, d = X.shape
    psi = _f64(psi)
    Vc, R = _colmajor(V, n)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    U = np.zeros((d + 2, R, len(rows)))
    _load().orc_dkmv_all_rows(_ptr(X), n, d, _ptr(psi), _ptr(Vc), R, _ptr(rows), len(rows),
                              _ptr(U))
    return np.transpose(U, (0, 2, 1)).copy()


def omp_threads():
    """Threads the oracle's OpenMP loops use."""
    lib = _load()
    try:
        f = lib.omp_get_max_threads
        f.restype = ctypes.c_int
        return int(f())
    except AttributeError:
        return os.cpu_count() or 1


def cross_signal(X1, X2, psi):
    """Signal covariance k_s(x1_a, x2_b) between two point sets (n1 x n2)."""
    X1 = _f64(X1)
    X2 = _f64(X2)
    n1, d = X1.shape
    n2 = X2.shape[0]
    psi = _f64(psi)
    C = np.zeros((n1, n2))
    _load().orc_cross_signal(_ptr(X1), n1, _ptr(X2), n2, d, _ptr(psi), _ptr(C))
    return C


def dkmv_all(X, psi, V):
    """All p derivative products dK/dpsi_q V, returned as (p, n, R)."""
    X = _f64(X)
    n, d = X.shape
    psi = _f64(psi)
    Vc, R = _colmajor(V, n)
    p = d + 2
    U = np.zeros((p, R, n))
    _load().orc_dkmv_all(_ptr(X), n, d, _ptr(psi), _ptr(Vc), R, _ptr(U))
    return np.transpose(U, (0, 2, 1)).copy()


def dk_bilinear(X, psi, A, B, scale=None):
    """out_i = sum_m scale_m a_m^T (dK/dpsi_i) b_m for all p parameters: the bilinear forms
    the gradient estimate (Eq. gradient:unbiased) is assembled from.  A, B: (n, M).  The
    derivative products dK/dpsi_i b_m come from dkmv_all; the rest is a plain sum."""
    A = _f64(A)
    B = _f64(B)
    if A.ndim == 1:
        A = A[:, None]
        B = B[:, None]
    M = A.shape[1]
    s = np.ones(M) if scale is None else _f64(scale)
    U = dkmv_all(X, psi, B)                      # (p, n, M)
    return np.einsum("jm,ijm,m->i", A, U, s)


# ----------------------------------------------------------------------------------------
# CG (Algorithm 1) and ULISSE (Sec. 4)
# ----------------------------------------------------------------------------------------
def cg_record(X, psi, b, s0=None, eps=1e-8, max_iter=None):
    """Algorithm 1 on K s = b with every iterate recorded.

    Returns dict(S, E, D: (T+1, n); alpha, beta: (T,); T)."""
    X = _f64(X)
    n, d = X.shape
    psi = _f64(psi)
    b = _f64(b)
    max_iter = max_iter or 4 * n
    S = np.zeros((max_iter + 1, n))
    E = np.zeros((max_iter + 1, n))
    D = np.zeros((max_iter + 1, n))
    al = np.zeros(max_iter)
    bt = np.zeros(max_iter)
    s0a = _f64(s0) if s0 is not None else None
    T = _load().orc_cg_record(_ptr(X), n, d, _ptr(psi), _ptr(b), _ptr(s0a), eps, max_iter,
                              _ptr(S), _ptr(E), _ptr(D), _ptr(al), _ptr(bt))
    return dict(S=S[: T + 1], E=E[: T + 1], D=D[: T + 1], alpha=al[:T], beta=bt[:T], T=T)


def ulisse_solve(X, psi, B, n_est=None, colid=None, S0=None, q=1.0, beta=1.0, eps=1e-8,
                 max_iter=None, seed=0, step=0):
    """ULISSE estimates for the columns of B (n x R).

    n_est[c] independent estimators per column (default 1).  Returns (S_est, stats):
    S_est is n x sum(n_est) (estimators of column 0 first); stats is R x 5 with
    [l, iterations, outcome, J_0, J_1] (outcome 0 ok, 3 breakdown, 4 max_iter)."""
    X = _f64(X)
    n, d = X.shape
    psi = _f64(psi)
    Bc, R = _colmajor(B, n)
    n_est = np.ascontiguousarray(n_est if n_est is not None else np.ones(R), dtype=np.int32)
    colid = np.ascontiguousarray(colid if colid is not None else np.arange(R), dtype=np.int64)
    S0c = _colmajor(S0, n)[0] if S0 is not None else None
    max_iter = max_iter or 4 * n
    tot = int(n_est.sum())
    S_est = np.zeros((tot, n))
    stats = np.zeros((R, 5), dtype=np.int64)
    _load().orc_ulisse_solve(_ptr(X), n, d, _ptr(psi), _ptr(Bc), R, _ptr(S0c), _ptr(n_est),
                             _ptr(colid), q, beta, eps, max_iter, seed, step, _ptr(S_est),
                             _ptr(stats))
    return S_est.T.copy(), stats


def grad_estimate(X, y, psi, nr=4, probe_kind=0, probe_refresh=1, q=1.0, beta=1.0, eps=1e-8,
                  max_iter=None, seed=0, step=0):
    """Unbiased gradient estimate g~ (Eq. gradient:unbiased) in psi coordinates."""
    X = _f64(X)
    n, d = X.shape
    y = _f64(y)
    psi = _f64(psi)
    max_iter = max_iter or 4 * n
    g = np.zeros(d + 2)
    stats = np.zeros((1 + nr, 5), dtype=np.int64)
    _load().orc_grad_estimate(_ptr(X), _ptr(y), n, d, _ptr(psi), nr, probe_kind, probe_refresh,
                              q, beta, eps, max_iter, seed, step, _ptr(g), _ptr(stats))
    return g, stats


def chol(M):
    M = _f64(M)
    p = M.shape[0]
    L = np.zeros((p, p))
    rc = _load().orc_chol(p, _ptr(M), _ptr(L))
    if rc != 0:
        raise np.linalg.LinAlgError("matrix not positive definite")
    return L


def sgld_update(psi, g, eps_t, M=None, prior_grad=None, seed=0, step=0):
    """SGLD proposal (Sec. 2.1) given the gradient estimate g."""
    psi = _f64(psi)
    p = psi.shape[0]
    g = _f64(g)
    Mc = _f64(M) if M is not None else None
    pg = _f64(prior_grad) if prior_grad is not None else None
    out = np.zeros(p)
    rc = _load().orc_sgld_update(p, _ptr(psi), _ptr(g), _ptr(Mc), _ptr(pg), eps_t, seed, step,
                                 _ptr(out))
    if rc != 0:
        raise np.linalg.LinAlgError("M not positive definite")
    return out


def sgld_step(X, y, psi, eps_t, nr=4, probe_kind=0, probe_refresh=1, q=1.0, beta=1.0,
              eps=1e-8, max_iter=None, seed=0, step=0, M=None, prior_grad=None):
    """One full SGLD step: probes, ULISSE solves, gradient estimate, update."""
    X = _f64(X)
    n, d = X.shape
    y = _f64(y)
    psi = _f64(psi)
    p = d + 2
    max_iter = max_iter or 4 * n
    Mc = _f64(M) if M is not None else None
    pg = _f64(prior_grad) if prior_grad is not None else None
    out = np.zeros(p)
    g = np.zeros(p)
    stats = np.zeros((1 + nr, 5), dtype=np.int64)
    rc = _load().orc_sgld_step(_ptr(X), _ptr(y), n, d, _ptr(psi), nr, probe_kind, probe_refresh,
                               q, beta, eps, max_iter, seed, step, eps_t, _ptr(Mc), _ptr(pg),
                               _ptr(out), _ptr(g), _ptr(stats))
    if rc != 0:
        raise np.linalg.LinAlgError("M not positive definite")
    return out, g, stats


# ----------------------------------------------------------------------------------------
# Exact small-n path (Sec. 2): Cholesky factorisation of the stored K
# ----------------------------------------------------------------------------------------
def _chol_solve(L, b):
    z = np.linalg.solve(L, b)          # forward substitution (L lower triangular)
    return np.linalg.solve(L.T, z)     # back substitution


def exact_solve(X, psi, b):
    """K^{-1} b through the Cholesky factor K = L L^T."""
    K = cov_matrix(X, psi)
    L = np.linalg.cholesky(K)
    return _chol_solve(L, np.asarray(b, dtype=np.float64))


def log_marginal_likelihood(X, y, psi):
    """log p(y | theta, X) = -1/2 log|K| - 1/2 y^T K^{-1} y - n/2 log(2 pi)  (Sec. 2)."""
    K = cov_matrix(X, psi)
    L = np.linalg.cholesky(K)
    y = np.asarray(y, dtype=np.float64)
    a = _chol_solve(L, y)
    n = len(y)
    return -np.sum(np.log(np.diag(L))) - 0.5 * y @ a - 0.5 * n * np.log(2 * np.pi)


def exact_gradient(X, y, psi):
    """g_i = -1/2 Tr(K^{-1} dK_i) + 1/2 y^T K^{-1} dK_i K^{-1} y  (Eq. gradient:exact)."""
    X = _f64(X)
    d = X.shape[1]
    K = cov_matrix(X, psi)
    L = np.linalg.cholesky(K)
    n = K.shape[0]
    Kinv = _chol_solve(L, np.eye(n))
    a = _chol_solve(L, np.asarray(y, dtype=np.float64))
    g = np.zeros(d + 2)
    for i in range(d + 2):
        dK = cov_matrix(X, psi, which=i)
        g[i] = -0.5 * np.sum(Kinv * dK.T) + 0.5 * a @ dK @ a
    return g


def predict(X, y, psi, Xs):
    """Posterior predictive at new inputs Xs (Sec. 2): p(y*_j | y, psi) = N(mean_j, var_j),
    mean_j = k*_j^T K^{-1} y, var_j = sigma^2 + lambda - k*_j^T K^{-1} k*_j, with k*_j the
    signal covariance between X and x*_j, through the Cholesky factor of K."""
    X = _f64(X)
    Xs = _f64(Xs)
    d = X.shape[1]
    K = cov_matrix(X, psi)
    L = np.linalg.cholesky(K)
    Ks = cross_signal(X, Xs, psi)                   # n x m
    a = _chol_solve(L, np.asarray(y, dtype=np.float64))
    W = np.linalg.solve(L, Ks)                      # L^{-1} k*, so k*^T K^{-1} k* = |W_j|^2
    sigma2, lam = np.exp(psi[d]), np.exp(psi[d + 1])
    return Ks.T @ a, sigma2 + lam - np.sum(W * W, axis=0)


def exact_trace_term(X, psi, i):
    """Tr(K^{-1} dK_i) through the Cholesky factor."""
    K = cov_matrix(X, psi)
    L = np.linalg.cholesky(K)
    Kinv = _chol_solve(L, np.eye(K.shape[0]))
    dK = cov_matrix(X, psi, which=i)
    return float(np.sum(Kinv * dK.T))


# ----------------------------------------------------------------------------------------
# ULISSE closed forms used by the pins (Sec. 4)
# ----------------------------------------------------------------------------------------
def weight_product(j, beta):
    """prod_{r=0}^{j} w_r with w_r = exp(beta r)."""
    return float(np.prod([np.exp(beta * r) for r in range(j + 1)]))


def expected_tail_steps(beta, tol=1e-300):
    """Expected number of steps run after the early stop: sum_j prod_{r<=j} 1/w_r."""
    total, j = 0.0, 0
    while True:
        inv = 1.0
        for r in range(j + 1):
            inv /= np.exp(beta * r)
        if inv < tol or j > 100000:
            return float(total)
        total += inv
        j += 1
