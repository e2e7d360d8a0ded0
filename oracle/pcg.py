"""FP64 oracle of preconditioned CG (PCG) with the ULISSE truncation on the outer iteration.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): plain numpy on the dense covariance matrix,
for the small sizes the tests use; the library never imports it.

Sec. 3 ("Preconditioned CG") preconditions K s = b with J = K + delta I (delta > 0): the
system becomes K J^{-1} (J s) = b, and every iteration solves an inner system J z = e, itself
by CG.  With K and J symmetric positive definite this is the standard preconditioned CG:

    e_0 = b - K s_0,  z_0 = J^{-1} e_0,  d_0 = z_0
    alpha_i = e_i^T z_i / d_i^T K d_i
    s_{i+1} = s_i + alpha_i d_i,   e_{i+1} = e_i - alpha_i K d_i      (stop when ||e|| < eps)
    z_{i+1} = J^{-1} e_{i+1}
    beta_i = e_{i+1}^T (z_{i+1} - z_i) / e_i^T z_i
    d_{i+1} = z_{i+1} + beta_i d_i

Readings where the paper is silent:
  * the inner CG starts from 0 and stops at the first iteration k with ||r_k|| <= tau ||e||
    (relative tolerance tau), or after inner_max iterations;
  * because the inner solve is inexact the preconditioner changes from one iteration to the
    next, so beta takes the flexible (Polak-Ribiere) form above; with exact inner solves
    e_{i+1}^T z_i = 0 and it equals the usual e_{i+1}^T z_{i+1} / e_i^T z_i;
  * Sec. 4 applies ULISSE to any CG variant: the increments are delta_i = s_i - s_{i-1} of the
    outer iteration, the early stop compares the outer residual ||e_i|| with q sqrt(n), and
    the accepted steps J come from the same counter-based draws as plain CG's (column c,
    estimator t), so the reconstruction and its expectation are those of Sec. 4.
"""
from __future__ import annotations

import math

import numpy as np

from . import cov_matrix, draw_J


def inner_cg(Jm, r0, tau, inner_max):
    """CG on Jm x = r0 from x = 0 until ||r|| <= tau ||r0|| or inner_max iterations.
    Returns (x, iterations)."""
    x = np.zeros_like(r0)
    r = r0.copy()
    p = r.copy()
    rr = float(r @ r)
    thr = tau * tau * rr
    k = 0
    while k < inner_max:
        q = Jm @ p
        a = rr / float(p @ q)
        x = x + a * p
        r = r - a * q
        k += 1
        rr1 = float(r @ r)
        if rr1 <= thr:
            break
        p = r + (rr1 / rr) * p
        rr = rr1
    return x, k


def pcg_record(X, psi, b, delta, tau=1e-2, inner_max=100, eps=1e-8, max_iter=None,
               exact_inner=False, K=None):
    """Preconditioned CG on K s = b with J = K + delta I, every iterate recorded.

    exact_inner: solve J z = e exactly (dense solve) instead of by the inner CG.
    Returns dict(S, E, D, Z: (T+1, n); alpha, beta: (T,); T; inner: inner iterations of
    every preconditioner solve, in order)."""
    X = np.asarray(X, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = len(b)
    K = cov_matrix(X, psi) if K is None else K
    Jm = K + delta * np.eye(n)
    max_iter = max_iter or 4 * n
    inner = []

    def precondition(e):
        if exact_inner:
            return np.linalg.solve(Jm, e)
        z, k = inner_cg(Jm, e, tau, inner_max)
        inner.append(k)
        return z

    s = np.zeros(n)
    e = b.copy()
    z = precondition(e)
    d = z.copy()
    ez = float(e @ z)
    S, E, D, Z = [s], [e], [d], [z]
    al, bt = [], []
    for _ in range(max_iter):
        Kd = K @ d
        a = ez / float(d @ Kd)
        s = s + a * d
        e = e - a * Kd
        al.append(a)
        S.append(s)
        E.append(e)
        if math.sqrt(float(e @ e)) < eps:
            bt.append(0.0)
            break
        z1 = precondition(e)
        beta = float(e @ (z1 - z)) / ez
        bt.append(beta)
        d = z1 + beta * d
        ez = float(e @ z1)
        z = z1
        D.append(d)
        Z.append(z)
    return dict(S=np.array(S), E=np.array(E), D=np.array(D), Z=np.array(Z),
                alpha=np.array(al), beta=np.array(bt), T=len(al), inner=inner)


def weight(j, beta):
    """prod_{r=0}^{j} w_r with w_r = exp(beta r) = exp(beta j (j + 1) / 2)."""
    return math.exp(beta * j * (j + 1) / 2.0)


def ulisse_pcg_solve(X, psi, B, delta, tau=1e-2, inner_max=100, n_est=None, q=1.0, beta=1.0,
                     eps=1e-8, max_iter=None, seed=0, step=0):
    """ULISSE estimates of K^{-1} B[:, c] from the outer PCG iteration (Sec. 4).

    Column c, estimator t: s~ = s_l + sum_{j=1}^{J_t} (prod_{r<=j} w_r) delta_{l+j}, l the
    first outer iteration i >= 1 with ||e_i|| < q sqrt(n), J_t the accepted steps drawn for
    (seed, step, c, t); the column's outer iteration runs to l + max_t J_t (or converges or
    stops at max_iter first).  Returns (S_est: n x sum(n_est), stats: R x 5 with [l,
    outer iterations, outcome, J_0, J_1], kv_rounds: the K V products of every column, outer
    and inner, counted as in the library: the first preconditioner solve plus, per outer
    iteration, one product and the next preconditioner solve's)."""
    X = np.asarray(X, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[:, None]
    n, R = B.shape
    n_est = np.ones(R, dtype=int) if n_est is None else np.asarray(n_est, dtype=int)
    max_iter = max_iter or 4 * n
    K = cov_matrix(X, psi)
    a_thr = q * math.sqrt(n)
    out = np.zeros((n, int(n_est.sum())))
    stats = np.zeros((R, 5), dtype=np.int64)
    rounds = []
    col = 0
    for c in range(R):
        Js = [draw_J(seed, step, c, t, beta, max_iter) for t in range(n_est[c])]
        jmax = max(Js)
        tr = pcg_record(X, psi, B[:, c], delta, tau, inner_max, eps, max_iter, K=K)
        norms = np.linalg.norm(tr["E"], axis=1)
        T = tr["T"]
        l = next((i for i in range(1, T + 1) if norms[i] < a_thr), 0)
        if l == 0:
            # never below the early-stop threshold: the converged (or capped) iterate
            iters = T
            outcome = 4 if (T == max_iter and norms[T] >= eps) else 0
            est = [tr["S"][T]] * n_est[c]
        else:
            iters = min(l + jmax, T)
            outcome = 0
            est = []
            for J in Js:
                s = tr["S"][l].copy()
                for j in range(1, J + 1):
                    if l + j > T:
                        break
                    s += weight(j, beta) * (tr["S"][l + j] - tr["S"][l + j - 1])
                est.append(s)
        for t in range(n_est[c]):
            out[:, col + t] = est[t]
        stats[c] = [l, iters, outcome, Js[0], Js[1] if n_est[c] > 1 else -1]
        # products actually formed up to `iters` outer iterations: the first preconditioner
        # solve, then per iteration K d and (unless it was the last) the next solve
        inner = tr["inner"]
        rounds.append(sum(inner[:iters]) + iters)
        col += n_est[c]
    return out, stats, rounds
