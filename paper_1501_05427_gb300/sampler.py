"""Host-side control of an SGLD run (Sec. 2.1 and the experimental choices of Sec. 5.1): the
decreasing step size, the monitor of the Langevin dynamics phase with the step-size freeze,
and the preconditioner M from a subset of the data.  Everything per step runs in the
library (one ulisse_sgld_step per step); what is here is small host arithmetic on p x p
matrices, plus one FP64 fit on a few hundred points for M.

* Step size (Sec. 2.1): eps_t = a (b + t)^(-gamma) with gamma = 1; Sec. 5.1 fixes it by its
  first and last values (1e-1 and 1e-4 over the run).
* Langevin phase (Sec. 2.1, after Welling and Teh): the ratio
      eps_t / 4 * lambda_max(M^(1/2) V M^(1/2)),
  V the sampling covariance of the stochastic gradients, is small once the injected noise
  dominates the gradient noise.  Sec. 5.1 estimates V on batches of one hundred iterations and
  freezes eps_t once the ratio is below 0.002.
* Preconditioner (Sec. 5.1): M = (-H)^(-1), H the Hessian of the log posterior at its mode,
  computed on a subset of five hundred inputs.  With the flat prior in psi the log posterior is
  the log marginal likelihood of Sec. 2; it is evaluated here by a dense Cholesky factor
  in FP64, its gradient by the trace formula of Eq. gradient:exact, the mode by Newton steps and
  H by central differences of that gradient.
"""
from __future__ import annotations

import math

import numpy as np


# ------------------------------------------------------------------------------------------
# Step size
# ------------------------------------------------------------------------------------------
def step_size_schedule(eps_first, eps_last, n_steps, gamma=1.0):
    """(a, b) of eps_t = a (b + t)^(-gamma) with eps_0 = eps_first and eps_{n_steps-1} =
    eps_last (Sec. 5.1 uses 1e-1 and 1e-4 with gamma = 1)."""
    if not (eps_first > eps_last > 0.0) or n_steps < 2 or gamma <= 0.0:
        raise ValueError("need eps_first > eps_last > 0, n_steps >= 2, gamma > 0")
    r = (eps_first / eps_last) ** (1.0 / gamma)      # ((b + T - 1) / b)
    b = (n_steps - 1) / (r - 1.0)
    a = eps_first * b ** gamma
    return a, b


def step_size(a, b, t, gamma=1.0):
    return a * (b + t) ** (-gamma)


# ------------------------------------------------------------------------------------------
# Langevin-phase monitor
# ------------------------------------------------------------------------------------------
def noise_ratio(eps_t, M, V):
    """eps_t / 4 * lambda_max(M^(1/2) V M^(1/2)).  With M = L L^T the matrix L^T V L has the
    same eigenvalues as M^(1/2) V M^(1/2) (both are similar to V M)."""
    L = np.linalg.cholesky(np.asarray(M, dtype=np.float64))
    S = L.T @ np.asarray(V, dtype=np.float64) @ L
    S = 0.5 * (S + S.T)
    return 0.25 * eps_t * float(np.linalg.eigvalsh(S)[-1])


class LangevinMonitor:
    """Collects the stochastic gradients of a run in batches (Sec. 5.1: one hundred iterations)
    and freezes the step size the first time the noise ratio of a completed batch is below the
    threshold (Sec. 5.1: 0.002).  `ratios` holds (step, ratio) per completed batch."""

    def __init__(self, M, batch=100, threshold=0.002):
        if batch < 2:
            raise ValueError("a batch needs at least two gradients")
        self.M = np.asarray(M, dtype=np.float64)
        self.batch = int(batch)
        self.threshold = float(threshold)
        self._g = []
        self.ratios = []
        self.frozen_at = None      # step at which the step size was frozen
        self.frozen_eps = None

    def update(self, step, eps_t, g):
        """Record the gradient of `step` (taken with step size eps_t).  Returns None while the
        schedule goes on, and the frozen step size from the batch whose noise ratio first falls
        below the threshold on (the step size to use for every later step)."""
        if self.frozen_at is not None:
            return self.frozen_eps
        self._g.append(np.asarray(g, dtype=np.float64))
        if len(self._g) == self.batch:
            G = np.stack(self._g)
            V = np.cov(G, rowvar=False, ddof=1)
            r = noise_ratio(eps_t, self.M, V)
            self.ratios.append((step, r))
            self._g = []
            if r < self.threshold:
                self.frozen_at = step
                self.frozen_eps = eps_t
                return eps_t
        return None


# ------------------------------------------------------------------------------------------
# Preconditioner from a subset (FP64, host)
# ------------------------------------------------------------------------------------------
def _cov(X, psi):
    d = X.shape[1]
    ls = np.exp(psi[:d])
    sig2, lam = math.exp(psi[d]), math.exp(psi[d + 1])
    Z = X / ls
    sq = np.sum(Z * Z, axis=1)
    D2 = np.maximum(sq[:, None] + sq[None, :] - 2.0 * Z @ Z.T, 0.0)
    Ks = sig2 * np.exp(-0.5 * D2)
    return Z, Ks, lam


def log_marginal_likelihood(X, y, psi):
    """log N(y | 0, K(psi)) (Sec. 2) by a dense Cholesky factor; FP64."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    psi = np.asarray(psi, dtype=np.float64)
    _, Ks, lam = _cov(X, psi)
    K = Ks + lam * np.eye(len(y))
    L = np.linalg.cholesky(K)
    a = np.linalg.solve(L, y)
    return -0.5 * a @ a - np.sum(np.log(np.diag(L))) - 0.5 * len(y) * math.log(2.0 * math.pi)


def lml_gradient(X, y, psi):
    """Gradient of the log marginal likelihood in psi (Eq. gradient:exact):
    g_i = 1/2 alpha^T dK_i alpha - 1/2 tr(K^-1 dK_i), alpha = K^-1 y; FP64."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    psi = np.asarray(psi, dtype=np.float64)
    n, d = X.shape
    Z, Ks, lam = _cov(X, psi)
    K = Ks + lam * np.eye(n)
    Kinv = np.linalg.inv(K)
    Kinv = 0.5 * (Kinv + Kinv.T)
    alpha = Kinv @ y
    W = np.outer(alpha, alpha) - Kinv           # g_i = 1/2 sum_ab W_ab dK_i,ab
    g = np.empty(d + 2)
    for k in range(d):
        Dk = (Z[:, k][:, None] - Z[:, k][None, :]) ** 2
        g[k] = 0.5 * np.sum(W * Ks * Dk)
    g[d] = 0.5 * np.sum(W * Ks)
    g[d + 1] = 0.5 * lam * np.trace(W)
    return g


def lml_hessian(X, y, psi, h=1e-4):
    """Hessian of the log marginal likelihood in psi by central differences of its gradient."""
    psi = np.asarray(psi, dtype=np.float64)
    p = len(psi)
    H = np.empty((p, p))
    for i in range(p):
        e = np.zeros(p)
        e[i] = h
        H[i] = (lml_gradient(X, y, psi + e) - lml_gradient(X, y, psi - e)) / (2.0 * h)
    return 0.5 * (H + H.T)


def posterior_mode(X, y, psi0, max_iter=50, tol=1e-8):
    """Mode of the log posterior (flat prior in psi) by damped Newton steps on the subset."""
    psi = np.asarray(psi0, dtype=np.float64).copy()
    f = log_marginal_likelihood(X, y, psi)
    for _ in range(max_iter):
        g = lml_gradient(X, y, psi)
        if np.max(np.abs(g)) < tol * max(1.0, abs(f)):
            break
        H = lml_hessian(X, y, psi)
        w, U = np.linalg.eigh(-H)
        step = U @ ((U.T @ g) / np.maximum(w, 1e-6 * max(1.0, w.max())))
        t = 1.0
        while t > 1e-6:
            cand = psi + t * step
            fc = log_marginal_likelihood(X, y, cand)
            if fc > f:
                psi, f = cand, fc
                break
            t *= 0.5
        else:
            break
    return psi


def preconditioner_from_subset(X, y, psi0, m=500, seed=0):
    """M = (-H)^(-1) at the log-posterior mode of a random subset of m inputs (Sec. 5.1).
    Returns (M, psi_mode)."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    idx = np.random.default_rng(seed).choice(len(y), min(m, len(y)), replace=False)
    Xs, ys = X[idx], y[idx]
    mode = posterior_mode(Xs, ys, psi0)
    H = lml_hessian(Xs, ys, mode)
    w, U = np.linalg.eigh(-H)
    w = np.maximum(w, 1e-8 * max(1.0, w.max()))    # guard a flat direction of the subset
    M = (U / w) @ U.T
    return 0.5 * (M + M.T), mode


# ------------------------------------------------------------------------------------------
# A run
# ------------------------------------------------------------------------------------------
def run_sgld(ctx, psi0, n_steps, eps_first=1e-1, eps_last=1e-4, M=None, batch=100,
             threshold=0.002, step0=0, prior_grad=None, record=None):
    """SGLD as Sec. 5.1 runs it: eps_t = a (b + t)^-1 from eps_first to eps_last, the Langevin
    monitor on batches of `batch` gradients, the step size frozen once the noise ratio is below
    `threshold`.  ctx is a ulisse.Context (one ulisse_sgld_step per step).  prior_grad: None
    (flat prior in psi), a vector, or a function of psi giving grad_psi log p(psi).  record:
    None, or a list to which (t, eps_t, g~) is appended every step.  Returns (trace of psi,
    the monitor)."""
    p = len(psi0)
    Mm = np.eye(p) if M is None else np.asarray(M, dtype=np.float64)
    a, b = step_size_schedule(eps_first, eps_last, n_steps)
    mon = LangevinMonitor(Mm, batch=batch, threshold=threshold)
    psi = np.asarray(psi0, dtype=np.float64).copy()
    trace = np.empty((n_steps, p))
    eps_frozen = None
    for t in range(n_steps):
        eps_t = eps_frozen if eps_frozen is not None else step_size(a, b, t)
        pg = prior_grad(psi) if callable(prior_grad) else prior_grad
        psi, g = ctx.sgld_step(psi, eps_t, step0 + t, M=None if M is None else Mm, prior_grad=pg)
        trace[t] = psi
        if record is not None:
            record.append((t, eps_t, np.array(g)))
        if eps_frozen is None:
            eps_frozen = mon.update(t, eps_t, g)
    return trace, mon


# ------------------------------------------------------------------------------------------
# Posterior predictive averaging (Sec. 2, Eq. monte:carlo:integration)
# ------------------------------------------------------------------------------------------
def posterior_predictive(ctx, psi_samples, Xs, step0=0, var=True):
    """The Monte Carlo estimate of p(y* | y) = integral p(y* | y, theta) p(theta | y) dtheta:
    for every posterior sample psi^(i) the library gives p(y* | y, psi^(i)) = N(mean_i, var_i)
    (ulisse_predict, one solve per sample, step step0 + i for its random draws), and the
    predictive is their equal-weight mixture.  Returns (means (N, m), variances (N, m) or None)
    as numpy arrays; see mixture_moments and mixture_density for the mixture."""
    means, varis = [], []
    for i, psi in enumerate(np.asarray(psi_samples, dtype=np.float64)):
        m, v = ctx.predict(psi, Xs, step=step0 + i, var=var)
        means.append(m.cpu().numpy().astype(np.float64))
        if var:
            varis.append(v.cpu().numpy().astype(np.float64))
    return np.array(means), (np.array(varis) if var else None)


def mixture_moments(means, variances):
    """Mean and variance of the equal-weight mixture of N(means[i], variances[i]) (per test
    input): E[y*] = mean_i means, Var[y*] = mean_i (variances + means^2) - E[y*]^2 (the law of
    total variance)."""
    means = np.asarray(means, dtype=np.float64)
    variances = np.asarray(variances, dtype=np.float64)
    mu = means.mean(axis=0)
    return mu, (variances + means * means).mean(axis=0) - mu * mu


def mixture_density(y_star, means, variances):
    """The Monte Carlo predictive density (1/N) sum_i N(y_star; means[i], variances[i]) at the
    values y_star (one per test input)."""
    means = np.asarray(means, dtype=np.float64)
    variances = np.asarray(variances, dtype=np.float64)
    z = (np.asarray(y_star, dtype=np.float64)[None, :] - means) ** 2 / variances
    return (np.exp(-0.5 * z) / np.sqrt(2 * math.pi * variances)).mean(axis=0)
