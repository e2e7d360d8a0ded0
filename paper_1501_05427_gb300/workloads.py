"""Seeded synthetic inputs shaped like the paper's workloads.

This module only makes data (inputs X, labels y and starting parameters).  It holds none of
the method's arithmetic and imports neither the CUDA library nor the oracle, so both sides
can be fed from it.  The paper's datasets (UCI Concrete, n=1030, d=8, Sec. 3; DELVE
Census-house 8L, n=22,784, d=8, Sec. 5.2) are not available; these generators stand in for
them with the sizes and input distributions below.

Label generators:
  * ``gp_cholesky``: y = L z + noise with L L^T the ARD squared-exponential signal covariance
    of the inputs (an exact GP draw; used for the small 2-D workload).  The covariance for
    the draw is formed here with ``scipy.spatial.distance.cdist``, independently of the
    library and of the oracle.
  * ``rff``: a random-Fourier-feature draw (Rahimi & Recht, 2007) of the same ARD kernel,
    y = sqrt(2 sigma^2 / F) sum_f w_f cos(omega_f . x + b_f), omega_f ~ N(0, diag(l^-2)),
    b_f ~ U[0, 2 pi), w_f ~ N(0, 1), plus Gaussian noise (used for the large workloads).

Seeds: workload k of the list below uses seed 20150122 + k.
"""
from __future__ import annotations

import os
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20150122


@dataclass
class Problem:
    """One GP regression problem: inputs, labels and the parameters used to draw them."""
    name: str
    X: np.ndarray            # n x d float32, row-major
    y: np.ndarray            # n float32
    psi_true: np.ndarray     # (log l_1..log l_d, log sigma^2, log lambda), float64
    seed: int
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.X.shape[0]

    @property
    def d(self):
        return self.X.shape[1]


def _psi(lengthscales, sigma2, noise):
    return np.concatenate([np.log(np.asarray(lengthscales, dtype=np.float64)),
                           [np.log(sigma2), np.log(noise)]])


def _rff_labels(rng, X, lengthscales, sigma2, n_features=4096, chunk=8192):
    n, d = X.shape
    omega = rng.standard_normal((d, n_features)) / np.asarray(lengthscales)[:, None]
    b = rng.uniform(0.0, 2.0 * np.pi, n_features)
    w = rng.standard_normal(n_features)
    y = np.empty(n)
    scale = np.sqrt(2.0 * sigma2 / n_features)

    def block(s):
        Z = X[s:s + chunk].astype(np.float64) @ omega + b
        y[s:s + chunk] = scale * (np.cos(Z) @ w)

    # the blocks are independent (same arithmetic whatever the thread), so the labels do not
    # depend on how many run at once; numpy releases the GIL inside cos and the products
    starts = list(range(0, n, chunk))
    if len(starts) > 1:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(max_workers=min(len(starts), os.cpu_count() or 1)) as ex:
            list(ex.map(block, starts))
    else:
        block(0)
    return y


def _gp_cholesky_labels(rng, X, lengthscales, sigma2):
    from scipy.spatial.distance import cdist
    Xs = X.astype(np.float64) / np.asarray(lengthscales)
    C = sigma2 * np.exp(-0.5 * cdist(Xs, Xs, "sqeuclidean"))
    C[np.diag_indices_from(C)] += 1e-8 * sigma2
    L = np.linalg.cholesky(C)
    return L @ rng.standard_normal(X.shape[0])


def small_2d(n=1000, seed=SEED_BASE + 0):
    """Concrete-sized problem: X ~ U[0,1]^2, exact GP draw with l = 0.3, sigma^2 = 1,
    noise variance 0.1."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.0, (n, 2))
    ls = [0.3, 0.3]
    y = _gp_cholesky_labels(rng, X, ls, 1.0) + rng.normal(0.0, np.sqrt(0.1), n)
    return Problem("small_2d", X.astype(np.float32), y.astype(np.float32), _psi(ls, 1.0, 0.1),
                   seed, dict(labels="gp_cholesky"))


def census_like(n=50_000, d=8, noise=0.05, seed=SEED_BASE + 1):
    """Census-shaped problem: X ~ N(0, I_d), RFF draw with l_d log-uniform in [0.5, 2],
    sigma^2 = 1, noise variance 0.05."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d))
    ls = np.exp(rng.uniform(np.log(0.5), np.log(2.0), d))
    y = _rff_labels(rng, X, ls, 1.0) + rng.normal(0.0, np.sqrt(noise), n)
    return Problem("census_like", X.astype(np.float32), y.astype(np.float32),
                   _psi(ls, 1.0, noise), seed, dict(labels="rff"))


def near_duplicates(n=200_000, d=16, dup_frac=0.01, jitter=1e-4, noise=0.01,
                    seed=SEED_BASE + 2):
    """High-dimensional problem with 1% near-duplicate inputs: X ~ N(0, I_16); a random 1%
    of rows are replaced by copies of other rows plus N(0, jitter^2) noise; RFF labels with
    l_d log-uniform in [0.5, 2] (times sqrt(d/8) so typical distances stay comparable),
    noise variance 0.01."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d))
    m = int(round(dup_frac * n))
    dst = rng.choice(n, m, replace=False)
    src = rng.integers(0, n, m)
    X[dst] = X[src] + rng.normal(0.0, jitter, (m, d))
    ls = np.exp(rng.uniform(np.log(0.5), np.log(2.0), d)) * np.sqrt(d / 8.0)
    y = _rff_labels(rng, X, ls, 1.0) + rng.normal(0.0, np.sqrt(noise), n)
    return Problem("near_duplicates", X.astype(np.float32), y.astype(np.float32),
                   _psi(ls, 1.0, noise), seed, dict(labels="rff", duplicates=m))


def uneven_batch(n_problems=64, n_lo=2_000, n_hi=40_000, dims=(2, 4, 8), noise=0.1,
                 seed=SEED_BASE + 3):
    """Many independent problems of uneven size: n ~ U{n_lo..n_hi}, d uniform in dims,
    X ~ U[0,1]^d, RFF labels with l_d log-uniform in [0.2, 1], noise variance 0.1."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_problems):
        n = int(rng.integers(n_lo, n_hi + 1))
        d = int(rng.choice(dims))
        X = rng.uniform(0.0, 1.0, (n, d))
        ls = np.exp(rng.uniform(np.log(0.2), np.log(1.0), d))
        y = _rff_labels(rng, X, ls, 1.0, n_features=1024) + rng.normal(0.0, np.sqrt(noise), n)
        out.append(Problem("uneven_%02d" % k, X.astype(np.float32), y.astype(np.float32),
                           _psi(ls, 1.0, noise), seed, dict(labels="rff", index=k)))
    return out


def warm_start_problem(n=100_000, seed=SEED_BASE + 4):
    """As ``census_like`` with n = 100,000 (the learned warm-start workload)."""
    p = census_like(n=n, d=8, noise=0.05, seed=seed)
    p.name = "warm_start"
    return p


def random_problem(n, d, seed, lengthscale=0.5, sigma2=1.0, noise=0.1, dist="uniform"):
    """Small generic problem for tests: X ~ U[0,1]^d (or N(0,I)), RFF labels."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.0, (n, d)) if dist == "uniform" else rng.standard_normal((n, d))
    ls = np.full(d, lengthscale) * np.exp(rng.uniform(-0.3, 0.3, d))
    y = _rff_labels(rng, X, ls, sigma2, n_features=512) + rng.normal(0.0, np.sqrt(noise), n)
    return Problem("random_%d_%d" % (n, d), X.astype(np.float32), y.astype(np.float32),
                   _psi(ls, sigma2, noise), seed, dict(labels="rff"))


# Workload list: index k uses seed SEED_BASE + k.
WORKLOADS = {
    "small_2d": dict(make=small_2d, n_probes=4, probe_kind="gaussian", steps=100,
                     eps_t=1e-4, precision="fp64"),
    "census_like": dict(make=census_like, n_probes=16, probe_kind="rademacher", steps=500,
                        eps_t=1e-4, precision="fp32"),
    "near_duplicates": dict(make=near_duplicates, n_probes=63, probe_kind="rademacher",
                            precision="mixed"),
    "uneven_batch": dict(make=uneven_batch, n_probes=8, probe_kind="rademacher",
                         precision="fp32"),
    "warm_start": dict(make=warm_start_problem, n_probes=16, probe_kind="rademacher",
                       steps=5000, precision="fp32"),
}
