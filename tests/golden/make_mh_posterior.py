"""Writes mh_posterior_small_2d.txt: the reference posterior of the chain-level validation.

Sec. 5 checks SGLD with ULISSE against Metropolis-Hastings run with the exact likelihood:
fifty thousand iterations, an initial adaptive phase that brings the acceptance rate between
0.2 and 0.4, the first ten thousand discarded.  This script does the same on a synthetic
stand-in for the Concrete data (the 2-D workload of paper_1501_05427_gb300.workloads with
n = 200: the exact GP draw with l = 0.3, sigma^2 = 1, noise 0.1), with the oracle's exact log
marginal likelihood (dense Cholesky) and the prior the test uses, psi ~ N(psi_true, I)
(psi = log of l_1, l_2, sigma^2, lambda; the paper leaves the prior unstated).

Proposal: Gaussian random walk in psi with covariance c * Sigma, Sigma the inverse negative
Hessian of the log posterior at its mode (central differences of the oracle's likelihood);
during the first 10,000 iterations c is rescaled every 500 iterations by the ratio of the
window's acceptance rate to 0.3, then frozen.  Recorded: the posterior mean and standard
deviation of every coordinate over the last 40,000 iterations, with Monte Carlo standard
errors from 40 batch means, the acceptance rate, the mode and Sigma.

Run from the repository root:  python tests/golden/make_mh_posterior.py   (~2 minutes)
Only oracle/ and the input generator are called.
"""
import os

os.environ.setdefault("OMP_NUM_THREADS", "1")          # small matrices: threads cost more
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
import sys  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
from paper_1501_05427_gb300 import workloads as w  # noqa: E402

N_POINTS = 200
ITERS, ADAPT, BATCHES = 50_000, 10_000, 40
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mh_posterior_small_2d.txt")


def main():
    prob = w.small_2d(n=N_POINTS)
    X, y, psi_true = prob.X.astype(np.float64), prob.y.astype(np.float64), prob.psi_true
    p = len(psi_true)

    def log_post(psi):
        return (oracle.log_marginal_likelihood(X, y, psi)
                - 0.5 * float(np.sum((psi - psi_true) ** 2)))

    from scipy.optimize import minimize
    mode = minimize(lambda t: -log_post(t), psi_true, method="BFGS").x
    h = 1e-4
    H = np.zeros((p, p))
    for i in range(p):
        for j in range(p):
            ei, ej = np.eye(p)[i] * h, np.eye(p)[j] * h
            H[i, j] = (log_post(mode + ei + ej) - log_post(mode + ei - ej)
                       - log_post(mode - ei + ej) + log_post(mode - ei - ej)) / (4 * h * h)
    Sigma = np.linalg.inv(-H)
    L = np.linalg.cholesky(Sigma)

    rng = np.random.default_rng(20150501)
    c = 2.38 ** 2 / p
    psi, lp = mode.copy(), log_post(mode)
    samples = np.zeros((ITERS - ADAPT, p))
    acc_window, acc_kept = 0, 0
    for it in range(ITERS):
        prop = psi + np.sqrt(c) * (L @ rng.standard_normal(p))
        lp_prop = log_post(prop)
        if np.log(rng.uniform()) < lp_prop - lp:
            psi, lp = prop, lp_prop
            if it < ADAPT:
                acc_window += 1
            else:
                acc_kept += 1
        if it < ADAPT and (it + 1) % 500 == 0:
            c *= max(0.5, min(2.0, (acc_window / 500) / 0.3))
            acc_window = 0
        if it >= ADAPT:
            samples[it - ADAPT] = psi
    acc = acc_kept / (ITERS - ADAPT)
    mean = samples.mean(axis=0)
    sd = samples.std(axis=0, ddof=1)
    bm = samples.reshape(BATCHES, -1, p)
    se_mean = bm.mean(axis=1).std(axis=0, ddof=1) / np.sqrt(BATCHES)
    se_sd = bm.std(axis=1, ddof=1).std(axis=0, ddof=1) / np.sqrt(BATCHES)
    fmt = lambda v: " ".join("%.10g" % x for x in np.ravel(v))  # noqa: E731
    with open(OUT, "w") as f:
        f.write("# Posterior of the 2-D workload (n = %d, seed %d) under psi ~ N(psi_true, I), by\n"
                "# Metropolis-Hastings with the oracle's exact log marginal likelihood (Sec. 5's\n"
                "# comparison): %d iterations, adaptive scale during the first %d (then discarded),\n"
                "# moments of the last %d with Monte Carlo standard errors from %d batch means.\n"
                "# Written by tests/golden/make_mh_posterior.py (calls only oracle/ and the input\n"
                "# generator).  Coordinates: log l_1, log l_2, log sigma^2, log lambda.\n"
                % (N_POINTS, prob.seed, ITERS, ADAPT, ITERS - ADAPT, BATCHES))
        f.write("n = %d\n" % N_POINTS)
        f.write("psi_true = %s\n" % fmt(psi_true))
        f.write("mode = %s\n" % fmt(mode))
        f.write("sigma_laplace = %s\n" % fmt(Sigma))
        f.write("acceptance = %.4f\n" % acc)
        f.write("proposal_scale = %.6g\n" % c)
        f.write("mean = %s\n" % fmt(mean))
        f.write("sd = %s\n" % fmt(sd))
        f.write("se_mean = %s\n" % fmt(se_mean))
        f.write("se_sd = %s\n" % fmt(se_sd))
    print(open(OUT).read())


if __name__ == "__main__":
    main()
