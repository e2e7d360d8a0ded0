"""FP64 oracle of the learned warm start (test infrastructure only; see oracle/__init__.py).

The solver may start the K s = y solve from any s_0 that does not depend on the current
step's random draws (Algorithm 1 takes s_0 as an input; the ULISSE estimate stays unbiased
for K^{-1} y).  The warm start proposes s_0 = K_s(X, Z) c with c = MLP(psi) and Z a fixed
set of anchor inputs:

    z  = (psi - mu) / sd                      (standardisation from the training pairs)
    h1 = tanh(z W1 + b1),  h2 = tanh(h1 W2 + b2),  c = h2 W3 + b3

What decides how long the y solve runs is its initial residual e_0 = y - K s_0 (Algorithm
1; the early stop of Sec. 4 compares ||e_i|| with q sqrt(n)).  Each pair the chain records
at its parameters psi_t carries m row indices I_t drawn uniformly with replacement and
M_t = K(X_{I_t}, X; psi_t) K_s(X, Z; psi_t), the rows I_t of K applied to the anchor
columns, so that y_{I_t} - M_t c is the initial residual on those rows.  The loss is

    loss = 1/T sum_t ( 1/m || y_{I_t} - M_t c_t ||^2 + rho || c_t ||^2 ),

an unbiased estimate (up to the ridge term) of the mean squared initial residual per
input.  Weights are stored row-major with inputs along rows (W1: p x H, W2: H x H,
W3: H x A), and flattened in the order W1, b1, W2, b2, W3, b3.

Everything here is plain numpy in float64; the backward pass is written out by hand and
pinned against central finite differences in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import numpy as np

from . import cross_signal, kmv_rows


def shapes(p, hidden, n_anchors):
    return [(p, hidden), (hidden,), (hidden, hidden), (hidden,), (hidden, n_anchors),
            (n_anchors,)]


def unflatten(w, p, hidden, n_anchors):
    out, k = [], 0
    for shp in shapes(p, hidden, n_anchors):
        size = int(np.prod(shp))
        out.append(np.asarray(w[k:k + size], dtype=np.float64).reshape(shp))
        k += size
    assert k == len(w)
    return out


def flatten(parts):
    return np.concatenate([np.asarray(a, dtype=np.float64).ravel() for a in parts])


def forward(w_flat, Psi, mu, sd, p, hidden, n_anchors):
    """c for every row of Psi (T x p); also returns the activations for the backward pass."""
    W1, b1, W2, b2, W3, b3 = unflatten(w_flat, p, hidden, n_anchors)
    Z = (np.asarray(Psi, dtype=np.float64) - mu) / sd
    H1 = np.tanh(Z @ W1 + b1)
    H2 = np.tanh(H1 @ W2 + b2)
    C = H2 @ W3 + b3
    return C, (Z, H1, H2)


def residual_matrices(X, Rows, Zanch, Psi):
    """M_t = K(X_{I_t}, X; psi_t) K_s(X, Z; psi_t) for every pair t, shape (T, m, A)."""
    return np.stack([kmv_rows(X, psi, cross_signal(X, Zanch, psi), rows)
                     for psi, rows in zip(np.asarray(Psi), np.asarray(Rows))])


def loss_and_grad(w_flat, Psi, Rows, X, y, Zanch, mu, sd, hidden, ridge, M=None):
    """The warm-start loss over the pairs (Psi[t], Rows[t]) and its gradient in the weights.
    M (the residual matrices) may be passed in to avoid recomputing them."""
    Psi = np.asarray(Psi, dtype=np.float64)
    T, p = Psi.shape
    M = residual_matrices(X, Rows, Zanch, Psi) if M is None else M
    m, n_anchors = M.shape[1], M.shape[2]
    W1, b1, W2, b2, W3, b3 = unflatten(w_flat, p, hidden, n_anchors)
    C, (Z, H1, H2) = forward(w_flat, Psi, mu, sd, p, hidden, n_anchors)
    Y = np.asarray(y, dtype=np.float64)[np.asarray(Rows)]
    R = Y - np.einsum("tma,ta->tm", M, C)
    loss = float((np.sum(R * R) / m + ridge * np.sum(C * C)) / T)
    dC = (-2.0 * np.einsum("tma,tm->ta", M, R) / m + 2.0 * ridge * C) / T
    dW3 = H2.T @ dC
    db3 = dC.sum(axis=0)
    dH2 = dC @ W3.T
    dA2 = dH2 * (1.0 - H2 * H2)
    dW2 = H1.T @ dA2
    db2 = dA2.sum(axis=0)
    dH1 = dA2 @ W2.T
    dA1 = dH1 * (1.0 - H1 * H1)
    dW1 = Z.T @ dA1
    db1 = dA1.sum(axis=0)
    return loss, flatten([dW1, db1, dW2, db2, dW3, db3])


def pooled_constant(M, Y, ridge):
    """The constant c minimising the loss over all pairs: the solution of the pooled normal
    equations (sum_t M_t^T M_t / (T m) + rho I) c = sum_t M_t^T y_t / (T m)."""
    T, m, A = M.shape
    G = np.einsum("tma,tmb->ab", M, M) / (T * m) + ridge * np.eye(A)
    rhs = np.einsum("tma,tm->a", M, Y) / (T * m)
    return np.linalg.solve(G, rhs)


def warm_start_vector(w_flat, psi, X, Zanch, mu, sd, hidden):
    """s_0 = K_s(X, Z; psi) MLP(psi) for all inputs X."""
    p = len(psi)
    n_anchors = Zanch.shape[0]
    C, _ = forward(w_flat, np.asarray(psi)[None, :], mu, sd, p, hidden, n_anchors)
    return cross_signal(X, Zanch, psi) @ C[0]
