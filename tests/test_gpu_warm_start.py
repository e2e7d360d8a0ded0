"""Learned warm start on the GPU (ulisse_ws_*): the training kernels against the FP64 oracle
(oracle/mlp.py), the warm start vector, unbiasedness of the gradient with the warm start on,
and what the trained network saves in CG iterations.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU runs deselect this module
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1501_05427_gb300 import ulisse as u  # noqa: E402
from paper_1501_05427_gb300 import workloads as w  # noqa: E402


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _ctx(prob, **cfg):
    X = torch.from_numpy(prob.X).cuda()
    y = torch.from_numpy(prob.y).cuda()
    return u.Context(X, y, u.ulisse_config_default(**cfg))


def _record(ctx, prob, n_pairs, scale=0.05, seed=0, step0=0):
    """Gradient steps with recording on, at parameters exactly representable in FP32 (the
    recorded copy of psi is FP32)."""
    rng = np.random.default_rng(seed)
    for k in range(n_pairs):
        psi = (prob.psi_true + scale * rng.standard_normal(prob.d + 2)).astype(np.float32)
        ctx.grad(psi.astype(np.float64), step=step0 + k)


def test_ws_loss_and_gradient_match_oracle(orc):
    from oracle import mlp
    prob = w.census_like(n=3000, seed=901)
    H, A, m = 32, 64, 200
    ridge = 1e-3
    with _ctx(prob, n_probes=4, seed=3) as ctx:
        ctx.ws_init(n_anchors=A, hidden=H, n_rows=m, max_pairs=16, seed=5, ridge=ridge)
        ctx.ws_set(record=True)
        _record(ctx, prob, 7)                         # < 8 pairs: nothing held out, so the
        ctx.ws_train(steps=20, batch=8, lr=1e-2)     # Adam steps move every layer
        st = ctx.ws_export()
        loss, g = ctx.ws_loss_grad()
    T = st["n_pairs"]
    assert T == 7
    rows = st["pair_rows"][:T]
    assert rows.min() >= 0 and rows.max() < prob.n and len(np.unique(rows)) > T * m // 2
    assert np.max(np.abs(mlp.unflatten(st["weights"], prob.d + 2, H, A)[4])) > 0
    Xd = prob.X.astype(np.float64)
    loss_ref, g_ref = mlp.loss_and_grad(
        st["weights"].astype(np.float64), st["pair_psi"][:T].astype(np.float64), rows, Xd,
        prob.y.astype(np.float64), Xd[st["anchors"]], st["mu"].astype(np.float64),
        st["sd"].astype(np.float64), H, ridge)
    assert abs(loss - loss_ref) <= 1e-4 * loss_ref
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    # every parameter block moved and carries gradient
    blocks = np.cumsum([0] + [int(np.prod(s)) for s in mlp.shapes(prob.d + 2, H, A)])
    for a, b in zip(blocks[:-1], blocks[1:]):
        assert np.linalg.norm(g_ref[a:b]) > 0


def test_ws_pooled_start_matches_oracle(orc):
    """With no Adam steps, training leaves the network at the pooled least-squares constant
    (Gram matrix, FP64 Cholesky and whitening on the GPU): its loss equals the oracle's
    minimum over constants and the output layer weights are zero."""
    from oracle import mlp
    prob = w.census_like(n=2500, seed=905)
    H, A, m, ridge = 32, 96, 160, 1e-2
    with _ctx(prob, n_probes=4, seed=3) as ctx:
        ctx.ws_init(n_anchors=A, hidden=H, n_rows=m, max_pairs=12, seed=4, ridge=ridge)
        ctx.ws_set(record=True)
        _record(ctx, prob, 12)
        ctx.ws_train(steps=0, batch=8)
        st = ctx.ws_export()
        loss, _ = ctx.ws_loss_grad()
    T = st["n_pairs"]
    Xd = prob.X.astype(np.float64)
    yd = prob.y.astype(np.float64)
    rows = st["pair_rows"][:T]
    Psi = st["pair_psi"][:T].astype(np.float64)
    M = mlp.residual_matrices(Xd, rows, Xd[st["anchors"]], Psi)
    c = mlp.pooled_constant(M, yd[rows], ridge)
    Wt = mlp.unflatten(st["weights"].astype(np.float64), prob.d + 2, H, A)
    assert np.max(np.abs(Wt[4])) == 0.0
    R = yd[rows] - M @ c
    loss_min = float(np.mean(np.sum(R * R, axis=1) / m) + ridge * c @ c)
    loss0 = float(np.mean(np.sum(yd[rows] ** 2, axis=1) / m))
    print("pooled start: loss %.6g, oracle minimum %.6g, at c = 0 %.6g" % (loss, loss_min, loss0))
    assert loss_min <= loss <= loss_min + 1e-3 * (loss0 - loss_min)
    assert np.linalg.norm(Wt[5] - c) <= 2e-2 * np.linalg.norm(c)


def test_ws_x0_matches_oracle(orc):
    from oracle import mlp
    prob = w.census_like(n=2000, seed=902)
    H, A = 32, 64
    with _ctx(prob, n_probes=4, seed=3) as ctx:
        ctx.ws_init(n_anchors=A, hidden=H, n_rows=128, max_pairs=8, seed=6)
        ctx.ws_set(record=True)
        _record(ctx, prob, 6)
        ctx.ws_train(steps=30, batch=6, lr=1e-2)
        st = ctx.ws_export()
        psi = prob.psi_true + 0.01
        x32 = ctx.ws_x0(psi, bf16=False).cpu().numpy().astype(np.float64)
        x16 = ctx.ws_x0(psi, bf16=True).cpu().numpy().astype(np.float64)
    Xd = prob.X.astype(np.float64)
    ref = mlp.warm_start_vector(st["weights"].astype(np.float64), psi, Xd, Xd[st["anchors"]],
                                st["mu"].astype(np.float64), st["sd"].astype(np.float64), H)
    assert np.linalg.norm(ref) > 0
    assert np.linalg.norm(x32 - ref) <= 1e-4 * np.linalg.norm(ref)
    # BF16 inference weights (8-bit mantissa): a guess, not an exact quantity
    assert np.linalg.norm(x16 - ref) <= 3e-2 * np.linalg.norm(ref)


def test_ws_training_lowers_the_loss():
    prob = w.census_like(n=4000, seed=903)
    with _ctx(prob, n_probes=4, seed=3) as ctx:
        ctx.ws_init(n_anchors=256, hidden=64, n_rows=512, max_pairs=64, seed=7)
        ctx.ws_set(record=True)
        _record(ctx, prob, 40)
        l0, _ = ctx.ws_loss_grad()
        ctx.ws_train(steps=300, batch=32, lr=3e-3)
        l1, _ = ctx.ws_loss_grad()
    print("warm-start loss: before training %.4g, after %.4g" % (l0, l1))
    # the span of the anchor columns bounds how far the initial residual can fall
    assert l1 < 0.8 * l0, (l0, l1)


def test_ws_gradient_stays_unbiased(orc):
    """With the warm start on, the y solve runs on the correction K^{-1}(y - K x0): the mean
    of 3000 seeded gradient estimates stays within 4 SE of the exact gradient."""
    prob = w.census_like(n=600, seed=61)
    g_exact = orc.exact_gradient(prob.X.astype(np.float64), prob.y.astype(np.float64),
                                 prob.psi_true)
    N = 3000
    with _ctx(prob, n_probes=2, q=0.7, max_iter=600, seed=123) as ctx:
        ctx.ws_init(n_anchors=128, hidden=64, n_rows=256, max_pairs=64, seed=8)
        ctx.ws_set(record=True)
        _record(ctx, prob, 40, step0=10_000)
        ctx.ws_train(steps=200, batch=32, lr=3e-3)
        ctx.ws_set(record=False, use=True)
        G = np.array([ctx.grad(prob.psi_true, step=s)[0] for s in range(N)])
    se = G.std(axis=0, ddof=1) / math.sqrt(N)
    z = (G.mean(axis=0) - g_exact) / se
    assert np.max(np.abs(z)) < 4.0, (G.mean(axis=0), g_exact, se)


def test_ws_saves_iterations_on_the_y_solve():
    """Train on pairs the chain records, then compare the y solve with and without the warm
    start at the same parameters, probes and uniforms."""
    prob = w.census_like(n=6000, seed=904)
    rng = np.random.default_rng(11)
    with _ctx(prob, n_probes=4, seed=9) as ctx:
        ctx.ws_init(n_anchors=512, hidden=256, n_rows=1024, max_pairs=256, seed=9)
        ctx.ws_set(record=True)
        psis = [prob.psi_true + 0.05 * rng.standard_normal(prob.d + 2) for _ in range(160)]
        for k, psi in enumerate(psis[:120]):
            ctx.grad(psi, step=k)
        loss = ctx.ws_train(steps=600, batch=64, lr=2e-3)
        it_off, it_on = [], []
        for k, psi in enumerate(psis[120:]):
            ctx.ws_set(record=False, use=False)
            _, st0 = ctx.grad(psi, step=1000 + k)
            ctx.ws_set(record=False, use=True)
            _, st1 = ctx.grad(psi, step=1000 + k)
            it_off.append(st0[0][1])
            it_on.append(st1[0][1])
    print("y-solve CG iterations: without warm start %.2f, with %.2f (last loss %.3g)"
          % (np.mean(it_off), np.mean(it_on), loss))
    assert np.mean(it_on) < 0.8 * np.mean(it_off)
