"""The learned per-bond rank predictor on the GPU.

Gradients of the library's FP32 backward kernels are compared with the FP64
oracle backpropagation (oracle/mlp.py, itself pinned by finite differences);
training must fit; a solve with the trained predictor must reach the same
optimum as the adaptive-SVD solve while rounding most bonds by the
predicted-rank range finder.
"""
import math
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2509_11890_gb300 as tg  # noqa: E402
from oracle import mlp, sdp_dense as sd  # noqa: E402
from paper_2509_11890_gb300 import inputs  # noqa: E402


def test_gradient_matches_oracle_backprop():
    p = tg.RankPredictor(seed=11)
    theta = p.params().astype(np.float64)
    g = inputs.rng(12, 41)
    X = g.uniform(-1, 1, (300, mlp.NIN)).astype(np.float32)
    t = g.uniform(0, 1, 300).astype(np.float32)
    loss, grad = p.grad(X, t)
    ref_loss, ref_grad = mlp.loss_and_grad(theta, X.astype(np.float64), t.astype(np.float64))
    assert math.isclose(loss, ref_loss, rel_tol=1e-5)
    assert np.linalg.norm(grad - ref_grad) <= 1e-4 * np.linalg.norm(ref_grad)
    # forward agrees too
    y = p.predict(X)
    np.testing.assert_allclose(y, mlp.forward(theta, X.astype(np.float64))[0], atol=1e-5)


def test_training_fits_a_smooth_target():
    g = inputs.rng(13, 42)
    X = g.uniform(-1, 1, (2048, mlp.NIN)).astype(np.float32)
    t = (0.5 + 0.3 * np.tanh(X[:, 4] - 0.5 * X[:, 6])).astype(np.float32)
    p = tg.RankPredictor(seed=3)
    l0, _ = p.grad(X, t)
    loss = p.train(X, t, epochs=60, batch=128, lr=3e-3, seed=5)
    assert loss < 0.05 * l0 and loss < 1e-3, (l0, loss)


def _solve(inst, pred=None, trace=False):
    ctx = tg.Context.maxcut(inst["adjacency_cores"], tg.default_options(rank_cap=16, max_iters=40))
    if trace:
        ctx.set_trace(True)
    if pred is not None:
        ctx.set_rank_predictor(pred)
    t0 = time.perf_counter()
    res = ctx.solve()
    dt = time.perf_counter() - t0
    info = ctx.newton_step()
    return ctx, res, info, dt


def test_trained_predictor_on_held_out_instances():
    # traces from the method itself on training instances (seeds 0-2), then
    # held-out instances (seeds 4-6): with the predictor every solve still
    # certifies the gap, most bonds are rounded by the predicted-rank range
    # finder, and the time-to-gap with and without it is recorded
    X, t = [], []
    for seed in (0, 1, 2):
        ctx, res, _, _ = _solve(inputs.maxcut_kron(6, seed), trace=True)
        assert res["status"] == 0
        x, y = ctx.trace()
        X.append(x)
        t.append(y)
    X, t = np.concatenate(X), np.concatenate(t)
    assert X.shape[1] == mlp.NIN and len(t) > 50 and np.all((t > 0) & (t <= 1))
    # the decay feature is filled once a variable has been rounded before
    assert np.any(X[:, 9] < 0)
    p = tg.RankPredictor(seed=7)
    loss = p.train(X, t, epochs=300, batch=64, lr=2e-3, seed=1)
    assert loss < 0.01, loss
    rows = []
    for seed in (4, 5, 6):
        inst = inputs.maxcut_kron(6, seed)
        ref = sd.solve_dense(sd.maxcut_sdp(inst["weights"]))
        _, base, _, t_base = _solve(inst)
        _, lrn, info, t_lrn = _solve(inst, pred=p)
        assert base["status"] == 0 and lrn["status"] == 0, (base, lrn)
        for r in (base, lrn):
            assert abs(r["pobj"] - ref.pobj) / (1 + abs(ref.pobj)) <= 2e-3
            assert r["rel_gap"] <= 1e-4 / np.sqrt(6)
        used, fb = info["pred_used"], info["pred_fallbacks"]
        assert used > 0 and fb <= used, (used, fb)
        rows.append((seed, t_base, t_lrn, used, fb))
    for seed, tb, tl, used, fb in rows:
        print(f"held-out seed {seed}: adaptive SVD {tb:.3f} s, predictor {tl:.3f} s (gain {tb / tl:.2f}x), "
              f"{used} bonds by range finder, {fb} fallbacks")
