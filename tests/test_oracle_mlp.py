"""Pins of the damping-policy MLP oracle (float64): gradients by finite differences, closed
forms of the loss and of Adam's first step, bfloat16 rounding against its definition and
against torch's conversion."""
import numpy as np
import pytest

from oracle import mlp


def random_net(seed):
    g = np.random.default_rng(seed)
    return g.standard_normal(mlp.P) * 0.3


def test_gradient_matches_central_differences():
    g = np.random.default_rng(1)
    theta = random_net(2)
    X = g.standard_normal((7, mlp.F))
    lab = g.integers(0, mlp.C, size=7)
    loss, grad = mlp.loss_and_grad(mlp.unflatten(theta), X, lab)
    gflat = mlp.flatten(grad)
    h = 1e-6
    for idx in g.choice(mlp.P, size=60, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[idx] += h
        tm[idx] -= h
        lp, _ = mlp.loss_and_grad(mlp.unflatten(tp), X, lab)
        lm_, _ = mlp.loss_and_grad(mlp.unflatten(tm), X, lab)
        fd = (lp - lm_) / (2 * h)
        assert abs(fd - gflat[idx]) <= 1e-6 * max(1.0, abs(fd)), idx


def test_zero_network_loss_is_log_classes():
    X = np.random.default_rng(3).standard_normal((5, mlp.F))
    loss, grad = mlp.loss_and_grad(mlp.unflatten(np.zeros(mlp.P)), X, np.arange(5) % mlp.C)
    assert loss == pytest.approx(np.log(mlp.C), rel=1e-15)
    # with all logits equal the output bias gradient is mean(softmax - onehot) = 1/C - frequency
    freq = np.bincount(np.arange(5) % mlp.C, minlength=mlp.C) / 5.0
    np.testing.assert_allclose(grad["b3"], 1.0 / mlp.C - freq, atol=1e-15)


def test_adam_first_step_has_size_lr():
    g = np.random.default_rng(4).standard_normal(50)
    theta, m, v = mlp.adam_step(np.zeros(50), g, np.zeros(50), np.zeros(50), 1, lr=1e-3, eps=0.0)
    np.testing.assert_allclose(theta, -1e-3 * np.sign(g), rtol=1e-12)


def test_bf16_round_definition():
    exact = np.array([1.0, 0.5, -2.0, 1.0 + 2 ** -7, 3.0, 0.0], dtype=np.float32)
    np.testing.assert_array_equal(mlp.bf16_round(exact), exact.astype(np.float64))
    # halfway cases go to the even neighbour; anything above halfway rounds up
    assert mlp.bf16_round(np.float32(1.0 + 2 ** -8)) == 1.0
    assert mlp.bf16_round(np.float32(1.0 + 3 * 2 ** -8)) == 1.0 + 2 ** -6
    assert mlp.bf16_round(np.float32(1.0 + 2 ** -8 + 2 ** -20)) == 1.0 + 2 ** -7


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    x = (np.random.default_rng(5).standard_normal(10000) * 10.0 ** np.random.default_rng(6).uniform(-6, 6, 10000))
    x = x.astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16_round(x), ref)


def test_adam_training_reduces_loss():
    g = np.random.default_rng(7)
    X = g.standard_normal((64, mlp.F))
    lab = (X[:, 0] > 0).astype(np.int64) * 3
    theta = random_net(8) * 0.3
    m = np.zeros(mlp.P)
    v = np.zeros(mlp.P)
    l0, _ = mlp.loss_and_grad(mlp.unflatten(theta), X, lab)
    for t in range(1, 101):
        _, gr = mlp.loss_and_grad(mlp.unflatten(theta), X, lab)
        theta, m, v = mlp.adam_step(theta, mlp.flatten(gr), m, v, t, lr=1e-2)
    l1, _ = mlp.loss_and_grad(mlp.unflatten(theta), X, lab)
    assert l1 < 0.2 * l0
