"""Damping-policy MLP in float64 (test infrastructure only).

Not in the paper: a small network that proposes the next LM damping (the lambda control of
Sec. 2 / Sec. 5.2 is otherwise Nielsen's rule).  Definition, written out plainly:

  x (F = 16 features) -> h1 = relu(W1 x + b1) (64) -> h2 = relu(W2 h1 + b2) (64)
                      -> z = W3 h2 + b3 (C = 8 logits over a grid of lambda multipliers)
  loss = mean over samples of -log softmax(z)[label]      (softmax cross-entropy)
  Adam (Kingma & Ba 2015): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
  p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Parameters are one flat vector [W1 (64 x 16) | b1 | W2 (64 x 64) | b2 | W3 (8 x 64) | b3], row-major.
The GPU keeps the weight matrices in bfloat16 (biases in float32) for the forward and backward
passes; `bf16_round` gives the same rounding (round to nearest, ties to even, of the float32
value to 8 significant bits) so that the oracle can evaluate the same network in float64.

Pins (tests/test_oracle_mlp.py): gradients against central finite differences, the loss of a
zero network (log C), Adam's first step (|step| = lr per coordinate), bf16 rounding of
exactly representable values, ties and the largest finite values.
"""
from __future__ import annotations

import numpy as np

F, H, C = 16, 64, 8
SIZES = [("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (C, H)), ("b3", (C,))]
P = sum(int(np.prod(s)) for _, s in SIZES)


def unflatten(theta):
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def flatten(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def bf16_round(x):
    """float32 -> nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32).copy()
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def working_weights(theta):
    """The weights the GPU evaluates: matrices rounded to bfloat16, biases kept (float32)."""
    p = unflatten(theta)
    for name in ("W1", "W2", "W3"):
        p[name] = bf16_round(p[name])
    for name in ("b1", "b2", "b3"):
        p[name] = np.asarray(p[name], dtype=np.float32).astype(np.float64)
    return p


def forward(p, X):
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ p["W3"].T + p["b3"]
    return z, (X, a1, h1, a2, h2)


def loss_and_grad(p, X, labels):
    """Mean softmax cross-entropy and its gradient with respect to every parameter."""
    z, (X, a1, h1, a2, h2) = forward(p, X)
    n = X.shape[0]
    zmax = z.max(axis=1, keepdims=True)
    e = np.exp(z - zmax)
    sm = e / e.sum(axis=1, keepdims=True)
    lab = np.asarray(labels, dtype=np.int64)
    loss = float(np.mean(-np.log(sm[np.arange(n), lab])))
    dz = sm.copy()
    dz[np.arange(n), lab] -= 1.0
    dz /= n
    g = {"W3": dz.T @ h2, "b3": dz.sum(axis=0)}
    dh2 = (dz @ p["W3"]) * (a2 > 0)
    g["W2"], g["b2"] = dh2.T @ h1, dh2.sum(axis=0)
    dh1 = (dh2 @ p["W2"]) * (a1 > 0)
    g["W1"], g["b1"] = dh1.T @ X, dh1.sum(axis=0)
    return loss, g


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step on flat vectors; t is the 1-based step count.  Returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
