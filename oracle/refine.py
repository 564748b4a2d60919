"""Augmented-system iterative refinement of a least-squares solution (test infrastructure only).

Not in the paper: its goal (Sec. 1, Sec. 7) is single-precision QR that keeps the
accuracy of double; the textbook way to recover the last digits from low-precision QR
factors is Bjorck's refinement of the augmented system (Bjorck 1967)

    [ I   A ] [r]   [b]
    [ A^T 0 ] [x] = [0]

with residuals in high precision and corrections through the QR factors A = Q [R; 0]:
    f = b - r - A x,  g = -A^T r                  (high precision)
    [f1; f2] = Q^T f,  h = R^{-T} g,  dx = R^{-1} (f1 - h),  dr = Q [h; f2]
    x += dx,  r += dr.

`refine` runs these steps with caller-supplied solvers, so the test can feed it factors
computed in float32 (emulating the GPU's precision) while every residual is float64.
Pins (tests/test_oracle_refine.py): with exact factors one step reproduces the exact
solution; with float32 factors the error falls by orders of magnitude per step on
problems with condition number 1e4 while plain refinement stalls.
"""
from __future__ import annotations

import numpy as np


def refine(A, b, x0, apply_qt, apply_q, solve_r, solve_rt, steps=1):
    """Bjorck refinement.  A dense (float64), x0 initial solution; returns (x, r, history)."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    x = np.asarray(x0, dtype=np.float64).copy()
    N = A.shape[1]
    r = b - A @ x
    hist = []
    for _ in range(steps):
        f = b - r - A @ x
        g = -(A.T @ r)
        qf = apply_qt(f)
        f1, f2 = qf[:N], qf[N:]
        h = solve_rt(g)
        dx = solve_r(f1 - h)
        dr = apply_q(np.concatenate([h, f2]))
        x = x + dx
        r = r + dr
        hist.append(float(np.linalg.norm(dx)))
    return x, r, hist
