"""Normal equations, Eq. (1) of the paper, solved by Cholesky (test infrastructure only).

Eq. (1): (J^T J + lambda D^2) p = J^T b.  Its condition number is the square of that of
the augmented matrix of Eq. (2), which is the paper's reason to prefer QR (Sec. 1).
Used (a) as an independent cross-check of the QR solution on well-conditioned small
problems and (b) as the CPU counterpart of the FP32 Cholesky comparison path.

The Cholesky factorisation is the textbook column algorithm written out (L L^T = G);
the triangular solves are plain loops.  Pins (tests/test_oracle_normal.py): L L^T = G,
agreement with numpy.linalg.cholesky and numpy.linalg.solve.
"""
from __future__ import annotations

import numpy as np


def gram(J, D, lam):
    """G = J^T J + lambda D^2 and the rhs J^T b's matrix part (dense J)."""
    J = np.asarray(J, dtype=np.float64)
    return J.T @ J + lam * np.diag(np.asarray(D, dtype=np.float64) ** 2)


def cholesky(G, dtype=np.float64):
    """Lower-triangular L with L L^T = G, computed in `dtype` arithmetic (column algorithm)."""
    G = np.asarray(G, dtype=dtype)
    n = G.shape[0]
    L = np.zeros((n, n), dtype=dtype)
    for j in range(n):
        s = G[j, j] - np.dot(L[j, :j], L[j, :j])
        if not s > 0:
            raise np.linalg.LinAlgError("matrix is not positive definite")
        L[j, j] = np.sqrt(s)
        if j + 1 < n:
            L[j + 1:, j] = (G[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def solve_lower(L, y):
    n = L.shape[0]
    x = np.zeros(n, dtype=L.dtype)
    for i in range(n):
        x[i] = (y[i] - np.dot(L[i, :i], x[:i])) / L[i, i]
    return x


def solve_upper_lt(L, y):
    """Solve L^T x = y."""
    n = L.shape[0]
    x = np.zeros(n, dtype=L.dtype)
    for i in reversed(range(n)):
        x[i] = (y[i] - np.dot(L[i + 1:, i], x[i + 1:])) / L[i, i]
    return x


def solve(J, b, D, lam, dtype=np.float64):
    """p from Eq. (1) by Cholesky in `dtype` arithmetic (dense J; small problems)."""
    J = np.asarray(J, dtype=dtype)
    D = np.asarray(D, dtype=dtype)
    G = J.T @ J + dtype(lam) * np.diag(D * D)
    L = cholesky(G, dtype)
    rhs = J.T @ np.asarray(b, dtype=dtype)
    return solve_upper_lt(L, solve_lower(L, rhs)).astype(np.float64)
