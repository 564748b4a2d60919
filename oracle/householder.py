"""Dense Householder QR in float64 (test infrastructure only).

Follows Sec. 2 of the paper ("Background: QR decomposition"):
  * A = Q R with Q orthonormal and R upper triangular; economy Q is M x N, R is N x N,
    and the full-size Q_full = [Q | Q_perp], R_full = [R; 0]  (Eq. "Qfull").
  * A Householder matrix H = I - 2 v v^T with unit v zeroes a column below its first
    entry; R_full = H_{N-1} ... H_0 A = Q_full^T A.
  * Q is kept implicitly (the reflectors), and formed explicitly only by applying the
    implicit object to the identity.
  * The compact WY form writes a product of r reflectors as I + Y T Y^T with Y lower
    trapezoidal and T upper triangular (Schreiber and Van Loan).

Readings of the paper (listed with the rest of the readings in the design notes):
  * Sec. 2 names the matrix "n x m" with reflectors of size m x m; the dimension letters
    are swapped relative to the economy-size definition.  Here A is M x N with M >= N and
    there are N reflectors of size M.
  * A reflector is stored as v with v[0] = 1 and tau = 2 / (v^T v), so that
    H = I - tau v v^T is the paper's I - 2 u u^T with u = v / ||v||.
    beta = -sign(x0) ||x|| with sign(0) = +1; a zero column gives tau = 0 (H = I).
  * Compact WY sign: with T built forward and columnwise,
    H_0 H_1 ... H_{r-1} = I - Y T Y^T.  The paper's I + Y T Y^T is the same with T -> -T,
    and its update A + Y (T^T (Y^T A)) is our A - Y (T^T (Y^T A)).

Pins (tests/test_oracle_householder.py): worked 2-vector example (tests/golden),
Q^T Q = I, R upper triangular, Q R = A, agreement with numpy.linalg.qr up to row signs
and with numpy.linalg.lstsq, compact WY equals the explicit reflector product;
lstsq_stack equals lstsq block by block (zero columns included), and copies of it with a
planted mistake (tau without its 2, b not transformed) fail.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def house(x: np.ndarray):
    """Householder reflector for vector x (Sec. 2).

    Returns (v, tau, beta) with v[0] = 1 such that (I - tau v v^T) x = beta e_1.
    """
    x = np.asarray(x, dtype=np.float64)
    norm = float(np.sqrt(np.dot(x, x)))
    v = np.zeros_like(x)
    if norm == 0.0:
        v[0] = 1.0
        return v, 0.0, 0.0
    sign = 1.0 if x[0] >= 0.0 else -1.0
    beta = -sign * norm
    v[:] = x
    v[0] = x[0] - beta
    v = v / v[0]
    tau = 2.0 / float(np.dot(v, v))
    return v, tau, beta


@dataclass
class QRFactor:
    """Implicit Q (reflectors V, tau) and R of an M x N matrix, M >= N."""
    V: np.ndarray    # M x N, column k holds v_k in rows k..M-1 (V[k, k] = 1), zeros above
    tau: np.ndarray  # N
    R: np.ndarray    # N x N upper triangular

    @property
    def shape(self):
        return self.V.shape


def qr(A: np.ndarray) -> QRFactor:
    """Householder QR of A (M x N, M >= N): one reflector per column, in column order."""
    A = np.array(A, dtype=np.float64, copy=True)
    M, N = A.shape
    if M < N:
        raise ValueError("qr expects a portrait matrix (M >= N)")
    V = np.zeros((M, N))
    tau = np.zeros(N)
    for k in range(N):
        v, t, beta = house(A[k:, k])
        # apply H_k = I - t v v^T to the trailing columns
        if k + 1 < N:
            w = v @ A[k:, k + 1:]
            A[k:, k + 1:] -= t * np.outer(v, w)
        A[k, k] = beta
        A[k + 1:, k] = 0.0
        V[k:, k] = v
        tau[k] = t
    return QRFactor(V=V, tau=tau, R=np.triu(A[:N, :]))


def apply_qt(f: QRFactor, B: np.ndarray) -> np.ndarray:
    """Q_full^T B = H_{N-1} ... H_0 B (B has M rows; 1-D or 2-D)."""
    B = np.array(B, dtype=np.float64, copy=True)
    M, N = f.V.shape
    for k in range(N):
        v = f.V[k:, k]
        B[k:] -= f.tau[k] * np.multiply.outer(v, v @ B[k:])
    return B


def apply_q(f: QRFactor, B: np.ndarray) -> np.ndarray:
    """Q_full B = H_0 ... H_{N-1} B."""
    B = np.array(B, dtype=np.float64, copy=True)
    M, N = f.V.shape
    for k in reversed(range(N)):
        v = f.V[k:, k]
        B[k:] -= f.tau[k] * np.multiply.outer(v, v @ B[k:])
    return B


def q_explicit(f: QRFactor) -> np.ndarray:
    """Q_full (M x M) formed by applying the implicit Q to the identity (Sec. 2)."""
    M = f.V.shape[0]
    return apply_q(f, np.eye(M))


def back_substitute(R: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Solve R x = c for upper-triangular R by back-substitution (matrixR().solve, Sec. 5.1)."""
    R = np.asarray(R, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    N = R.shape[0]
    x = np.zeros(N)
    for i in reversed(range(N)):
        s = c[i] - np.dot(R[i, i + 1:], x[i + 1:])
        x[i] = s / R[i, i]
    return x


def forward_substitute_rt(R: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Solve R^T h = g for upper-triangular R (R^T is lower triangular)."""
    R = np.asarray(R, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    N = R.shape[0]
    h = np.zeros(N)
    for i in range(N):
        s = g[i] - np.dot(R[:i, i], h[:i])
        h[i] = s / R[i, i]
    return h


def lstsq(A: np.ndarray, b: np.ndarray):
    """Least-squares solve by QR (Sec. 5.1 usage: compute, Q^T b, R solve).

    Returns (x, factor, qtb).
    """
    f = qr(A)
    qtb = apply_qt(f, b)
    N = f.V.shape[1]
    x = back_substitute(f.R, qtb[:N])
    return x, f, qtb


def compact_wy_T(V: np.ndarray, tau: np.ndarray) -> np.ndarray:
    """T (r x r, upper) with H_0 H_1 ... H_{r-1} = I - V T V^T (Schreiber-Van Loan, Sec. 2).

    Built forward and columnwise: appending reflector j to the product I - V T V^T gives
    the new column [-tau_j T (V^T v_j); tau_j].
    """
    V = np.asarray(V, dtype=np.float64)
    r = V.shape[1]
    T = np.zeros((r, r))
    for j in range(r):
        T[j, j] = tau[j]
        if j > 0:
            z = V[:, :j].T @ V[:, j]
            T[:j, j] = -tau[j] * (T[:j, :j] @ z)
    return T


def normalise_row_signs(R: np.ndarray) -> np.ndarray:
    """R with each row multiplied by the sign of its diagonal (R is unique up to row signs)."""
    R = np.array(R, dtype=np.float64, copy=True)
    s = np.where(np.diag(R) < 0.0, -1.0, 1.0)
    return R * s[:, None]


def lstsq_stack(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    """lstsq for a stack of same-shape problems, A (K, M, N) and b (K, M); returns x (K, N).

    The same steps as house / qr / apply_qt / back_substitute (Sec. 2, Sec. 5.1), each numpy
    operation taken over the K problems at once so that a million small blocks solve in
    seconds: for each column k the reflector of A[:, k:, k] (v[0] = 1, beta = -sign(x0)||x||,
    tau = 2 / v^T v, tau = 0 for a zero column), applied to the trailing columns and to b,
    then back-substitution.  Pinned against lstsq block by block.
    """
    A = np.array(A, dtype=np.float64, copy=True)
    c = np.array(b, dtype=np.float64, copy=True)
    K, M, N = A.shape
    if M < N:
        raise ValueError("lstsq_stack expects portrait blocks (M >= N)")
    for k in range(N):
        x = A[:, k:, k]
        norm = np.sqrt(np.einsum("ki,ki->k", x, x))
        live = norm > 0.0
        beta = np.where(x[:, 0] >= 0.0, -norm, norm)
        v = x.copy()
        v[:, 0] = np.where(live, x[:, 0] - beta, 1.0)
        v = v / v[:, :1]
        tau = np.where(live, 2.0 / np.einsum("ki,ki->k", v, v), 0.0)
        if k + 1 < N:
            w = np.einsum("ki,kij->kj", v, A[:, k:, k + 1:])
            A[:, k:, k + 1:] -= tau[:, None, None] * v[:, :, None] * w[:, None, :]
        A[:, k, k] = np.where(live, beta, A[:, k, k])
        wc = np.einsum("ki,ki->k", v, c[:, k:])
        c[:, k:] -= (tau * wc)[:, None] * v
    xs = np.zeros((K, N))
    for i in reversed(range(N)):
        s = c[:, i] - np.einsum("kj,kj->k", A[:, i, i + 1:N], xs[:, i + 1:])
        xs[:, i] = s / A[:, i, i]
    return xs
