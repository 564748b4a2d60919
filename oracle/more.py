"""Moré's two-factorization Levenberg-Marquardt step (Sec. 5.2, Eq. "LMTwoStep"), in float64.
Test infrastructure only: imported by the tests, never by the library.

Stage 1 factors the Jacobian alone, J = Q R (economy size), and keeps c = the top N entries of
Q^T b and the squared norm of the rest.  Stage 2, once per damping value, factors the vertical
concatenation [R; lambda^(1/2) D] = Q' R' with the damping row of column k placed right after
row k of R (the row interleave of Sec. 4.5, which turns the stack into a banded / skewed
triangular matrix) and solves R' p = top N entries of Q'^T [c; 0].  Since
||J p - b||^2 = ||R p - c||^2 + ||bottom of Q^T b||^2, this p minimises
||J p - b||^2 + lambda ||D p||^2 (Eq. 2) exactly as the single factorization of
[J; lambda^(1/2) D] does; only stage 2 is repeated when lambda changes.

For block-diagonal J both stages work block by block; stage 2 of block i factors the
2 m_i x m_i matrix [R_i; lambda^(1/2) D_i].

Pins (tests/test_oracle_more.py): the damped least-squares solution of numpy.linalg.lstsq on
[J; lambda^(1/2) D], R'^T R' = J^T J + lambda D^2, lambda = 0 gives the plain least-squares
solution, the one-column closed form a^T b / (a^T a + lambda d^2), the minimum value of the
damped objective from the two residual norms, the block version against the composed solve of
Sec. 4.1, and a planted mistake (lambda instead of lambda^(1/2)) that fails them.  The
trust-region lambda: its step's scaled length within sigma Delta of Delta, the lambda inside
the bracket an independent bisection on the assembled problem gives, the step equal to
numpy's damped least squares there, lambda = 0 when the Gauss-Newton step is shorter, and the
derivative of the length against central differences (a planted mistake in z fails it).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import householder as hh


@dataclass
class Stage1:
    R: np.ndarray        # N x N upper triangular
    c: np.ndarray        # top N entries of Q^T b
    res2: float          # ||bottom of Q^T b||^2 = min ||J p - b||^2


def stage1(J: np.ndarray, b: np.ndarray) -> Stage1:
    """J = Q R; c = top of Q^T b (Sec. 5.2, first factorization of Eq. LMTwoStep)."""
    J = np.asarray(J, dtype=np.float64)
    f = hh.qr(J)
    qtb = hh.apply_qt(f, np.asarray(b, dtype=np.float64))
    N = J.shape[1]
    return Stage1(R=f.R, c=qtb[:N], res2=float(qtb[N:] @ qtb[N:]))


def damping_rows(d: np.ndarray, lam: float) -> np.ndarray:
    """The diagonal of lambda^(1/2) D."""
    return np.sqrt(lam) * np.asarray(d, dtype=np.float64)


def interleave_order(N: int) -> np.ndarray:
    """Row order of [R; lambda^(1/2) D] after the interleave of Sec. 4.5: row k of R (source
    row k), then the damping row of column k (source row N + k)."""
    order = np.empty(2 * N, dtype=np.int64)
    order[0::2] = np.arange(N)
    order[1::2] = N + np.arange(N)
    return order


def stage2(s1: Stage1, d: np.ndarray, lam: float):
    """[R; lambda^(1/2) D] = Q' R' (rows interleaved), R' p = top of Q'^T [c; 0].

    Returns (p, R', res2') with res2' = ||bottom of Q'^T [c; 0]||^2."""
    N = s1.R.shape[0]
    A = np.vstack([s1.R, np.diag(damping_rows(d, lam))])
    rhs = np.concatenate([s1.c, np.zeros(N)])
    order = interleave_order(N)
    f = hh.qr(A[order])
    qt = hh.apply_qt(f, rhs[order])
    p = hh.back_substitute(f.R, qt[:N])
    return p, f.R, float(qt[N:] @ qt[N:])


def step(J: np.ndarray, b: np.ndarray, d: np.ndarray, lam: float) -> np.ndarray:
    """The damped least-squares step by the two factorizations."""
    return stage2(stage1(J, b), d, lam)[0]


def block_steps(blocks, b: np.ndarray, d: np.ndarray, lam: float) -> np.ndarray:
    """Block-diagonal J = blkdiag(J_i): both stages per block.  b and d are concatenated by
    block (rows n_i, columns m_i); returns p concatenated by block."""
    p, r0, c0 = [], 0, 0
    for Ji in blocks:
        n, m = Ji.shape
        s1 = stage1(Ji, b[r0:r0 + n])
        p.append(stage2(s1, d[c0:c0 + m], lam)[0])
        r0 += n
        c0 += m
    return np.concatenate(p)


# ---- Moré's trust-region choice of lambda (Sec. 5.2: the damping of the two-factorization LM
# step chosen so that the step has a given scaled length; Moré 1977, Hebden's iteration) ----

def tr_parts(s1_list, d_list, lam: float):
    """For the block-diagonal step p(lam): ||q|| with q = D p, ||z|| with z = R'^{-T} D q
    (R'^T R' = J^T J + lam D^2), and p.  d/dlam ||q|| = -||z||^2 / ||q||."""
    ps, q2, z2 = [], 0.0, 0.0
    for s1, d in zip(s1_list, d_list):
        p, Rp, _ = stage2(s1, d, lam)
        q = d * p
        # R'^T z = D q by forward substitution (R' upper triangular)
        z = hh.forward_substitute_rt(Rp, d * q)
        ps.append(p)
        q2 += float(q @ q)
        z2 += float(z @ z)
    return np.concatenate(ps), np.sqrt(q2), np.sqrt(z2)


def trust_region_lambda(blocks, b, d, delta: float, sigma: float = 0.1, max_iter: int = 30):
    """The lambda >= 0 whose damped step has scaled length ||D p(lambda)|| within sigma Delta of
    Delta, or lambda = 0 when the Gauss-Newton step is already that short (the trust-region
    subproblem).  Newton's method on 1/||D p|| - 1/Delta (nearly linear in lambda), kept inside
    a bracket [lo, hi] that every iterate narrows: lo from a Newton step of ||D p|| - Delta at 0
    (that function is convex and decreasing), hi = ||D^{-1} J^T b|| / Delta.  Returns
    (lambda, p, iterations)."""
    s1s, ds, r0, c0 = [], [], 0, 0
    g2 = 0.0
    for Ji in blocks:
        n, m = Ji.shape
        s1 = stage1(Ji, b[r0:r0 + n])
        di = np.asarray(d[c0:c0 + m], dtype=np.float64)
        gi = s1.R.T @ s1.c            # J_i^T b_i
        g2 += float(np.sum((gi / di) ** 2))
        s1s.append(s1)
        ds.append(di)
        r0 += n
        c0 += m
    p, qn, zn = tr_parts(s1s, ds, 0.0)
    phi = qn - delta
    if phi <= sigma * delta:
        return 0.0, p, 0
    lo = phi * qn / (zn * zn) if zn > 0 else 0.0
    hi = np.sqrt(g2) / delta
    lam = max(0.001 * hi, np.sqrt(lo * hi))
    for it in range(1, max_iter + 1):
        p, qn, zn = tr_parts(s1s, ds, lam)
        phi = qn - delta
        if abs(phi) <= sigma * delta:
            return lam, p, it
        if phi > 0:
            lo = max(lo, lam)
        else:
            hi = min(hi, lam)
        lam_new = lam + (qn / zn) ** 2 * (phi / delta)
        lam = lam_new if lo < lam_new < hi else max(0.001 * hi, np.sqrt(lo * hi))
    return lam, p, max_iter
