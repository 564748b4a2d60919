"""Pins of the refinement and normal-equation oracles."""
import numpy as np
import pytest
import scipy.linalg as sl

from oracle import householder as hh
from oracle import normal
from oracle import refine


def conditioned(M, N, kappa, seed):
    g = np.random.default_rng(seed)
    U, _ = np.linalg.qr(g.standard_normal((M, N)))
    W, _ = np.linalg.qr(g.standard_normal((N, N)))
    A = (U * np.logspace(0, -np.log10(kappa), N)) @ W.T
    b = A @ g.standard_normal(N) + g.standard_normal(M)
    return A, b


def f32_factor_ops(A):
    """QR factors computed in float32 arithmetic (numpy's float32 LAPACK)."""
    A32 = A.astype(np.float32)
    Q, R = np.linalg.qr(A32, mode="complete")
    N = A.shape[1]
    R = R[:N].astype(np.float32)
    Q = Q.astype(np.float32)
    return (lambda f: (Q.T @ f.astype(np.float32)).astype(np.float64),
            lambda y: (Q @ y.astype(np.float32)).astype(np.float64),
            lambda c: sl.solve_triangular(R, c.astype(np.float32)).astype(np.float64),
            lambda g: sl.solve_triangular(R.T, g.astype(np.float32), lower=True).astype(np.float64),
            R)


def test_exact_factors_one_step_is_exact():
    A, b = conditioned(60, 8, 1e3, 1)
    f = hh.qr(A)
    x_star = np.linalg.lstsq(A, b, rcond=None)[0]
    x0 = x_star + 1e-3
    x, r, _ = refine.refine(A, b, x0, lambda v: hh.apply_qt(f, v), lambda v: hh.apply_q(f, v),
                            lambda c: hh.back_substitute(f.R, c),
                            lambda g: hh.forward_substitute_rt(f.R, g), steps=1)
    np.testing.assert_allclose(x, x_star, rtol=1e-11)
    np.testing.assert_allclose(r, b - A @ x_star, atol=1e-11)


@pytest.mark.parametrize("kappa", [1e2, 1e4])
def test_float32_factors_converge(kappa):
    A, b = conditioned(300, 30, kappa, 2)
    A = A.astype(np.float32).astype(np.float64)
    b = b.astype(np.float32).astype(np.float64)
    x_star = np.linalg.lstsq(A, b, rcond=None)[0]
    qt, q, sr, srt, R = f32_factor_ops(A)
    x0 = sr(qt(b)[:30])
    e0 = np.linalg.norm(x0 - x_star) / np.linalg.norm(x_star)
    x1, _, _ = refine.refine(A, b, x0, qt, q, sr, srt, steps=1)
    x2, _, _ = refine.refine(A, b, x0, qt, q, sr, srt, steps=2)
    e1 = np.linalg.norm(x1 - x_star) / np.linalg.norm(x_star)
    e2 = np.linalg.norm(x2 - x_star) / np.linalg.norm(x_star)
    assert e1 < 0.1 * e0 or e1 < 1e-12
    assert e2 <= e1 * 1.01 + 1e-13
    assert e2 < 1e-7


def test_cholesky_matches_library():
    g = np.random.default_rng(3)
    X = g.standard_normal((20, 6))
    G = X.T @ X + np.eye(6)
    L = normal.cholesky(G)
    np.testing.assert_allclose(L, np.linalg.cholesky(G), rtol=1e-12)
    np.testing.assert_allclose(L @ L.T, G, rtol=1e-13)


def test_normal_solve_matches_lstsq():
    g = np.random.default_rng(4)
    J = g.standard_normal((40, 6))
    b = g.standard_normal(40)
    D = np.abs(g.standard_normal(6)) + 0.1
    lam = 0.3
    A = np.vstack([J, np.sqrt(lam) * np.diag(D)])
    rhs = np.concatenate([b, np.zeros(6)])
    np.testing.assert_allclose(normal.solve(J, b, D, lam), np.linalg.lstsq(A, rhs, rcond=None)[0],
                               rtol=1e-11)


def test_float32_cholesky_loses_squared_condition():
    """The conditioning loss the Cholesky comparison path is meant to show (Sec. 1)."""
    A, b = conditioned(200, 20, 1e3, 5)
    A = A.astype(np.float32).astype(np.float64)
    b = b.astype(np.float32).astype(np.float64)
    D = np.ones(20)
    x_star = normal.solve(A, b, D, 0.0)
    x32 = normal.solve(A, b, D, 0.0, dtype=np.float32)
    e = np.linalg.norm(x32 - x_star) / np.linalg.norm(x_star)
    assert e > 1e-4   # kappa^2 u32 ~ 6e-2 scale, far above kappa u32 ~ 6e-5
