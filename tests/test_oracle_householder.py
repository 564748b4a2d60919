"""Pins of the dense Householder oracle (Sec. 2) against hand-derived values and mathematics."""
import json
import os

import numpy as np
import pytest

from oracle import householder as hh

GOLD = os.path.join(os.path.dirname(__file__), "golden", "householder_worked.json")
U64 = np.finfo(np.float64).eps


def gold():
    with open(GOLD) as f:
        return json.load(f)


def test_reflector_worked_examples():
    for case in gold()["reflector"]:
        v, tau, beta = hh.house(np.array(case["x"]))
        assert beta == pytest.approx(case["beta"], abs=1e-15)
        assert tau == pytest.approx(case["tau"], abs=1e-15)
        np.testing.assert_allclose(v, case["v"], atol=1e-15)
        x = np.array(case["x"])
        hx = x - tau * v * np.dot(v, x)
        e = np.zeros_like(x)
        e[0] = case["beta"]
        np.testing.assert_allclose(hx, e, atol=1e-14)


def test_qr_worked_examples():
    for case in gold()["qr"]:
        f = hh.qr(np.array(case["A"]))
        np.testing.assert_allclose(f.R, case["R"], atol=1e-14)


@pytest.mark.parametrize("M,N", [(2, 1), (3, 2), (5, 3), (8, 5), (8, 8), (40, 17)])
def test_qr_brute_force_properties(M, N):
    g = np.random.default_rng(M * 100 + N)
    A = g.standard_normal((M, N))
    f = hh.qr(A)
    Q = hh.q_explicit(f)
    nA = np.linalg.norm(A)
    tol = 10 * M * U64
    assert np.linalg.norm(Q.T @ Q - np.eye(M)) <= tol
    assert np.all(np.tril(f.R, -1) == 0.0)
    Rfull = np.vstack([f.R, np.zeros((M - N, N))])
    assert np.linalg.norm(Q @ Rfull - A) <= tol * nA
    # Q^T A = [R; 0] through the implicit object
    np.testing.assert_allclose(hh.apply_qt(f, A), Rfull, atol=tol * nA)
    # library routine, up to row signs
    R_np = np.linalg.qr(A, mode="r")
    np.testing.assert_allclose(hh.normalise_row_signs(f.R), hh.normalise_row_signs(R_np),
                               atol=tol * nA)
    # apply_q inverts apply_qt
    B = g.standard_normal((M, 3))
    np.testing.assert_allclose(hh.apply_q(f, hh.apply_qt(f, B)), B, atol=tol * 10)


def test_lstsq_matches_library():
    g = np.random.default_rng(7)
    A = g.standard_normal((30, 7))
    b = g.standard_normal(30)
    x, f, qtb = hh.lstsq(A, b)
    x_np = np.linalg.lstsq(A, b, rcond=None)[0]
    np.testing.assert_allclose(x, x_np, rtol=1e-12, atol=1e-13)
    # Parseval: ||b||^2 = ||Q^T b||^2; bottom part = residual norm
    assert np.dot(qtb, qtb) == pytest.approx(np.dot(b, b), rel=1e-13)
    r = b - A @ x
    assert np.linalg.norm(qtb[7:]) == pytest.approx(np.linalg.norm(r), rel=1e-12)


def test_triangular_solves():
    g = np.random.default_rng(8)
    R = np.triu(g.standard_normal((9, 9))) + 5 * np.eye(9)
    c = g.standard_normal(9)
    np.testing.assert_allclose(hh.back_substitute(R, c), np.linalg.solve(R, c), rtol=1e-13)
    np.testing.assert_allclose(hh.forward_substitute_rt(R, c), np.linalg.solve(R.T, c), rtol=1e-13)


def test_compact_wy_equals_reflector_product():
    g = np.random.default_rng(9)
    A = g.standard_normal((12, 5))
    f = hh.qr(A)
    T = hh.compact_wy_T(f.V, f.tau)
    assert np.all(np.tril(T, -1) == 0.0)
    Q_wy = np.eye(12) - f.V @ T @ f.V.T
    np.testing.assert_allclose(Q_wy, hh.q_explicit(f), atol=1e-14)
    # the paper's update form A' = A + Y (T'^T (Y^T A)) with T' = -T equals Q^T A
    C = g.standard_normal((12, 4))
    np.testing.assert_allclose(C + f.V @ ((-T).T @ (f.V.T @ C)), hh.apply_qt(f, C), atol=1e-13)


def test_zero_column_is_identity_reflector():
    A = np.array([[0.0, 1.0], [0.0, 2.0], [0.0, 3.0]])
    f = hh.qr(A)
    assert f.tau[0] == 0.0
    Q = hh.q_explicit(f)
    np.testing.assert_allclose(Q @ np.vstack([f.R, [[0, 0]]]), A, atol=1e-14)


def test_planted_mistake_wrong_tau_is_caught(monkeypatch):
    """A dropped factor of 2 in tau (H no longer orthogonal) fails the Q^T Q = I pin."""
    real = hh.house

    def bad(x):
        v, tau, beta = real(x)
        return v, tau / 2.0, beta
    monkeypatch.setattr(hh, "house", bad)
    A = np.random.default_rng(1).standard_normal((6, 3))
    f = hh.qr(A)
    Q = hh.q_explicit(f)
    assert np.linalg.norm(Q.T @ Q - np.eye(6)) > 1e-3


def test_planted_mistake_reversed_q_order_is_caught(monkeypatch):
    """Applying the reflectors of Q in Q^T's order breaks Q R = A."""
    monkeypatch.setattr(hh, "apply_q", lambda f, B: hh.apply_qt(f, B))
    A = np.random.default_rng(2).standard_normal((6, 3))
    f = hh.qr(A)
    Q = hh.q_explicit(f)
    Rfull = np.vstack([f.R, np.zeros((3, 3))])
    assert np.linalg.norm(Q @ Rfull - A) > 1e-3


def test_lstsq_stack_equals_per_block_lstsq():
    """The stack-vectorised solve is the per-block Householder solve, block by block,
    including a block with a zero column in the middle (tau = 0) and square blocks."""
    g = np.random.default_rng(31)
    for K, M, N in ((50, 9, 4), (20, 6, 6), (40, 16, 1), (30, 3, 2)):
        A = g.standard_normal((K, M, N)) * 10.0 ** g.uniform(-2, 2, size=(K, 1, N))
        b = g.standard_normal((K, M))
        xs = hh.lstsq_stack(A, b)
        for k in range(K):
            np.testing.assert_allclose(xs[k], hh.lstsq(A[k], b[k])[0], rtol=1e-12, atol=1e-13)
    # a zero first column below the diagonal only: the reflector is the identity's sign flip
    A = np.array([[[2.0, 1.0], [0.0, 1.0], [0.0, 3.0]]])
    np.testing.assert_allclose(hh.lstsq_stack(A, np.array([[1.0, 2.0, 3.0]]))[0],
                               np.linalg.lstsq(A[0], [1.0, 2.0, 3.0], rcond=None)[0], rtol=1e-14)


def test_lstsq_stack_planted_mistakes_fail():
    """Copies of lstsq_stack with a planted mistake (the 2 of tau = 2 / v^T v dropped; the
    reflector not applied to b) disagree with the per-block lstsq."""
    g = np.random.default_rng(32)
    A = g.standard_normal((30, 8, 3))
    b = g.standard_normal((30, 8))
    ref = np.stack([hh.lstsq(A[k], b[k])[0] for k in range(30)])
    np.testing.assert_allclose(hh.lstsq_stack(A, b), ref, rtol=1e-12, atol=1e-13)

    def planted(A, b, tau_factor, apply_to_b):
        A = np.array(A, dtype=np.float64, copy=True)
        c = np.array(b, dtype=np.float64, copy=True)
        K, M, N = A.shape
        for k in range(N):
            x = A[:, k:, k]
            norm = np.sqrt(np.einsum("ki,ki->k", x, x))
            beta = np.where(x[:, 0] >= 0.0, -norm, norm)
            v = x.copy()
            v[:, 0] = x[:, 0] - beta
            v = v / v[:, :1]
            tau = tau_factor / np.einsum("ki,ki->k", v, v)
            if k + 1 < N:
                w = np.einsum("ki,kij->kj", v, A[:, k:, k + 1:])
                A[:, k:, k + 1:] -= tau[:, None, None] * v[:, :, None] * w[:, None, :]
            A[:, k, k] = beta
            if apply_to_b:
                c[:, k:] -= (tau * np.einsum("ki,ki->k", v, c[:, k:]))[:, None] * v
        xs = np.zeros((K, N))
        for i in reversed(range(N)):
            xs[:, i] = (c[:, i] - np.einsum("kj,kj->k", A[:, i, i + 1:N], xs[:, i + 1:])) / A[:, i, i]
        return xs
    np.testing.assert_allclose(planted(A, b, 2.0, True), ref, rtol=1e-12, atol=1e-13)
    assert not np.allclose(planted(A, b, 1.0, True), ref, rtol=1e-6)
    assert not np.allclose(planted(A, b, 2.0, False), ref, rtol=1e-6)
