"""Pins of Moré's two-factorization LM step (Sec. 5.2, Eq. LMTwoStep)."""
import numpy as np
import pytest

from oracle import more
from oracle import structured as st


def damped_lstsq(J, b, d, lam):
    A = np.vstack([J, np.sqrt(lam) * np.diag(d)])
    return np.linalg.lstsq(A, np.concatenate([b, np.zeros(J.shape[1])]), rcond=None)[0]


@pytest.mark.parametrize("M,N,lam", [(12, 5, 1e-3), (30, 8, 0.5), (9, 9, 2.0), (40, 3, 1e2)])
def test_step_equals_damped_least_squares(M, N, lam):
    g = np.random.default_rng(M * 100 + N)
    J = g.standard_normal((M, N)) * 10.0 ** g.uniform(-1, 1, size=N)
    b = g.standard_normal(M)
    d = np.linalg.norm(J, axis=0)
    p = more.step(J, b, d, lam)
    np.testing.assert_allclose(p, damped_lstsq(J, b, d, lam), rtol=1e-10, atol=1e-12)


def test_second_factor_reproduces_the_damped_gram_matrix():
    g = np.random.default_rng(3)
    J = g.standard_normal((20, 6))
    d = np.abs(g.standard_normal(6)) + 0.1
    lam = 0.3
    _, R2, _ = more.stage2(more.stage1(J, g.standard_normal(20)), d, lam)
    assert np.allclose(np.tril(R2, -1), 0.0)
    np.testing.assert_allclose(R2.T @ R2, J.T @ J + lam * np.diag(d * d), rtol=1e-12, atol=1e-12)


def test_zero_damping_is_plain_least_squares():
    g = np.random.default_rng(5)
    J = g.standard_normal((15, 4))
    b = g.standard_normal(15)
    p = more.step(J, b, np.ones(4), 0.0)
    np.testing.assert_allclose(p, np.linalg.lstsq(J, b, rcond=None)[0], rtol=1e-12, atol=1e-13)


def test_one_column_closed_form():
    g = np.random.default_rng(8)
    a = g.standard_normal(7)
    b = g.standard_normal(7)
    d, lam = 1.7, 0.4
    p = more.step(a[:, None], b, np.array([d]), lam)
    assert p[0] == pytest.approx(a @ b / (a @ a + lam * d * d), rel=1e-13)


def test_minimum_value_from_the_two_residuals():
    """min ||J p - b||^2 + lambda ||D p||^2 = stage-1 residual + stage-2 residual."""
    g = np.random.default_rng(11)
    J = g.standard_normal((25, 5))
    b = g.standard_normal(25)
    d = np.abs(g.standard_normal(5)) + 0.5
    lam = 0.8
    s1 = more.stage1(J, b)
    p, _, res2b = more.stage2(s1, d, lam)
    value = float(np.sum((J @ p - b) ** 2) + lam * np.sum((d * p) ** 2))
    assert value == pytest.approx(s1.res2 + res2b, rel=1e-12)


def test_interleave_order_is_a_permutation_pairing_rows():
    order = more.interleave_order(4)
    assert order.tolist() == [0, 4, 1, 5, 2, 6, 3, 7]


def test_blocks_match_the_composed_solve():
    g = np.random.default_rng(13)
    K = 30
    n = g.integers(2, 9, size=K)
    m = np.minimum(g.integers(1, 5, size=K), n)
    blocks = [g.standard_normal((int(n[i]), int(m[i]))) for i in range(K)]
    b = g.standard_normal(int(n.sum()))
    d = np.abs(g.standard_normal(int(m.sum()))) + 0.2
    lam = 0.05
    P = st.BlockProblem(blocks=blocks, b=b, lam=lam, D=d)
    p_ref, _ = st.factor_and_solve(P)
    np.testing.assert_allclose(more.block_steps(blocks, b, d, lam), p_ref, rtol=1e-10, atol=1e-12)


def test_planted_mistake_lambda_instead_of_its_root_fails(monkeypatch):
    g = np.random.default_rng(17)
    J = g.standard_normal((12, 4))
    b = g.standard_normal(12)
    d = np.ones(4)
    lam = 0.25
    monkeypatch.setattr(more, "damping_rows", lambda dd, ll: ll * np.asarray(dd, dtype=np.float64))
    p = more.step(J, b, d, lam)
    assert np.max(np.abs(p - damped_lstsq(J, b, d, lam))) > 1e-4
