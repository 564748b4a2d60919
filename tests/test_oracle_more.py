"""Pins of Moré's two-factorization LM step (Sec. 5.2, Eq. LMTwoStep)."""
import numpy as np
import pytest

from oracle import householder as hh
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


# ---- Moré's trust-region lambda (Sec. 5.2, Moré 1977) ----

def tr_problem(seed):
    g = np.random.default_rng(seed)
    blocks = [g.standard_normal((int(g.integers(3, 9)), int(g.integers(1, 4)))) for _ in range(20)]
    n = sum(b.shape[0] for b in blocks)
    m = sum(b.shape[1] for b in blocks)
    b = g.standard_normal(n)
    J = np.zeros((n, m))
    r = c = 0
    for B in blocks:
        J[r:r + B.shape[0], c:c + B.shape[1]] = B
        r += B.shape[0]
        c += B.shape[1]
    d = np.sqrt((J * J).sum(0))
    return blocks, J, b, d


def scaled_length(J, b, d, lam):
    """||D p(lam)|| with p from numpy's least squares on the assembled [J; lam^(1/2) D]."""
    A = np.vstack([J, np.sqrt(lam) * np.diag(d)])
    p = np.linalg.lstsq(A, np.concatenate([b, np.zeros(J.shape[1])]), rcond=None)[0]
    return float(np.linalg.norm(d * p))


def bisect_lambda(J, b, d, target):
    """The lambda with ||D p(lambda)|| = target, by bisection (the length falls as lambda grows)."""
    lo, hi = 0.0, 1.0
    while scaled_length(J, b, d, hi) > target:
        hi *= 4.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if scaled_length(J, b, d, mid) > target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("seed,delta", [(1, 0.1), (1, 1.0), (2, 2.5), (3, 0.5)])
def test_trust_region_lambda_within_the_bisection_bracket(seed, delta):
    blocks, J, b, d = tr_problem(seed)
    lam, p, it = more.trust_region_lambda(blocks, b, d, delta, sigma=0.1)
    assert lam > 0 and it >= 1
    length = float(np.linalg.norm(d * p))
    assert abs(length - delta) <= 0.1 * delta + 1e-12
    # an independent root finder on the assembled problem brackets it
    lam_a = bisect_lambda(J, b, d, 1.1 * delta)
    lam_b = bisect_lambda(J, b, d, 0.9 * delta)
    assert lam_a * (1 - 1e-9) <= lam <= lam_b * (1 + 1e-9)
    # the step is the damped least-squares solution at that lambda
    A = np.vstack([J, np.sqrt(lam) * np.diag(d)])
    p_ref = np.linalg.lstsq(A, np.concatenate([b, np.zeros(J.shape[1])]), rcond=None)[0]
    np.testing.assert_allclose(p, p_ref, rtol=1e-9, atol=1e-12)


def test_trust_region_gauss_newton_step_inside():
    blocks, J, b, d = tr_problem(4)
    p_gn = np.linalg.lstsq(J, b, rcond=None)[0]
    big = 2.0 * float(np.linalg.norm(d * p_gn))
    lam, p, it = more.trust_region_lambda(blocks, b, d, big)
    assert lam == 0.0 and it == 0
    np.testing.assert_allclose(p, p_gn, rtol=1e-9, atol=1e-12)


def derivative_pin_passes(parts):
    """d/dlam ||D p|| = -||z||^2 / ||q|| from `parts`, against central differences of the
    length on the assembled problem."""
    blocks, J, b, d = tr_problem(5)
    s1s, ds, r0, c0 = [], [], 0, 0
    for Ji in blocks:
        n, m = Ji.shape
        s1s.append(more.stage1(Ji, b[r0:r0 + n]))
        ds.append(d[c0:c0 + m])
        r0 += n
        c0 += m
    for lam in (0.05, 0.7, 3.0):
        _, qn, zn = parts(s1s, ds, lam)
        h = 1e-5 * lam
        fd = (scaled_length(J, b, d, lam + h) - scaled_length(J, b, d, lam - h)) / (2 * h)
        if not np.isclose(-zn * zn / qn, fd, rtol=1e-5):
            return False
    return True


def test_trust_region_derivative_pinned():
    assert derivative_pin_passes(more.tr_parts)


def test_trust_region_derivative_planted_mistake_fails():
    def missing_d(s1_list, d_list, lam):   # z = R'^{-T} q instead of R'^{-T} D q
        ps, q2, z2 = [], 0.0, 0.0
        for s1, dd in zip(s1_list, d_list):
            p, Rp, _ = more.stage2(s1, dd, lam)
            q = dd * p
            z = hh.forward_substitute_rt(Rp, q)
            q2 += float(q @ q)
            z2 += float(z @ z)
        return None, np.sqrt(q2), np.sqrt(z2)
    assert not derivative_pin_passes(missing_d)
