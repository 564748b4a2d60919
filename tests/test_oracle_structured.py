"""Pins of the composed block-angular solve (Secs. 4.1, 4.2, 4.5, 5.2)."""
import numpy as np
import pytest

from oracle import householder as hh
from oracle import normal
from oracle import structured as st


def small_problem(K=5, n=4, m=2, s=3, lam=0.1, seed=0, windowed=False, w=4):
    g = np.random.default_rng(seed)
    blocks = [g.standard_normal((n, m)) for _ in range(K)]
    if windowed:
        start = np.sort(g.integers(0, s - w + 1, size=K))
        coupled = [g.standard_normal((n, w)) for _ in range(K)]
    else:
        start = None
        coupled = [g.standard_normal((n, s)) for _ in range(K)] if s else None
    b = g.standard_normal(K * n)
    return st.BlockProblem(blocks=blocks, coupled=coupled, start=start, s=s, b=b, lam=lam)


def lstsq_augmented(P):
    A, rhs = st.assemble_augmented(P)
    return np.linalg.lstsq(A, rhs, rcond=None)[0]


@pytest.mark.parametrize("kw", [dict(), dict(lam=0.0, K=4, n=5, m=2, s=3),
                                dict(windowed=True, s=10, w=4, K=8),
                                dict(s=0), dict(K=1, n=6, m=3, s=2, lam=2.0)])
def test_composed_equals_dense_and_library(kw):
    P = small_problem(**kw)
    p, F = st.factor_and_solve(P)
    x_dense, f, qtb = st.solve_dense(P)
    x_np = lstsq_augmented(P)
    np.testing.assert_allclose(p, x_np, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(x_dense, x_np, rtol=1e-11, atol=1e-12)
    J = st.assemble_J(P)
    D = st.damping(P)
    assert st.optimality_residual(J, P.b, D, P.lam, p) < 1e-14
    # Parseval: ||[b;0]||^2 = ||top of Q^T [b;0]||^2 + residual^2
    top = sum(float(np.dot(c, c)) for c in F.c_blocks)
    if F.c_S is not None:
        top += float(np.dot(F.c_S, F.c_S))
    assert top + F.residual_sq == pytest.approx(float(np.dot(P.b, P.b)), rel=1e-12)


def test_banded_reduced_solver_matches_dense():
    P = small_problem(windowed=True, s=14, w=4, K=12, lam=0.05, seed=3)
    p1, _ = st.factor_and_solve(P)
    p2, _ = st.factor_and_solve(P, reduced_solver=st.banded_reduced_solver(group=3))
    np.testing.assert_allclose(p1, p2, rtol=1e-11, atol=1e-12)


def test_composed_R_reproduces_gram():
    """R^T R = A^T A for the R assembled from the composed pieces (R unique up to signs)."""
    P = small_problem(K=4, n=4, m=2, s=3, lam=0.3, seed=5)
    p, F = st.factor_and_solve(P)
    N, nb, s = P.N, P.n_block_cols, P.s
    R = np.zeros((N, N))
    co = P.col_offsets()
    for i, f in enumerate(F.block_factors):
        R[co[i]:co[i + 1], co[i]:co[i + 1]] = f.R
        R[co[i]:co[i + 1], nb:] = F.R12[i]
    R[nb:, nb:] = F.reduced_factor.R
    A, _ = st.assemble_augmented(P)
    np.testing.assert_allclose(R.T @ R, A.T @ A, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(hh.normalise_row_signs(R),
                               hh.normalise_row_signs(np.linalg.qr(A, mode="r")), atol=1e-12)


def test_closed_form_one_column_blocks():
    """s = 0, m_i = 1: p_i = a^T b / (a^T a + lambda d^2) (ridge scalar)."""
    g = np.random.default_rng(11)
    K, n, lam = 6, 3, 0.7
    blocks = [g.standard_normal((n, 1)) for _ in range(K)]
    b = g.standard_normal(K * n)
    D = np.abs(g.standard_normal(K)) + 0.5
    P = st.BlockProblem(blocks=blocks, b=b, lam=lam, D=D)
    p, _ = st.factor_and_solve(P)
    for i in range(K):
        a = blocks[i][:, 0]
        bi = b[i * n:(i + 1) * n]
        assert p[i] == pytest.approx(a @ bi / (a @ a + lam * D[i] ** 2), rel=1e-13)


def test_closed_form_identity():
    """J = I, D = I: p = b / (1 + lambda)."""
    K, lam = 7, 0.25
    b = np.arange(1.0, K + 1.0)
    P = st.BlockProblem(blocks=[np.ones((1, 1)) for _ in range(K)], b=b, lam=lam, D=np.ones(K))
    p, _ = st.factor_and_solve(P)
    np.testing.assert_allclose(p, b / (1 + lam), rtol=1e-14)


def test_normal_equations_cross_check():
    P = small_problem(K=6, n=5, m=2, s=4, lam=0.2, seed=21)
    p, _ = st.factor_and_solve(P)
    J = st.assemble_J(P)
    p_ne = normal.solve(J, P.b, st.damping(P), P.lam)
    np.testing.assert_allclose(p, p_ne, rtol=1e-9)


def test_row_permutation_metadata():
    """P_r makes [J; lambda^(1/2) D] block-angular with sorted leading columns."""
    P = small_problem(K=3, n=2, m=2, s=2, lam=0.5, seed=4)
    order = st.row_permutation(P)
    M, N = P.M, P.N
    # block i: its 2 J rows then the damping rows of its 2 columns; then the S damping rows
    expect = []
    for i in range(3):
        expect += [2 * i, 2 * i + 1, M + 2 * i, M + 2 * i + 1]
    expect += [M + 6, M + 7]
    assert order.tolist() == expect
    A, _ = st.assemble_augmented(P)
    lead = [int(np.nonzero(row)[0][0]) for row in A]
    assert lead == sorted(lead)


def test_planted_mistake_missing_damping_is_caught(monkeypatch):
    """Dropping the damping rows of the blocks fails the optimality identity."""
    real = st.augmented_block

    def bad(P, i, D, *offsets):
        B, C, rhs = real(P, i, D, *offsets)
        n = P.blocks[i].shape[0]
        return B[:n], (None if C is None else C[:n]), rhs[:n]
    monkeypatch.setattr(st, "augmented_block", bad)
    P = small_problem(K=4, n=4, m=2, s=3, lam=0.5, seed=6)
    p, _ = st.factor_and_solve(P)
    J = st.assemble_J(P)
    assert st.optimality_residual(J, P.b, st.damping(P), P.lam, p) > 1e-6


def test_planted_mistake_sign_of_coupling_is_caught():
    """A sign error in the coupled columns (S -> -S) is caught by the optimality identity."""
    P = small_problem(K=4, n=4, m=2, s=3, lam=0.5, seed=7)
    p_ok, _ = st.factor_and_solve(P)
    P2 = small_problem(K=4, n=4, m=2, s=3, lam=0.5, seed=7)
    P2.coupled = [-c for c in P2.coupled]
    p_bad, _ = st.factor_and_solve(P2)
    J = st.assemble_J(P)
    assert st.optimality_residual(J, P.b, st.damping(P), P.lam, p_bad) > 1e-6
    assert st.optimality_residual(J, P.b, st.damping(P), P.lam, p_ok) < 1e-14


@pytest.mark.parametrize("kw,damped", [(dict(K=5, n=4, m=2, s=3), True), (dict(K=6, n=3, m=2, s=0), True),
                                       (dict(windowed=True, s=12, w=4, K=9), True),
                                       (dict(windowed=True, s=12, w=4, K=9, lam=0.0), False),
                                       (dict(K=4, n=5, m=3, s=2, lam=0.0), False)])
def test_structural_metadata_matches_the_numerical_factor(kw, damped):
    """The structural P_r equals the value-based one on random data, and the symbolic R
    pattern is exactly the non-zero pattern of the R that dense Householder QR of
    P_r [J; lambda^(1/2) D] produces (random values: no cancellation)."""
    P = small_problem(**kw)
    order = st.structural_row_order(P, damped)
    if damped:
        np.testing.assert_array_equal(order, st.row_permutation(P))
    ptr, idx = st.r_pattern(P, damped)
    A, _ = st.assemble_augmented(P)
    if not damped:
        A = st.assemble_J(P)[order]
    R = hh.qr(A).R
    for c in range(P.N):
        nz = np.nonzero(np.abs(R[c]) > 1e-13 * np.abs(R).max())[0]
        assert nz.tolist() == idx[ptr[c]:ptr[c + 1]].tolist(), c


def test_structural_pattern_planted_mistake_fails():
    """Merging without carrying the union (a row keeps only its own columns) gives a pattern
    that misses fill, so it differs from the numerical one."""
    P = small_problem(windowed=True, s=12, w=4, K=9)
    rows = st.structural_rows(P, True)
    R = [None] * P.N
    for k in st.structural_row_order(P, True):
        cur = sorted(set(rows[int(k)]))
        while cur:
            c = cur[0]
            if R[c] is None:
                R[c] = cur
                break
            cur = cur[1:]                       # planted: no union with R row c
    ptr, idx = st.r_pattern(P, True)
    bad = [x for c in range(P.N) for x in (R[c] or [])]
    assert bad != idx.tolist()
