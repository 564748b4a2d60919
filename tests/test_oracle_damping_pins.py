"""Pins of the damping diagonal D and of the LM model decrease (Sec. 2, Sec. 5.2).

D = diag(J^T J)^(1/2) is the column norms of J (Backtrack LM, Sec. 5.2), a zero norm taken
as 1 (MINPACK's convention; the paper is silent).  Every GPU test that passes D = None is
compared against the oracle's D, so D is pinned here against values fixed by hand and by
the definition, and each plausible mistake (squared norms, no zero -> 1, norms over the
damping rows too) is planted in a copy of the oracle function and must fail a pin.

The gain ratio's denominator (Sec. 2) is the decrease of the undamped linear model
L(p) = 1/2 ||b - J p||^2, which at the damped minimiser p* of Eq. 2 equals
1/2 p*^T (lambda D^2 p* + J^T b).  That decrease is computed here from J p alone, so the
pin does not share the formula it checks; for a residual that is linear in x the gain
ratio is then exactly 1.
"""
import numpy as np
import pytest

from oracle import banded as bd
from oracle import lm
from oracle import structured as st


# ---------------------------------------------------------------- column norms, block-angular

def worked_block_problem():
    """Two 2 x 2 blocks and a windowed S (w = 2, s = 4) with norms that are whole numbers.

    Block columns: [3, 4] -> 5, [0, 0] -> 0 -> 1, [1, 2] -> sqrt(5), [6, 8] -> 10.
    S columns: 0 touched by block 0 with [1, 2] -> sqrt(5); 1 by both blocks, [2, 2] and
    [1, 0] -> 3; 2 by block 1 with [0, 0] -> 0 -> 1; 3 by nobody -> 1.
    """
    blocks = [np.array([[3.0, 0.0], [4.0, 0.0]]), np.array([[1.0, 6.0], [2.0, 8.0]])]
    coupled = [np.array([[1.0, 2.0], [2.0, 2.0]]), np.array([[1.0, 0.0], [0.0, 0.0]])]
    start = np.array([0, 1])
    P = st.BlockProblem(blocks=blocks, coupled=coupled, start=start, s=4,
                        b=np.zeros(4), lam=0.5)
    expect = np.array([5.0, 1.0, np.sqrt(5.0), 10.0, np.sqrt(5.0), 3.0, 1.0, 1.0])
    return P, expect


def random_block_problem(seed, windowed, zero_cols=True):
    g = np.random.default_rng(seed)
    K, s, w = 6, 9, 3
    blocks = [g.standard_normal((int(g.integers(2, 5)), int(g.integers(1, 3)))) for _ in range(K)]
    if zero_cols:
        blocks[2][:, 0] = 0.0
    if windowed:
        start = g.integers(0, s - w, size=K)
        start[:] = np.minimum(start, s - w - 1)   # the last shared column is never touched
        coupled = [g.standard_normal((blk.shape[0], w)) for blk in blocks]
    else:
        start = None
        coupled = [g.standard_normal((blk.shape[0], s)) for blk in blocks]
        if zero_cols:
            for c in coupled:
                c[:, 4] = 0.0
    b = g.standard_normal(sum(blk.shape[0] for blk in blocks))
    return st.BlockProblem(blocks=blocks, coupled=coupled, start=start, s=s, b=b, lam=0.3)


def dense_norms(J):
    d = np.sqrt(np.einsum("ij,ij->j", J, J))
    return np.where(d == 0.0, 1.0, d)


def block_norm_pins_pass(fn):
    P, expect = worked_block_problem()
    if not np.allclose(fn(P), expect, rtol=1e-15, atol=0):
        return False
    for seed, windowed in ((1, False), (2, True), (3, True)):
        P = random_block_problem(seed, windowed)
        if not np.allclose(fn(P), dense_norms(st.assemble_J(P)), rtol=1e-14, atol=0):
            return False
    return True


def test_block_column_norms_pinned():
    assert block_norm_pins_pass(st.column_norms)


def _squared(P):
    d = st.column_norms(P)
    return d * d


def _no_zero_to_one(P):
    J = st.assemble_J(P)
    return np.sqrt(np.einsum("ij,ij->j", J, J))


def _over_augmented_rows(P):
    # norms of [J; lambda^(1/2) D] with D the true norms: the damping rows counted too
    d = st.column_norms(P)
    return np.sqrt(d * d + P.lam * d * d)


@pytest.mark.parametrize("mistake", [_squared, _no_zero_to_one, _over_augmented_rows])
def test_block_column_norms_planted_mistakes_fail(mistake):
    assert not block_norm_pins_pass(mistake)


# ---------------------------------------------------------------- column norms, banded

def banded_norm_pins_pass(fn):
    # worked: rows (start, values) over N = 4 columns, w = 2.  Column 0: [3, 4] -> 5;
    # column 1: [1, 2, 0] -> sqrt(5); column 2: [2] -> 2; column 3: only row 3's leading 0
    # and the entry 5 past the last column, which is dropped -> 0 -> 1
    start = np.array([0, 0, 1, 3])
    vals = np.array([[3.0, 1.0], [4.0, 2.0], [0.0, 2.0], [0.0, 5.0]])
    expect = np.array([5.0, np.sqrt(5.0), 2.0, 1.0])
    try:
        if not np.allclose(fn(start, vals, 4), expect, rtol=1e-15, atol=0):
            return False
    except ValueError:
        return False
    g = np.random.default_rng(5)
    for n, rpc, w in ((30, 4, 8), (17, 3, 5), (12, 1, 3)):
        start = np.arange(rpc * n) // rpc
        vals = g.standard_normal((rpc * n, w))
        cols = start[:, None] + np.arange(w)[None, :]
        vals[cols >= n] = 0.0          # truncated band end
        vals[cols == 4] = 0.0          # column 4 is empty
        A = bd.assemble_dense(start, vals, n)
        if not np.allclose(fn(start, vals, n), dense_norms(A), rtol=1e-14, atol=0):
            return False
    return True


def test_banded_column_norms_pinned():
    assert banded_norm_pins_pass(bd.column_norms)


def _banded_squared(start, vals, N):
    d = bd.column_norms(start, vals, N)
    return d * d


def _banded_no_zero_to_one(start, vals, N):
    cols = np.asarray(start)[:, None] + np.arange(vals.shape[1])[None, :]
    ok = cols < N
    sq = np.zeros(N)
    np.add.at(sq, cols[ok], (np.asarray(vals) ** 2)[ok])
    return np.sqrt(sq)


def _banded_untruncated(start, vals, N):
    # entries past the last column folded onto it instead of dropped
    s = np.minimum(np.asarray(start)[:, None] + np.arange(vals.shape[1])[None, :], N - 1)
    sq = np.zeros(N)
    np.add.at(sq, s.ravel(), (np.asarray(vals) ** 2).ravel())
    d = np.sqrt(sq)
    d[d == 0] = 1.0
    return d


@pytest.mark.parametrize("mistake", [_banded_squared, _banded_no_zero_to_one, _banded_untruncated])
def test_banded_column_norms_planted_mistakes_fail(mistake):
    assert not banded_norm_pins_pass(mistake)


# ---------------------------------------------------------------- predicted decrease / rho

def Jp_blocks(P, p):
    """J p of a block-angular problem by per-block products (no assembled matrix)."""
    ro, co, nb = P.row_offsets(), P.col_offsets(), P.n_block_cols
    out = np.zeros(P.M)
    for i, blk in enumerate(P.blocks):
        y = blk @ p[co[i]:co[i + 1]]
        if P.coupled is not None and P.s > 0:
            w = P.coupled[i].shape[1]
            s0 = 0 if P.start is None else int(P.start[i])
            y = y + P.coupled[i] @ p[nb + s0:nb + s0 + w]
        out[ro[i]:ro[i + 1]] = y
    return out


def model_decrease(P, p):
    """L(0) - L(p) for L(p) = 1/2 ||b - J p||^2 (the undamped linear model)."""
    r = P.b - Jp_blocks(P, p)
    return 0.5 * (float(P.b @ P.b) - float(r @ r))


def pred_pins_pass(fn):
    for seed, windowed, lam in ((7, False, 0.3), (8, True, 2.0), (9, True, 1e-3)):
        P = random_block_problem(seed, windowed, zero_cols=False)
        P.lam = lam
        p, _ = st.factor_and_solve(P)
        if not np.isclose(fn(P, p), model_decrease(P, p), rtol=1e-12, atol=0):
            return False
    return True


def test_predicted_decrease_is_the_linear_model_decrease():
    assert pred_pins_pass(lm.predicted_decrease)


def _pred_without_half(P, p):
    return 2.0 * lm.predicted_decrease(P, p)


def _pred_lambda_D(P, p):
    # lambda D p instead of lambda D^2 p
    D = st.damping(P)
    J = st.assemble_J(P)
    return 0.5 * float(p @ (P.lam * D * p + J.T @ P.b))


def _pred_minus_jtb(P, p):
    D = st.damping(P)
    J = st.assemble_J(P)
    return 0.5 * float(p @ (P.lam * D * D * p - J.T @ P.b))


@pytest.mark.parametrize("mistake", [_pred_without_half, _pred_lambda_D, _pred_minus_jtb])
def test_predicted_decrease_planted_mistakes_fail(mistake):
    assert not pred_pins_pass(mistake)


def test_gain_ratio_is_one_for_a_linear_residual():
    """f(x) = A x - y with A = J of a block-angular problem: the cost is exactly quadratic,
    so the actual decrease of an LM step equals the model decrease and rho = 1."""
    P = random_block_problem(11, True, zero_cols=False)
    P.lam = 0.7
    x = np.random.default_rng(12).standard_normal(P.N)
    y = np.random.default_rng(13).standard_normal(P.M)
    f = Jp_blocks(P, x) - y
    P.b = -f
    p, _ = st.factor_and_solve(P)
    cost = 0.5 * float(f @ f)
    f_new = Jp_blocks(P, x + p) - y
    cost_new = 0.5 * float(f_new @ f_new)
    rho = (cost - cost_new) / lm.predicted_decrease(P, p)
    assert rho == pytest.approx(1.0, abs=1e-12)
    assert (cost - cost_new) / _pred_without_half(P, p) == pytest.approx(0.5, abs=1e-12)


def test_large_problem_branch_of_the_decrease():
    """Large problems take J^T b per block instead of from the assembled J: same values."""
    for seed, windowed in ((21, False), (22, True)):
        P = random_block_problem(seed, windowed, zero_cols=False)
        np.testing.assert_allclose(lm._jt_vec(P, P.b), st.assemble_J(P).T @ P.b, rtol=1e-14, atol=1e-14)
