"""Pins of the band-exposing row and column permutations (Sec. 4.3) of the oracle."""
import numpy as np
import pytest

from oracle import reorder


def csr(rows_cols):
    row_ptr = np.concatenate([[0], np.cumsum([len(r) for r in rows_cols])]).astype(np.int64)
    col_idx = np.array([c for r in rows_cols for c in r], dtype=np.int32)
    return row_ptr, col_idx


def test_worked_example():
    """Columns form the chain 2 - 0 - 3 - 1 (rows {0,3}, {0,2}, {1,3}) plus single-entry rows.
    Degrees 2, 1, 1, 2: the search starts at column 1 (least degree, lower index), visits
    1, 3, 0, 2; reversed, P_c = [2, 0, 3, 1] (new positions: col 2 -> 0, 0 -> 1, 3 -> 2,
    1 -> 3).  Rows as (first, last): row 0 (1, 2), row 1 (3, 3), row 2 (0, 1), row 3 (2, 3),
    row 4 (0, 0); sorted: rows 4, 2, 0, 3, 1 with starts 0, 0, 1, 2, 3; band width 2."""
    rows_cols = [[0, 3], [1], [0, 2], [1, 3], [2]]
    rp, ci = csr(rows_cols)
    col_perm, row_perm, row_start, w = reorder.band_order(5, 4, rp, ci)
    assert col_perm.tolist() == [2, 0, 3, 1]
    assert row_perm.tolist() == [4, 2, 0, 3, 1]
    assert row_start.tolist() == [0, 0, 1, 2, 3]
    assert w == 2


def scrambled_band(n, rows_per_col, w, seed):
    """Row i touches columns floor(i / rows_per_col) .. + w - 1 (truncated), then rows and
    columns shuffled."""
    g = np.random.default_rng(seed)
    M = rows_per_col * n
    rows = [list(range(i // rows_per_col, min(n, i // rows_per_col + w))) for i in range(M)]
    cperm = g.permutation(n)            # original column c is stored as cperm[c]
    rows = [[int(cperm[c]) for c in r] for r in rows]
    rorder = g.permutation(M)
    return [rows[i] for i in rorder]


def check_band(rows_cols, cols, col_perm, row_perm, row_start, w):
    rows = len(rows_cols)
    assert sorted(col_perm.tolist()) == list(range(cols))
    assert sorted(row_perm.tolist()) == list(range(rows))
    newpos = np.empty(cols, dtype=np.int64)
    newpos[col_perm] = np.arange(cols)
    for k, i in enumerate(row_perm):
        p = newpos[rows_cols[i]]
        if p.size:
            assert p.min() == row_start[k]
            assert p.max() < row_start[k] + w
    assert np.all(np.diff(row_start) >= 0)


@pytest.mark.parametrize("n,rpc,w,seed", [(40, 1, 2, 0), (60, 2, 3, 1), (80, 4, 4, 2), (50, 3, 8, 3)])
def test_scrambled_band_is_recovered(n, rpc, w, seed):
    rows_cols = scrambled_band(n, rpc, w, seed)
    rp, ci = csr(rows_cols)
    col_perm, row_perm, row_start, width = reorder.band_order(len(rows_cols), n, rp, ci)
    check_band(rows_cols, n, col_perm, row_perm, row_start, width)
    assert width == w


def test_random_pattern_is_a_valid_band():
    g = np.random.default_rng(9)
    rows_cols = [sorted(set(g.integers(0, 30, size=g.integers(0, 5)).tolist())) for _ in range(70)]
    rp, ci = csr(rows_cols)
    col_perm, row_perm, row_start, w = reorder.band_order(70, 30, rp, ci)
    check_band(rows_cols, 30, col_perm, row_perm, row_start, w)
    # empty rows sort last with start = cols
    empty = [k for k, i in enumerate(row_perm) if not rows_cols[i]]
    assert all(row_start[k] == 30 for k in empty)
    assert empty == list(range(70 - len(empty), 70))


def test_planted_mistake_without_reversal_changes_the_worked_example(monkeypatch):
    """Cuthill-McKee without the final reversal gives a different P_c on the worked example."""
    rows_cols = [[0, 3], [1], [0, 2], [1, 3], [2]]
    rp, ci = csr(rows_cols)
    real = reorder.reverse_cuthill_mckee
    monkeypatch.setattr(reorder, "reverse_cuthill_mckee", lambda c, r: real(c, r)[::-1])
    col_perm, _, _, _ = reorder.band_order(5, 4, rp, ci)
    assert col_perm.tolist() != [2, 0, 3, 1]
