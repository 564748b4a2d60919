"""Host logic, no GPU: the library's band-exposing permutations (Sec. 4.3) equal the oracle's
index for index, and exposed bands hold every row."""
import numpy as np
import pytest

from oracle import reorder
from paper_1802_03773_gb300 import qrkit
from tests.test_oracle_reorder import check_band, csr, scrambled_band


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1802_03773_gb300 import build as b
    b.build()
    return qrkit.load()


def same(rows_cols, rows, cols):
    rp, ci = csr(rows_cols)
    ours = qrkit.band_order(rows, cols, rp, ci)
    ref = reorder.band_order(rows, cols, rp, ci)
    np.testing.assert_array_equal(ours[0], ref[0])
    np.testing.assert_array_equal(ours[1], ref[1])
    np.testing.assert_array_equal(ours[2], ref[2])
    assert ours[3] == ref[3]
    check_band(rows_cols, cols, *ours)
    return ours


@pytest.mark.parametrize("n,rpc,w,seed", [(40, 1, 2, 0), (200, 4, 8, 1), (500, 2, 5, 2), (3000, 4, 8, 3)])
def test_scrambled_bands_match_oracle(n, rpc, w, seed):
    rows_cols = scrambled_band(n, rpc, w, seed)
    ours = same(rows_cols, len(rows_cols), n)
    assert ours[3] == w


@pytest.mark.parametrize("seed", range(6))
def test_random_patterns_match_oracle(seed):
    g = np.random.default_rng(100 + seed)
    rows, cols = int(g.integers(1, 120)), int(g.integers(1, 60))
    rows_cols = [g.integers(0, cols, size=g.integers(0, 6)).tolist() for _ in range(rows)]   # repeats allowed
    same(rows_cols, rows, cols)


def test_worked_example_and_edge_cases():
    col_perm, row_perm, row_start, w = same([[0, 3], [1], [0, 2], [1, 3], [2]], 5, 4)
    assert col_perm.tolist() == [2, 0, 3, 1] and w == 2
    # no rows; one column; an all-empty pattern
    same([], 0, 3)
    same([[0], [0], []], 3, 1)
    _, _, starts, w = same([[], []], 2, 4)
    assert starts.tolist() == [4, 4] and w == 0


def test_rejects_malformed_patterns():
    lib = qrkit.load()
    cp = np.empty(4, dtype=np.int32)
    rp_out = np.empty(2, dtype=np.int64)
    rs = np.empty(2, dtype=np.int32)
    import ctypes
    w = ctypes.c_int32(0)

    def call(rows, cols, row_ptr, col_idx):
        row_ptr = np.asarray(row_ptr, dtype=np.int64)
        col_idx = np.asarray(col_idx, dtype=np.int32)
        return lib.qrkit_band_order(rows, cols, row_ptr.ctypes.data, col_idx.ctypes.data, cp.ctypes.data,
                                    rp_out.ctypes.data, rs.ctypes.data, ctypes.addressof(w))

    assert call(2, 4, [0, 1, 2], [0, 3]) == 0
    assert call(2, 4, [0, 1, 2], [0, 4]) == 1      # column out of range
    assert call(2, 4, [0, 2, 1], [0, 1]) == 1      # offsets decrease
    assert call(2, 4, [1, 1, 2], [0, 1]) == 1      # offsets do not start at 0
    assert call(2, 0, [0, 0, 0], [0]) == 1         # no columns


def test_fuzz_patterns_match_oracle():
    """Many small patterns: isolated columns, repeated entries, empty rows, dense rows."""
    g = np.random.default_rng(2024)
    for _ in range(150):
        rows, cols = int(g.integers(0, 40)), int(g.integers(1, 25))
        dens = g.uniform(0.0, 0.5)
        rows_cols = []
        for _ in range(rows):
            k = int(g.binomial(cols, dens))
            rows_cols.append(g.integers(0, cols, size=k).tolist())
        same(rows_cols, rows, cols)
