"""Host logic, no GPU: the structure metadata of a block-angular descriptor (offsets, the row
permutation P_r of [J; lambda^(1/2) D] and the structural pattern of R) equals the oracle's,
integer for integer (Sec. 3, Sec. 4.5 / 5.2)."""
import numpy as np
import pytest

from oracle import structured as st
from paper_1802_03773_gb300 import qrkit


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1802_03773_gb300 import build as b
    b.build()
    return qrkit.load()


def problem(K, s, windowed, w, seed):
    g = np.random.default_rng(seed)
    n = g.integers(1, 7, size=K)
    m = np.minimum(g.integers(1, 4, size=K), n)
    blocks = [g.standard_normal((int(a), int(c))) for a, c in zip(n, m)]
    if windowed:
        start = g.integers(0, s, size=K)
        coupled = [g.standard_normal((int(a), w)) for a in n]
        # entries past the last shared column are structurally absent
        for c, st0 in zip(coupled, start):
            if st0 + w > s:
                c[:, s - st0:] = 0.0
    else:
        start = None
        coupled = [g.standard_normal((int(a), s)) for a in n] if s else None
    b = g.standard_normal(int(n.sum()))
    return st.BlockProblem(blocks=blocks, coupled=coupled, start=start, s=s, b=b, lam=0.3), n, m, start


@pytest.mark.parametrize("K,s,windowed,w,seed", [(7, 0, False, 0, 1), (9, 4, False, 0, 2), (12, 15, True, 4, 3),
                                                 (30, 40, True, 6, 4), (1, 3, False, 0, 5)])
@pytest.mark.parametrize("damped", [True, False])
def test_metadata_equals_oracle(K, s, windowed, w, seed, damped):
    P, n, m, start = problem(K, s, windowed, w, seed)
    kw = {}
    if s and windowed:
        kw = dict(coupled=qrkit.COUPLED_WINDOW, shared_cols=s, window=w, window_start=start)
    elif s:
        kw = dict(coupled=qrkit.COUPLED_DENSE, shared_cols=s)
    vo, ro, co, order, ptr, idx = qrkit.structure_metadata(n, m, damped, **kw)
    np.testing.assert_array_equal(ro, P.row_offsets())
    np.testing.assert_array_equal(co, P.col_offsets())
    np.testing.assert_array_equal(vo, np.concatenate([[0], np.cumsum(n * m)]))
    np.testing.assert_array_equal(order, st.structural_row_order(P, damped))
    rp, ci = st.r_pattern(P, damped)
    np.testing.assert_array_equal(ptr, rp)
    np.testing.assert_array_equal(idx, ci)


def test_metadata_segments_cut_windows():
    """Two segments: a window that would run past its segment's end is cut there; the
    pattern equals the oracle's on the problem whose windows are cut the same way."""
    n = np.array([2, 3, 2, 2])
    m = np.array([1, 1, 2, 1])
    start = np.array([3, 0, 5, 6], dtype=np.int32)     # segment 0: columns 0..4, segment 1: 5..7
    vo, ro, co, order, ptr, idx = qrkit.structure_metadata(
        n, m, True, coupled=qrkit.COUPLED_WINDOW, shared_cols=8, window=3, window_start=start,
        segment_cols=[5, 3], segment_blocks=[2, 2])
    g = np.random.default_rng(9)
    blocks = [g.standard_normal((int(a), int(c))) for a, c in zip(n, m)]
    ends = [5, 5, 8, 8]
    coupled = []
    for a, st0, e in zip(n, start, ends):
        c = g.standard_normal((int(a), 3))
        c[:, max(0, e - st0):] = 0.0
        coupled.append(c)
    P = st.BlockProblem(blocks=blocks, coupled=coupled, start=start, s=8, b=np.zeros(int(n.sum())), lam=0.1)
    # the oracle's structural rows use min(start + w, s): emulate the segment cut on a copy
    rows = st.structural_rows(P, True)
    nb = P.n_block_cols
    for i, (st0, e) in enumerate(zip(start, ends)):
        for r in range(P.row_offsets()[i], P.row_offsets()[i + 1]):
            rows[int(r)] = [c for c in rows[int(r)] if c < nb or c - nb < e]
    R = [None] * P.N
    for k in st.structural_row_order(P, True):
        cur = sorted(set(rows[int(k)]))
        while cur:
            c = cur[0]
            if R[c] is None:
                R[c] = cur
                break
            R[c] = sorted(set(R[c]) | set(cur))
            cur = [x for x in R[c] if x > c]
    assert idx.tolist() == [x for c in range(P.N) for x in (R[c] or [])]


def test_metadata_rejects_bad_descriptors():
    with pytest.raises(qrkit.QRKitError) as e:
        qrkit.structure_metadata([2, 2], [1, 1], False, coupled=qrkit.COUPLED_WINDOW, shared_cols=4, window=2,
                                 window_start=[0, 4])
    assert e.value.status == 1
    with pytest.raises(qrkit.QRKitError) as e:
        qrkit.structure_metadata([2, 0], [1, 1], False)
    assert e.value.status == 1
