"""Host logic of the block plan, no GPU: the warp-task lists of the fused block solve
(Sec. 4.1 "Block diagonal": independent blocks, grouped by shape so that one warp factors
blocks of a single shape) checked against a direct restatement of their definition and
against the invariants every task list must satisfy."""
import numpy as np
import pytest

from paper_1802_03773_gb300 import qrkit


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1802_03773_gb300 import build as b
    b.build()
    return qrkit.load()


def shapes(K, seed, wide=False):
    rng = np.random.default_rng(seed)
    n = rng.integers(1, 17, size=K)
    hi = 9 if wide else np.minimum(n, 8) + 1
    m = rng.integers(1, hi, size=K)
    return n.astype(np.uint8), m.astype(np.uint8)


def key_of(n, m):
    return 8 * ((n.astype(np.int64) - 1) // 4) + (m.astype(np.int64) - 1)


def expected(n, m, supertile, key_major):
    """The definition: per supertile of consecutive blocks, blocks in ascending key order
    (ties by block index), each key's run cut into tasks of 32 / G blocks, G = row class + 1."""
    K = n.size
    nm = n.astype(np.int64) * m
    voff = np.concatenate([[0], np.cumsum(nm)])
    roff = np.concatenate([[0], np.cumsum(n.astype(np.int64))])
    coff = np.concatenate([[0], np.cumsum(m.astype(np.int64))])
    keys = key_of(n, m)
    tasks = []
    for s0 in range(0, K, supertile):
        idx = np.arange(s0, min(K, s0 + supertile))
        for k in range(32):
            run = idx[keys[idx] == k]
            per = 32 // (k // 8 + 1)
            for c0 in range(0, run.size, per):
                slots = -np.ones((32, 4), dtype=np.int64)
                for l, i in enumerate(run[c0:c0 + per]):
                    slots[l] = (i, voff[i], roff[i], coff[i])
                tasks.append((k, slots))
    if key_major:
        tasks.sort(key=lambda t: t[0])   # stable
    key = np.array([t[0] for t in tasks], dtype=np.int32)
    return key, np.stack([t[1] for t in tasks])


@pytest.mark.parametrize("K,supertile,key_major,wide", [
    (1, 65536, False, False),
    (33, 32, False, False),
    (1000, 32, False, True),
    (5000, 256, False, False),
    (5000, 256, True, False),
    (20000, 65536, False, True),
    (70000, 65536, True, False),      # two supertiles, the second ragged
])
def test_layout_matches_definition(K, supertile, key_major, wide):
    n, m = shapes(K, seed=K + supertile + int(key_major), wide=wide)
    key, slots = qrkit.task_layout(n, m, supertile, key_major)
    ek, es = expected(n, m, supertile, key_major)
    np.testing.assert_array_equal(key, ek)
    np.testing.assert_array_equal(slots, es)


@pytest.mark.parametrize("supertile,key_major", [(64, False), (64, True), (65536, False)])
def test_layout_invariants(supertile, key_major):
    K = 3001
    n, m = shapes(K, seed=7, wide=True)
    key, slots = qrkit.task_layout(n, m, supertile, key_major)
    blk = slots[:, :, 0]
    used = blk >= 0
    # every block in exactly one slot
    np.testing.assert_array_equal(np.sort(blk[used]), np.arange(K))
    keys = key_of(n, m)
    per = 32 // (key // 8 + 1)
    for t in range(key.size):
        b = blk[t][used[t]]
        # one shape key per task, slots used from the front, at most 32 / G of them
        assert np.all(keys[b] == key[t])
        assert used[t, :b.size].all() and not used[t, b.size:].any()
        assert 1 <= b.size <= per[t]
        # all blocks of a task in one supertile, ascending
        assert np.all(b // supertile == b[0] // supertile)
        assert np.all(np.diff(b) > 0)
    # a task with unused slots is the last of its key in its supertile
    st = blk[:, 0] // supertile
    for t in range(key.size):
        if used[t].sum() < per[t]:
            later = (key == key[t]) & (st == st[t]) & (np.arange(key.size) > t)
            assert not later.any()
    if key_major:
        assert np.all(np.diff(key) >= 0)
    else:
        order = st * 64 + key
        assert np.all(np.diff(order) >= 0)


def test_layout_offsets_are_prefix_sums():
    n = np.array([3, 16, 1, 8, 4, 5], dtype=np.uint8)
    m = np.array([2, 8, 1, 8, 4, 1], dtype=np.uint8)
    key, slots = qrkit.task_layout(n, m, 32)
    rows = {int(s[0]): tuple(s[1:]) for s in slots.reshape(-1, 4) if s[0] >= 0}
    # hand-computed: values n_i m_i = 6, 128, 1, 64, 16, 5; rows n_i; columns m_i
    assert rows == {0: (0, 0, 0), 1: (6, 3, 2), 2: (134, 19, 10), 3: (135, 20, 11),
                    4: (199, 28, 19), 5: (215, 32, 23)}
    # keys: (3,2) -> 1, (16,8) -> 31, (1,1) -> 0, (8,8) -> 15, (4,4) -> 3, (5,1) -> 8
    np.testing.assert_array_equal(key, [0, 1, 3, 8, 15, 31])


def test_layout_task_counts():
    # 100 blocks of 16 x 8 (G = 4, 8 per task) and 100 of 2 x 1 (G = 1, 32 per task)
    n = np.array([16] * 100 + [2] * 100, dtype=np.uint8)
    m = np.array([8] * 100 + [1] * 100, dtype=np.uint8)
    key, _ = qrkit.task_layout(n, m, 65536)
    assert key.size == 4 + 13
    key, _ = qrkit.task_layout(n, m, 100)   # each key alone in its supertile
    assert key.size == 4 + 13


def test_layout_rejects_bad_arguments():
    import ctypes
    lib = qrkit.load()
    n = np.array([4, 4], dtype=np.uint8)
    m = np.array([2, 2], dtype=np.uint8)
    cnt = ctypes.c_int64(-1)

    def call(nn, mm, supertile=65536, cap=0, key=None):
        return lib.qrkit_task_layout(nn.shape[0], nn.ctypes.data, mm.ctypes.data, supertile, 0,
                                     ctypes.addressof(cnt), key, None, cap)

    assert call(n, m, supertile=31) == 1
    assert call(n, m, supertile=65537) == 1
    assert call(np.array([0, 4], dtype=np.uint8), m) == 1
    assert call(np.array([17, 4], dtype=np.uint8), m) == 8
    assert call(n, np.array([9, 2], dtype=np.uint8)) == 8
    key = np.zeros(4, dtype=np.int32)
    assert call(n, m) == 0 and cnt.value == 1
    assert call(n, m, cap=0, key=key.ctypes.data) == 1 and cnt.value == 1
    assert call(n, m, cap=1, key=key.ctypes.data) == 0 and key[0] == 1
    assert lib.qrkit_task_layout(0, n.ctypes.data, m.ctypes.data, 64, 0, ctypes.addressof(cnt),
                                 None, None, 0) == 1


def test_layout_fuzz():
    """Random batch sizes, supertiles and orders against the definition."""
    g = np.random.default_rng(77)
    for _ in range(25):
        K = int(g.integers(1, 3000))
        supertile = int(g.integers(32, 400))
        key_major = bool(g.integers(0, 2))
        n, m = shapes(K, seed=int(g.integers(0, 1 << 30)), wide=bool(g.integers(0, 2)))
        key, slots = qrkit.task_layout(n, m, supertile, key_major)
        ek, es = expected(n, m, supertile, key_major)
        np.testing.assert_array_equal(key, ek)
        np.testing.assert_array_equal(slots, es)
