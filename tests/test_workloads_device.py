"""The device-side batch generator (workloads/device.py) lays out instances as the banded
solver expects: 4 n rows of w values per instance, row i starting at column floor(i / 4), and
exactly the entries past an instance's last column set to zero.  Run with the CPU generator."""
import numpy as np

from workloads.device import banded_batch_device


def test_banded_batch_device_layout_and_truncation():
    torch = __import__("torch")
    cols = np.array([10, 3, 17, 8], dtype=np.int64)
    d = banded_batch_device(cols, rows_per_col=4, w=8, seed_offset=3, device="cpu", dtype=torch.float64)
    v = d["vals"].numpy()
    assert v.shape == (int(4 * cols.sum()), 8) and d["b"].shape == (int(4 * cols.sum()),)
    assert list(d["row0"]) == [0, 40, 52, 120, 152] and list(d["col0"]) == [0, 10, 13, 30, 38]
    for k, n in enumerate(cols):
        for i in range(4 * n):
            s = i // 4
            for c in range(8):
                zero = v[d["row0"][k] + i, c] == 0.0
                assert zero == (s + c >= n), (k, i, c)


def test_banded_batch_device_is_seeded():
    torch = __import__("torch")
    cols = np.array([12, 5], dtype=np.int64)
    a = banded_batch_device(cols, seed_offset=1, device="cpu")
    b = banded_batch_device(cols, seed_offset=1, device="cpu")
    c = banded_batch_device(cols, seed_offset=2, device="cpu")
    assert torch.equal(a["vals"], b["vals"]) and torch.equal(a["b"], b["b"])
    assert not torch.equal(a["vals"], c["vals"])
