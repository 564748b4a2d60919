"""Seeded synthetic inputs generated directly in GPU memory, for workloads too large to draw
on the host and copy (tens of GB).  Like the rest of this package it holds no arithmetic of
the method: it draws random numbers with torch's device generator and lays them out.

A batch of banded instances (workload 4): instance k has n_k columns and 4 n_k rows; row i of
an instance starts at column floor(i / rows_per_col) and holds w values, N(0,1), with the
entries that would fall at columns >= n_k set to zero (truncated band end, as in
`banded_problem`); b ~ N(0,1).  The draws differ from `banded_problem`'s (device Philox
instead of numpy), so the oracle checks such a batch on copies of sampled instances.
"""
from __future__ import annotations

import numpy as np

from .gen import SEED_BASE


def banded_batch_device(cols, rows_per_col=4, w=8, seed_offset=0, device="cuda", dtype=None):
    """Returns dict(vals (M, w) tensor, b (M,) tensor, cols, row0 (K + 1,), col0 (K + 1,) int64
    host arrays, lam) for instances of the given column counts, all on `device`."""
    import torch
    dtype = dtype or torch.float32
    cols = np.asarray(cols, dtype=np.int64)
    rows = rows_per_col * cols
    row0 = np.concatenate([[0], np.cumsum(rows)]).astype(np.int64)
    col0 = np.concatenate([[0], np.cumsum(cols)]).astype(np.int64)
    M = int(row0[-1])
    gen = torch.Generator(device=device)
    gen.manual_seed(SEED_BASE + 4 + 1000003 * seed_offset)
    vals = torch.randn((M, w), generator=gen, device=device, dtype=dtype)
    b = torch.randn((M,), generator=gen, device=device, dtype=dtype)
    # truncated band ends: the last rows_per_col * (w - 1) rows of each instance reach past it
    last = rows_per_col * (w - 1)
    local = np.arange(last, dtype=np.int64)
    for_rows, for_cols = [], []
    for k in range(cols.size):
        n = int(cols[k])
        i = rows[k] - last + local                       # local rows near the end
        i = i[i >= 0]
        s = i // rows_per_col
        c = np.arange(w, dtype=np.int64)[None, :]
        mask = (s[:, None] + c) >= n
        rr, cc = np.nonzero(mask)
        for_rows.append(row0[k] + i[rr])
        for_cols.append(cc)
    if for_rows:
        r = torch.from_numpy(np.concatenate(for_rows)).to(device)
        c = torch.from_numpy(np.concatenate(for_cols)).to(device)
        vals[r, c] = 0
    return dict(vals=vals, b=b, cols=cols, row0=row0, col0=col0, lam=1e-3, w=w, rows_per_col=rows_per_col)
