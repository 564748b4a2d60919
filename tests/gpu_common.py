"""Helpers shared by the GPU parity tests (inputs to tensors, oracle per-block solves)."""
import numpy as np

from oracle import householder as hh


def cuda_or_skip():
    import pytest
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def blocks_of(d, i):
    n, m = int(d["n"][i]), int(d["m"][i])
    v0 = int(d["val_off"][i])
    r0 = int(d["row_off"][i])
    A = np.asarray(d["vals"][v0:v0 + n * m], dtype=np.float64).reshape(m, n).T
    b = np.asarray(d["b"][r0:r0 + n], dtype=np.float64)
    return A, b


def oracle_block(d, i):
    A, b = blocks_of(d, i)
    x, f, qtb = hh.lstsq(A, b)
    return x, f, qtb, A, b


def optimality_all(d, x):
    """max over blocks of ||A^T (b - A x)|| / (||A||^2 ||x|| + ||A|| ||b||), vectorised by shape."""
    n = d["n"].astype(np.int64)
    m = d["m"].astype(np.int64)
    worst = 0.0
    for nn in np.unique(n):
        for mm in np.unique(m[n == nn]):
            idx = np.nonzero((n == nn) & (m == mm))[0]
            vo = d["val_off"][idx][:, None] + np.arange(nn * mm)[None, :]
            A = d["vals"][vo].astype(np.float64).reshape(-1, mm, nn).transpose(0, 2, 1)
            ro = d["row_off"][idx][:, None] + np.arange(nn)[None, :]
            b = d["b"][ro].astype(np.float64)
            co = d["col_off"][idx][:, None] + np.arange(mm)[None, :]
            xx = x[co].astype(np.float64)
            r = b - np.einsum("kij,kj->ki", A, xx)
            g = np.einsum("kij,ki->kj", A, r)
            nA = np.sqrt((A * A).sum(axis=(1, 2)))
            scale = nA * nA * np.linalg.norm(xx, axis=1) + nA * np.linalg.norm(b, axis=1)
            worst = max(worst, float((np.linalg.norm(g, axis=1) / scale).max()))
    return worst
