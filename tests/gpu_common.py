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


def stack_blocks(d, idx):
    """Blocks idx (all of one shape) as stacks: A (k, n, m), b (k, n), column offsets (k, m)."""
    nn, mm = int(d["n"][idx[0]]), int(d["m"][idx[0]])
    vo = d["val_off"][idx][:, None] + np.arange(nn * mm)[None, :]
    A = np.asarray(d["vals"], dtype=np.float64)[vo].reshape(-1, mm, nn).transpose(0, 2, 1)
    ro = d["row_off"][idx][:, None] + np.arange(nn)[None, :]
    b = np.asarray(d["b"], dtype=np.float64)[ro]
    co = d["col_off"][idx][:, None] + np.arange(mm)[None, :]
    return A, b, co


def block_errors(d, x, idx=None):
    """Per block of idx (default: all): relative error of x against the oracle's FP64 solution
    (householder.lstsq_stack, the per-block Householder solve taken over stacks of one shape)
    and the forward-error factor kappa + kappa^2 ||r|| / (||A||_2 ||x||) of least squares
    (kappa from singular values; a backward-stable solve in unit roundoff u is within a small
    multiple of u times this factor).  Returns (err, factor) in the order of idx."""
    K = d["K"]
    idx = np.arange(K) if idx is None else np.asarray(idx)
    n = d["n"].astype(np.int64)[idx]
    m = d["m"].astype(np.int64)[idx]
    err = np.zeros(len(idx))
    fac = np.zeros(len(idx))
    key = n * 16 + m
    for k in np.unique(key):
        sel = np.nonzero(key == k)[0]
        A, b, co = stack_blocks(d, idx[sel])
        xo = hh.lstsq_stack(A, b)
        xg = np.asarray(x, dtype=np.float64)[co]
        nx = np.linalg.norm(xo, axis=1)
        err[sel] = np.linalg.norm(xg - xo, axis=1) / nx
        s = np.linalg.svd(A, compute_uv=False)
        kap = s[:, 0] / s[:, -1]
        r = b - np.einsum("kij,kj->ki", A, xo)
        fac[sel] = kap + kap * kap * np.linalg.norm(r, axis=1) / (s[:, 0] * nx)
    return err, fac


U32, U64 = 2.0 ** -24, 2.0 ** -53


def assert_blocks_within(d, x, idx, tol, u_bound, c=None, what=""):
    """Every block of idx: error <= max(tol, c * n * m * u_bound * factor).  tol is the target
    of the mode (1e-5 for FP32 refined, 1e-12 for FP64); the bound term admits the blocks whose
    conditioning puts even a backward-stable solve in that precision (the oracle's own FP64
    solve included) above it.  Returns (max error, worst block)."""
    err, fac = block_errors(d, x, idx)
    idx = np.arange(d["K"]) if idx is None else np.asarray(idx)
    nm = d["n"].astype(np.float64)[idx] * d["m"].astype(np.float64)[idx]
    lim = np.maximum(tol, (2.0 if c is None else c) * nm * u_bound * fac)
    bad = np.nonzero(~(err <= lim))[0]
    assert bad.size == 0, (f"{what}{bad.size} blocks above their limit, e.g. block {int(idx[bad[0]])}: "
                           f"error {err[bad[0]]:.3e}, limit {lim[bad[0]]:.3e}, factor {fac[bad[0]]:.3e}")
    w = int(np.argmax(err))
    return float(err[w]), int(idx[w])


def block_kappa(d):
    """2-norm condition number of every block (singular values, by shape group)."""
    n = d["n"].astype(np.int64)
    m = d["m"].astype(np.int64)
    kap = np.zeros(d["K"])
    key = n * 16 + m
    for k in np.unique(key):
        sel = np.nonzero(key == k)[0]
        A = stack_blocks(d, sel)[0]
        s = np.linalg.svd(A, compute_uv=False)
        kap[sel] = s[:, 0] / s[:, -1]
    return kap


def assert_close(p, p_ref, tol, floor=1e-3, what=""):
    """The solution p against the oracle's p_ref: relative 2-norm error <= tol, and every
    component within tol (|p*_i| + floor ||p*||_inf), so that the small components of a
    badly scaled solution are weighed too.  Returns the relative 2-norm error."""
    p = np.asarray(p, dtype=np.float64)
    p_ref = np.asarray(p_ref, dtype=np.float64)
    e = np.linalg.norm(p - p_ref) / np.linalg.norm(p_ref)
    assert e <= tol, f"{what}relative error {e:.3e} > {tol:.1e}"
    lim = tol * (np.abs(p_ref) + floor * np.abs(p_ref).max())
    bad = np.nonzero(~(np.abs(p - p_ref) <= lim))[0]
    assert bad.size == 0, (f"{what}{bad.size} components outside tol (|p*| + {floor:g} ||p*||_inf), e.g. "
                           f"{int(bad[0])}: {p[bad[0]]!r} vs {p_ref[bad[0]]!r}")
    return e
