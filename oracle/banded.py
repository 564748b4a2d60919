"""Block-banded QR with short block-wise Householder vectors, float64 (test infrastructure only).

Follows Sec. 4.4 of the paper ("Block banded"): instead of Householder vectors of length
M over the whole matrix, each step factorizes a group of r columns of a small dense
front whose rows are the rows that can touch those columns, so every Householder
vector has the length of its front; Q is kept as the sequence of per-front reflectors
(Eq. "blockBandedYTY") and R comes out banded.

Matrix format: a row-sorted banded matrix given row by row as a window
    row k has values vals[k, 0..w-1] at columns start[k] .. start[k] + w - 1,
with start non-decreasing (the row permutation P_r of Sec. 4.3 / 4.5 has been applied)
and window entries at columns >= N equal to zero (a truncated band end).

Front of column group [c0, c1):
    rows  = rows carried from the previous front (non-zero only in columns >= c0)
            + the rows whose window starts in [c0, c1)
    cols  = [c0, min(c1 + w - 1, N))   (the farthest column those rows reach)
  Householder reflectors (householder.house) on every column of the front, in column
  order (a dense QR of the front; a front may be wider than tall at the band end).
  Its first c1 - c0 rows are final
  rows of R; the next rows (at most w - 1, non-zero only in columns >= c1) are carried;
  any further rows are zero and their transformed right-hand side is residual.

Readings (the paper gives the update formula and the block sizes, not a row schedule):
  * The row set of a front is "carried rows + rows that start in the group", the
    schedule that keeps each Householder vector short (the paper's n_k + n_{k+1}).
  * R is stored as windows: row j holds R[j, j .. j + w - 1].  R of a matrix whose rows
    span w consecutive columns has upper bandwidth w - 1, and the front reduction keeps
    the entries outside it exactly zero (checked).

Pins (tests/test_oracle_banded.py): same R (up to row signs) and the same solution as
dense Householder QR (householder.qr) of the assembled matrix and numpy.linalg.lstsq;
the optimality identity at sizes the dense solve cannot reach; the result does not
depend on the group size r.  column_norms (tests/test_oracle_damping_pins.py): a hand-worked
example (with an entry past the last column, dropped), the norms of the assembled matrix,
and planted mistakes (squared norms, no zero -> 1, entries past the end kept) that fail.
"""
from __future__ import annotations

import numpy as np

from . import householder as hh


def assemble_dense(start, vals, N):
    """Dense M x N matrix of a windowed row set (small problems only)."""
    start = np.asarray(start, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    M, w = vals.shape
    A = np.zeros((M, N))
    for k in range(M):
        for t in range(w):
            col = start[k] + t
            if col < N:
                A[k, col] += vals[k, t]
            elif vals[k, t] != 0.0:
                raise ValueError("window entry beyond the last column must be zero")
    return A


def matvec(start, vals, p):
    """J p for a windowed row set (vectorised; any size)."""
    start = np.asarray(start, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    M, w = vals.shape
    N = p.shape[0]
    out = np.zeros(M)
    for t in range(w):
        col = start + t
        ok = col < N
        out[ok] += vals[ok, t] * p[col[ok]]
    return out


def rmatvec(start, vals, r, N):
    """J^T r for a windowed row set (vectorised; any size)."""
    start = np.asarray(start, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    M, w = vals.shape
    out = np.zeros(N)
    for t in range(w):
        col = start + t
        ok = col < N
        np.add.at(out, col[ok], vals[ok, t] * r[ok])
    return out


def column_norms(start, vals, N):
    """D = diag(J^T J)^(1/2) (Sec. 5.2); a zero norm becomes 1 (reading, MINPACK)."""
    start = np.asarray(start, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    M, w = vals.shape
    sq = np.zeros(N)
    for t in range(w):
        col = start + t
        ok = col < N
        np.add.at(sq, col[ok], vals[ok, t] ** 2)
    d = np.sqrt(sq)
    d[d == 0.0] = 1.0
    return d


def with_damping(start, vals, b, N, lam, D):
    """P_r [J; lambda^(1/2) D] and P_r [b; 0] (Sec. 4.5 / Sec. 5.2), as a sorted window set.

    The damping row of column j is the window starting at j with lambda^(1/2) D_j first.
    Rows are sorted stably by (start column, J rows before damping rows, original index).
    Returns (start, vals, rhs, order) where order[k] is the source row of row k
    (J rows 0..M-1, damping row of column j = M + j).
    """
    start = np.asarray(start, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    M, w = vals.shape
    lam_half = np.sqrt(lam)
    d_start = np.arange(N, dtype=np.int64)
    d_vals = np.zeros((N, w))
    d_vals[:, 0] = lam_half * np.asarray(D, dtype=np.float64)
    all_start = np.concatenate([start, d_start])
    all_vals = np.vstack([vals, d_vals])
    all_rhs = np.concatenate([np.asarray(b, dtype=np.float64), np.zeros(N)])
    src = np.concatenate([np.zeros(M, dtype=np.int64), np.ones(N, dtype=np.int64)])
    order = np.lexsort((np.arange(M + N), src, all_start))
    return all_start[order], all_vals[order], all_rhs[order], order


def qr_fronts(start, vals, rhs, N, group=8):
    """Sec. 4.4 block-banded QR.  Returns (Rw, c, residual_sq, fronts).

    Rw[j, t] = R[j, j + t] (t < w); c = top N entries of Q^T rhs; residual_sq = squared
    norm of the rest of Q^T rhs; fronts = list of (c0, n_rows, n_cols) (the Householder
    vector lengths, for the short-vector check).
    """
    start = np.asarray(start, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    rhs = np.asarray(rhs, dtype=np.float64)
    M, w = vals.shape
    if M and np.any(np.diff(start) < 0):
        raise ValueError("rows must be sorted by start column (apply P_r first)")
    Rw = np.zeros((N, w))
    c = np.zeros(N)
    res_sq = 0.0
    carried = np.zeros((0, 0))     # carried rows, dense over columns [c_prev1, ...)
    carried_rhs = np.zeros(0)
    carried_c0 = 0
    fronts = []
    ptr = 0
    for c0 in range(0, N, group):
        c1 = min(c0 + group, N)
        hi = min(c1 + w - 1, N)
        width = hi - c0
        # rows starting in this group
        end = ptr
        while end < M and start[end] < c1:
            end += 1
        if end > ptr and start[ptr] < c0:
            raise ValueError("row starts before its group: rows are not sorted")
        new = np.zeros((end - ptr, width))
        for k in range(ptr, end):
            for t in range(w):
                col = start[k] + t
                if col < N:
                    new[k - ptr, col - c0] = vals[k, t]
                elif vals[k, t] != 0.0:
                    raise ValueError("window entry beyond the last column must be zero")
        old = np.zeros((carried.shape[0], width))
        if carried.shape[0]:
            off = carried_c0 - c0
            ncol = min(carried.shape[1], width - off)
            old[:, off:off + ncol] = carried[:, :ncol]
            if np.any(carried[:, ncol:] != 0.0):
                raise ValueError("carried row reaches past the front")
        F = np.vstack([old, new])
        f_rhs = np.concatenate([carried_rhs, rhs[ptr:end]])
        ptr = end
        g = c1 - c0
        if F.shape[0] < g:
            raise ValueError("front has fewer rows than columns: rank deficient")
        fronts.append((c0, F.shape[0], width))
        Rf, qt = _reduce_front(F, f_rhs)
        nR = Rf.shape[0]
        for j in range(g):
            row = Rf[j]
            gj = c0 + j
            tw = min(w, N - gj)
            Rw[gj, :tw] = row[j:j + tw]
            if np.any(row[j + tw:] != 0.0):
                raise ValueError("R entry outside the band")
            c[gj] = qt[j]
        ncarry = nR - g
        carried = Rf[g:nR, g:] if ncarry > 0 else np.zeros((0, 0))
        carried_rhs = qt[g:nR]
        carried_c0 = c1
        res_sq += float(np.dot(qt[nR:], qt[nR:]))
    return Rw, c, res_sq, fronts


def _reduce_front(F, f_rhs):
    """Householder reflectors (Sec. 2) on columns 0 .. min(rows, cols) - 1 of a front.

    Returns the upper-trapezoidal rows of the reduced front and the reflected rhs.
    """
    F = np.array(F, dtype=np.float64, copy=True)
    q = np.array(f_rhs, dtype=np.float64, copy=True)
    f, width = F.shape
    kmax = min(f, width)
    for k in range(kmax):
        v, t, beta = hh.house(F[k:, k])
        if k + 1 < width:
            F[k:, k + 1:] -= t * np.outer(v, v @ F[k:, k + 1:])
        F[k, k] = beta
        F[k + 1:, k] = 0.0
        q[k:] -= t * v * np.dot(v, q[k:])
    return F[:kmax], q


def back_substitute(Rw, c):
    """Solve the banded R x = c (R row j stored as Rw[j, t] = R[j, j + t])."""
    N, w = Rw.shape
    x = np.zeros(N)
    for j in reversed(range(N)):
        tw = min(w, N - j)
        x[j] = (c[j] - np.dot(Rw[j, 1:tw], x[j + 1:j + tw])) / Rw[j, 0]
    return x


def solve(start, vals, rhs, N, group=8):
    """Banded least-squares solve: returns (x, Rw, c, residual_sq)."""
    Rw, c, res_sq, _ = qr_fronts(start, vals, rhs, N, group)
    return back_substitute(Rw, c), Rw, c, res_sq


def damped_solve(start, vals, b, N, lam, D=None, group=8):
    """min || P_r [J; lambda^(1/2) D] p - P_r [b; 0] || for a banded J (Secs. 4.4, 4.5, 5.2)."""
    if D is None:
        D = column_norms(start, vals, N)
    s2, v2, r2, _ = with_damping(start, vals, b, N, lam, D)
    x, Rw, c, res_sq = solve(s2, v2, r2, N, group)
    return x, Rw, c, res_sq, D


def dense_R_from_windows(Rw):
    N, w = Rw.shape
    R = np.zeros((N, N))
    for j in range(N):
        tw = min(w, N - j)
        R[j, j:j + tw] = Rw[j, :tw]
    return R
