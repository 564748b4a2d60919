"""Composed sparse QR of the damped least-squares system, float64 (test infrastructure only).

The problem is Eq. (2) of the paper: min || [J; lambda^(1/2) D] p - [b; 0] ||, the
QR form of the LM step Eq. (1), (J^T J + lambda D^2) p = J^T b.

Structures covered (the compositions the workloads use):
  * block-angular  J = [blkdiag(J_1..J_K) | S]  with S dense (every block row touches all
    s shared columns) or windowed (block i's rows touch w consecutive shared columns
    starting at start_i), plus the damping rows lambda^(1/2) D;
  * plain block diagonal (S absent, s = 0).

Steps, in the paper's order:
  * D = diag(J^T J)^(1/2), the column norms of J (Sec. 5.2, Backtrack LM).  A zero column
    norm is replaced by 1 (reading: the paper is silent; MINPACK's convention).
  * Vertical concatenation by row interleave (Sec. 4.5, Sec. 5.2): P_r puts the damping
    row of each block column right after that block's J rows, and the damping rows of
    the shared columns after everything else, so that P_r [J; lambda^(1/2) D] is again
    block-angular:  [[blkdiag(B_i), C], [0, lambda^(1/2) D_S]] with
    B_i = [J_i; lambda^(1/2) D_i] and C_i = [S_i; 0].
  * Block diagonal QR (Sec. 4.1): Q_i R_i = qr(B_i) for every block independently.
  * Horizontal concatenation (Sec. 4.2): Q_1^T A_2 splits into the top rows
    (R12_i = Q_i^T C_i, top m_i rows) and the bottom rows (Q_perp_i^T C_i), which are
    stacked with lambda^(1/2) D_S into the reduced shared block; Q' R' = qr(reduced).
  * Solve (Sec. 5.1): R_S p_S = c_S, then R_i p_i = c_i - R12_i p_S per block.

P_r ordering rule (reading: the paper gives no tie rule): rows sorted stably by
(leading column, J rows before damping rows, original index).

Pins (tests/test_oracle_structured.py): the composed solve equals a dense Householder
solve of the assembled matrix and numpy.linalg.lstsq; the optimality identity
J^T (b - J p) = lambda D^2 p; closed forms for one-column blocks and for J = I, D = I;
R^T R = A^T A for the composed R; Parseval for Q^T [b; 0].  column_norms
(tests/test_oracle_damping_pins.py): a hand-worked example with whole-number norms, the
norms of the assembled J, and planted mistakes (squared norms, no zero -> 1, damping rows
counted) that fail.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import householder as hh


@dataclass
class BlockProblem:
    """Block-angular damped least-squares problem (all arrays float64, host).

    blocks[i]   : n_i x m_i dense J block
    coupled[i]  : n_i x w dense rows of S for block i (w = s for dense S) or None
    start[i]    : first shared column touched by block i (0 for dense S)
    s           : number of shared columns
    b           : right-hand side, length sum(n_i), in block order
    D           : length N = sum(m_i) + s diagonal (None: column norms of J)
    lam         : damping lambda >= 0
    """
    blocks: list
    b: np.ndarray
    lam: float = 0.0
    coupled: list | None = None
    start: np.ndarray | None = None
    s: int = 0
    D: np.ndarray | None = None

    @property
    def K(self):
        return len(self.blocks)

    def shapes(self):
        return [blk.shape for blk in self.blocks]

    def col_offsets(self):
        m = np.array([blk.shape[1] for blk in self.blocks], dtype=np.int64)
        return np.concatenate([[0], np.cumsum(m)])

    def row_offsets(self):
        n = np.array([blk.shape[0] for blk in self.blocks], dtype=np.int64)
        return np.concatenate([[0], np.cumsum(n)])

    @property
    def n_block_cols(self):
        return int(self.col_offsets()[-1])

    @property
    def N(self):
        return self.n_block_cols + self.s

    @property
    def M(self):
        return int(self.row_offsets()[-1])


def assemble_J(P: BlockProblem) -> np.ndarray:
    """J = [blkdiag(J_i) | S] as a dense M x N matrix (small problems only)."""
    ro, co = P.row_offsets(), P.col_offsets()
    J = np.zeros((P.M, P.N))
    nb = P.n_block_cols
    for i, blk in enumerate(P.blocks):
        J[ro[i]:ro[i + 1], co[i]:co[i + 1]] = blk
        if P.coupled is not None and P.s > 0:
            w = P.coupled[i].shape[1]
            st = 0 if P.start is None else int(P.start[i])
            J[ro[i]:ro[i + 1], nb + st:nb + st + w] = P.coupled[i]
    return J


def column_norms(P: BlockProblem) -> np.ndarray:
    """D = diag(J^T J)^(1/2) (Sec. 5.2); a zero norm becomes 1 (reading, MINPACK)."""
    nb = P.n_block_cols
    sq = np.zeros(P.N)
    co = P.col_offsets()
    for i, blk in enumerate(P.blocks):
        sq[co[i]:co[i + 1]] += np.sum(blk * blk, axis=0)
        if P.coupled is not None and P.s > 0:
            w = P.coupled[i].shape[1]
            st = 0 if P.start is None else int(P.start[i])
            sq[nb + st:nb + st + w] += np.sum(P.coupled[i] ** 2, axis=0)
    d = np.sqrt(sq)
    d[d == 0.0] = 1.0
    return d


def damping(P: BlockProblem) -> np.ndarray:
    return column_norms(P) if P.D is None else np.asarray(P.D, dtype=np.float64)


def row_permutation(P: BlockProblem):
    """P_r for [J; lambda^(1/2) D] (Sec. 4.5, Sec. 5.2), as a list of source rows.

    Source row ids: J rows are 0..M-1, the damping row of column j is M + j.
    Sorted stably by (leading column, J rows before damping rows, original index).
    Returns an int64 array `order` with augmented row k = source row order[k].
    Rows of an all-zero block row would have no leading column; they are placed by their
    block's first column (reading).
    """
    ro, co = P.row_offsets(), P.col_offsets()
    keys = []
    for i, blk in enumerate(P.blocks):
        for r in range(blk.shape[0]):
            nz = np.nonzero(blk[r])[0]
            lead = co[i] + (int(nz[0]) if nz.size else 0)
            keys.append((lead, 0, ro[i] + r))
    for j in range(P.N):
        keys.append((j, 1, P.M + j))
    keys.sort()
    return np.array([k[2] for k in keys], dtype=np.int64)


def assemble_augmented(P: BlockProblem):
    """(A, rhs) = P_r [J; lambda^(1/2) D], P_r [b; 0] as dense arrays (small problems)."""
    J = assemble_J(P)
    D = damping(P)
    lam_half = np.sqrt(P.lam)
    A_src = np.vstack([J, lam_half * np.diag(D)])
    rhs_src = np.concatenate([np.asarray(P.b, dtype=np.float64), np.zeros(P.N)])
    order = row_permutation(P)
    return A_src[order], rhs_src[order]


@dataclass
class ComposedFactor:
    """The composed factorization of Secs. 4.1, 4.2, 4.5 for a block-angular problem."""
    block_factors: list = field(default_factory=list)   # hh.QRFactor of each B_i
    R12: list = field(default_factory=list)             # m_i x w (Q_i^T C_i, top rows)
    c_blocks: list = field(default_factory=list)        # m_i (top of Q_i^T [b_i; 0])
    reduced: np.ndarray | None = None                   # (sum n_i + s) x s reduced block
    reduced_rhs: np.ndarray | None = None
    reduced_factor: hh.QRFactor | None = None
    c_S: np.ndarray | None = None
    residual_sq: float = 0.0                            # ||bottom of Q^T [b; 0]||^2


def augmented_block(P: BlockProblem, i: int, D: np.ndarray, co=None, ro=None):
    """B_i = [J_i; lambda^(1/2) D_i], C_i = [S_i; 0], rhs [b_i; 0] (Sec. 4.5 row interleave).
    co, ro: the problem's column and row offsets, if the caller already has them."""
    blk = np.asarray(P.blocks[i], dtype=np.float64)
    n, m = blk.shape
    if co is None or ro is None:
        co, ro = P.col_offsets(), P.row_offsets()
    lam_half = np.sqrt(P.lam)
    rows = [blk]
    if P.lam > 0.0:
        rows.append(lam_half * np.diag(D[co[i]:co[i + 1]]))
    B = np.vstack(rows)
    rhs = np.concatenate([np.asarray(P.b[ro[i]:ro[i + 1]], dtype=np.float64),
                          np.zeros(B.shape[0] - n)])
    C = None
    if P.coupled is not None and P.s > 0:
        w = P.coupled[i].shape[1]
        C = np.vstack([np.asarray(P.coupled[i], dtype=np.float64), np.zeros((B.shape[0] - n, w))])
    return B, C, rhs


def factor_and_solve(P: BlockProblem, reduced_solver=None):
    """Composed QR solve of the damped block-angular problem.

    reduced_solver(rows, rhs, start, s, src) -> (p_S, R_S, c_S, residual_sq) factors the
    reduced shared block; default is dense Householder (hh.qr) on the assembled reduced
    block (the windowed case may pass the banded solver of Sec. 4.4 instead).
    Returns (p, ComposedFactor).
    """
    D = damping(P)
    F = ComposedFactor()
    nb = P.n_block_cols
    s = P.s
    red_rows, red_rhs, red_start = [], [], []
    p_blocks = []
    co, ro = P.col_offsets(), P.row_offsets()
    for i in range(P.K):
        B, C, rhs = augmented_block(P, i, D, co, ro)
        m = B.shape[1]
        f = hh.qr(B)                                  # Sec. 4.1: Q_i R_i = qr(B_i)
        qtb = hh.apply_qt(f, rhs)
        F.block_factors.append(f)
        F.c_blocks.append(qtb[:m])
        if C is not None:
            qtc = hh.apply_qt(f, C)                   # Sec. 4.2: Q_i^T C_i
            F.R12.append(qtc[:m])
            red_rows.append(qtc[m:])
            st = 0 if P.start is None else int(P.start[i])
            red_start.extend([st] * (qtc.shape[0] - m))
            red_rhs.append(qtb[m:])
        else:
            F.R12.append(np.zeros((m, 0)))
            F.residual_sq += float(np.dot(qtb[m:], qtb[m:]))
    if s > 0:
        w = P.coupled[0].shape[1]
        lam_half = np.sqrt(P.lam)
        red_src = [0] * len(red_start)
        # damping rows of the shared columns (Sec. 4.5): the row of column j has its one
        # non-zero at column j; as a window it starts at j (dense S: window = all columns)
        for j in range(s):
            if P.lam > 0.0:
                row = np.zeros(w)
                if w == s:
                    row[j] = lam_half * D[nb + j]
                    red_start.append(0)
                else:
                    row[0] = lam_half * D[nb + j]
                    red_start.append(j)
                red_rows.append(row[None, :])
                red_rhs.append(np.zeros(1))
                red_src.append(1)
        A_red_rows = np.vstack(red_rows)
        rhs_red = np.concatenate(red_rhs)
        start_arr = np.array(red_start, dtype=np.int64)
        if reduced_solver is None:
            A_red = _expand_windows(A_red_rows, start_arr, s)
            fr = hh.qr(A_red)                         # Sec. 4.2: Q' R' = qr(bottom rows)
            qt = hh.apply_qt(fr, rhs_red)
            c_S = qt[:s]
            p_S = hh.back_substitute(fr.R, c_S)
            F.reduced_factor = fr
            F.reduced = A_red
            F.residual_sq += float(np.dot(qt[s:], qt[s:]))
            R_S = fr.R
        else:
            p_S, R_S, c_S, res_sq = reduced_solver(A_red_rows, rhs_red, start_arr, s,
                                                   np.array(red_src, dtype=np.int64))
            F.residual_sq += res_sq
        F.reduced_rhs = rhs_red
        F.c_S = c_S
    else:
        p_S = np.zeros(0)
    for i in range(P.K):
        f = F.block_factors[i]
        rhs = F.c_blocks[i]
        if s > 0:
            w = F.R12[i].shape[1]
            st = 0 if P.start is None else int(P.start[i])
            rhs = rhs - F.R12[i] @ p_S[st:st + w]
        p_blocks.append(hh.back_substitute(f.R, rhs))   # R_i p_i = c_i - R12_i p_S
    p = np.concatenate(p_blocks + [p_S])
    return p, F


def _expand_windows(rows: np.ndarray, start: np.ndarray, s: int) -> np.ndarray:
    w = rows.shape[1]
    if w == s:
        return np.array(rows, dtype=np.float64)
    A = np.zeros((rows.shape[0], s))
    for r in range(rows.shape[0]):
        tw = min(w, s - int(start[r]))
        A[r, start[r]:start[r] + tw] = rows[r, :tw]
        if np.any(rows[r, tw:] != 0.0):
            raise ValueError("window entry beyond the last shared column must be zero")
    return A


def banded_reduced_solver(group=8):
    """Reduced-block solver for windowed S: P_r sort, then the Sec. 4.4 banded QR."""
    from . import banded

    def solve(rows, rhs, start, s, src):
        order = np.lexsort((np.arange(rows.shape[0]), src, start))
        x, Rw, c, res_sq = banded.solve(start[order], rows[order], rhs[order], s, group)
        return x, Rw, c, res_sq
    return solve


def solve_dense(P: BlockProblem):
    """O1: dense Householder QR of the assembled P_r [J; lambda^(1/2) D] (small problems)."""
    A, rhs = assemble_augmented(P)
    x, f, qtb = hh.lstsq(A, rhs)
    return x, f, qtb


def optimality_residual(J, b, D, lam, p) -> float:
    """|| J^T (b - J p) - lambda D^2 p || / (||J||_F^2 ||p|| + ||J||_F ||b||): zero at the optimum.

    The first-order condition of Eq. (2) is J^T (b - J p) = lambda D^2 p, i.e. Eq. (1).
    J may be a dense array or a scipy.sparse matrix.
    """
    r = b - J @ p
    g = J.T @ r - lam * (D * D) * p
    if hasattr(J, "multiply"):
        fro = float(np.sqrt(J.multiply(J).sum()))
    else:
        fro = float(np.linalg.norm(J))
    scale = fro * fro * float(np.linalg.norm(p)) + fro * float(np.linalg.norm(b))
    return float(np.linalg.norm(g)) / max(scale, 1e-300)


def structural_rows(P: BlockProblem, damped: bool):
    """The column sets of the rows of [J; lambda^(1/2) D] from the structure alone (Sec. 3, 4.1,
    4.2, 4.5): a J row of block i touches the block's columns and its coupled columns (all s
    for a dense S; start_i .. start_i + w - 1 within the s shared columns for a window); the
    damping row of column j (when damped) touches j.  Source row ids as in row_permutation."""
    ro, co = P.row_offsets(), P.col_offsets()
    nb = P.n_block_cols
    rows = {}
    for i, blk in enumerate(P.blocks):
        cols = list(range(int(co[i]), int(co[i + 1])))
        if P.coupled is not None and P.s > 0:
            w = P.coupled[i].shape[1]
            st0 = 0 if P.start is None else int(P.start[i])
            cols += [nb + c for c in range(st0, min(st0 + w, P.s))]
        for r in range(blk.shape[0]):
            rows[int(ro[i]) + r] = cols
    if damped:
        for j in range(P.N):
            rows[P.M + j] = [j]
    return rows


def r_pattern(P: BlockProblem, damped: bool):
    """Structural non-zero pattern of R for the rows of P_r [J; lambda^(1/2) D] in natural column
    order, by symbolic row merging (the structure of the row-merge QR of Sec. 5.2 / the oracle
    O2 description): rows are taken in P_r order; a row whose leading column c has no R row yet
    becomes R row c, otherwise it is merged with R row c (the 2 x 2 reflection mixes them: R
    row c takes the union of the two patterns, and the row continues from its next column with
    that union).  Returns (row_ptr (N + 1), col_idx) with each R row's
    columns ascending; an R row that no row reaches stays empty."""
    rows = structural_rows(P, damped)
    order = [k for k in structural_row_order(P, damped)]
    R = [None] * P.N
    for k in order:
        cur = sorted(set(rows[int(k)]))
        while cur:
            c = cur[0]
            if R[c] is None:
                R[c] = cur
                break
            # the 2 x 2 reflection mixes the two rows: both take the union of the patterns
            R[c] = sorted(set(R[c]) | set(cur))
            cur = [x for x in R[c] if x > c]
    ptr = [0]
    idx = []
    for c in range(P.N):
        if R[c] is not None:
            idx += R[c]
        ptr.append(len(idx))
    return np.array(ptr, dtype=np.int64), np.array(idx, dtype=np.int32)


def structural_row_order(P: BlockProblem, damped: bool):
    """P_r from the structure alone: the J rows of block i lead at the block's first column,
    the damping row of column j (when damped) at j; sorted stably by (leading column, J rows
    before damping rows, source index).  Equal to row_permutation when no J row starts with a
    zero (the tie rule of reading 7)."""
    ro, co = P.row_offsets(), P.col_offsets()
    keys = []
    for i, blk in enumerate(P.blocks):
        for r in range(blk.shape[0]):
            keys.append((int(co[i]), 0, int(ro[i]) + r))
    if damped:
        for j in range(P.N):
            keys.append((j, 1, P.M + j))
    keys.sort()
    return np.array([k[2] for k in keys], dtype=np.int64)
