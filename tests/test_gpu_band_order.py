"""The band-exposing permutations of Sec. 4.3 handed to the GPU banded QR (Sec. 4.4).

A banded matrix with its rows and columns shuffled has no visible band; qrkit_band_order finds
P_r, P_c, the row starts and the width, the caller packs the permuted rows as windows, and a
QRKIT_STRUCT_BANDED plan with explicit row starts factors and solves them.  The solution,
mapped back through P_c, must equal the oracle's on the windowed system and the dense
least-squares solution of the original (scrambled) damped system.
"""
import numpy as np
import pytest

from oracle import banded as bd
from paper_1802_03773_gb300 import qrkit
from tests.gpu_common import assert_close, cuda_or_skip
from tests.test_oracle_reorder import csr, scrambled_band

pytestmark = pytest.mark.gpu


def scrambled_system(n, rpc, w, seed, dtype):
    rows_cols = scrambled_band(n, rpc, w, seed)
    g = np.random.default_rng(seed + 77)
    M = len(rows_cols)
    A = np.zeros((M, n))
    for i, r in enumerate(rows_cols):
        A[i, r] = g.standard_normal(len(r))
    A = A.astype(dtype).astype(np.float64)
    b = g.standard_normal(M).astype(dtype).astype(np.float64)
    return rows_cols, A, b


def windows(A, b, rows_cols):
    """P_r A P_c as rows of `width` values starting at row_start, and P_r b."""
    M, n = A.shape
    col_perm, row_perm, row_start, width = qrkit.band_order(M, n, *csr(rows_cols))
    Ap = A[row_perm][:, col_perm]
    vals = np.zeros((M, width))
    for k in range(M):
        hi = min(n, row_start[k] + width)
        vals[k, :hi - row_start[k]] = Ap[k, row_start[k]:hi]
    return col_perm, row_start, width, vals, b[row_perm]


def dense_damped(A, b, lam):
    D = np.sqrt((A * A).sum(axis=0))
    D[D == 0] = 1.0
    Aa = np.vstack([A, np.sqrt(lam) * np.diag(D)])
    return np.linalg.lstsq(Aa, np.concatenate([b, np.zeros(A.shape[1])]), rcond=None)[0]


@pytest.mark.parametrize("solver", [qrkit.BAND_SWEEP, qrkit.BAND_PARALLEL])
@pytest.mark.parametrize("precision,steps,tol", [("fp64", 0, 1e-11), ("fp32_refined", 2, 1e-5)])
def test_band_order_feeds_the_banded_qr(solver, precision, steps, tol):
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context
    dt = np.float64 if precision == "fp64" else np.float32
    n, rpc, w, lam = 600, 3, 6, 1e-3
    rows_cols, A, b = scrambled_system(n, rpc, w, 5, dt)
    col_perm, row_start, width, vals, bp = windows(A, b, rows_cols)
    assert width == w
    D = bd.column_norms(row_start, vals, n)
    x_ref = bd.damped_solve(row_start, vals, bp, n, lam, D)[0]
    ctx = Context(0, precision=precision)
    ctx.plan_banded([n], window=width, solver=solver, row_start=row_start)
    J = torch.from_numpy(vals.astype(dt)).cuda()
    tb = torch.from_numpy(bp.astype(dt)).cuda()
    p = torch.empty(n, device="cuda", dtype=ctx.dtype)
    ctx.factor_solve(J, tb, p, None, None, lam, refine_steps=steps)
    ctx.sync_status()
    x = p.cpu().numpy().astype(np.float64)
    ctx.close()
    assert_close(x, x_ref, tol)
    # back through P_c: the solution of the original, scrambled system
    x_orig = np.empty(n)
    x_orig[col_perm] = x
    assert_close(x_orig, dense_damped(A, b, lam), tol * 10 if precision == "fp64" else tol)


def test_band_order_batch_of_instances():
    """Three scrambled systems of different sizes in one batch with explicit starts."""
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context
    lam = 1e-2
    sizes = [(150, 2, 5, 11), (400, 4, 8, 12), (75, 1, 3, 13)]
    cols, rows, starts, vals_all, b_all, refs = [], [], [], [], [], []
    for n, rpc, w, seed in sizes:
        rows_cols, A, b = scrambled_system(n, rpc, w, seed, np.float64)
        col_perm, row_start, width, vals, bp = windows(A, b, rows_cols)
        pad = np.zeros((vals.shape[0], 8))
        pad[:, :width] = vals
        cols.append(n)
        rows.append(vals.shape[0])
        starts.append(row_start)
        vals_all.append(pad)
        b_all.append(bp)
        refs.append(bd.damped_solve(row_start, pad, bp, n, lam)[0])
    ctx = Context(0, precision="fp64")
    ctx.plan_banded(cols, window=8, solver=qrkit.BAND_PARALLEL, row_start=np.concatenate(starts),
                    instance_rows=rows)
    J = torch.from_numpy(np.vstack(vals_all)).cuda()
    tb = torch.from_numpy(np.concatenate(b_all)).cuda()
    p = torch.empty(sum(cols), device="cuda", dtype=torch.float64)
    ctx.factor_solve(J, tb, p, None, None, lam, refine_steps=0)
    ctx.sync_status()
    x = p.cpu().numpy()
    ctx.close()
    off = np.concatenate([[0], np.cumsum(cols)])
    for k in range(len(sizes)):
        assert_close(x[off[k]:off[k + 1]], refs[k], 1e-11, what=f"instance {k}: ")


def test_explicit_starts_are_validated():
    cuda_or_skip()
    from paper_1802_03773_gb300 import Context, QRKitError
    ctx = Context(0, precision="fp64")
    with pytest.raises(QRKitError) as e:
        ctx.plan_banded([10], window=3, row_start=np.array([0, 2, 1, 5]))     # decreasing
    assert e.value.status == 1
    with pytest.raises(QRKitError) as e:
        ctx.plan_banded([10], window=3, row_start=np.array([0, 2, 10]))       # past the last column
    assert e.value.status == 1
    with pytest.raises(QRKitError) as e:
        ctx.plan_banded([10, 5], window=3, row_start=np.array([0, 1, 0]))     # batch without instance_rows
    assert e.value.status == 1
    ctx.close()
