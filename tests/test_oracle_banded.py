"""Pins of the Sec. 4.4 block-banded oracle."""
import numpy as np
import pytest

from oracle import banded as bd
from oracle import householder as hh
from workloads import banded_problem


def damped_dense(start, vals, b, n, lam, D):
    s2, v2, r2, _ = bd.with_damping(start, vals, b, n, lam, D)
    return bd.assemble_dense(s2, v2, n), r2, s2, v2


@pytest.mark.parametrize("n,rpc,w,group", [(20, 4, 8, 8), (17, 3, 5, 4), (9, 4, 8, 1), (30, 2, 3, 16)])
def test_banded_equals_dense(n, rpc, w, group):
    d = banded_problem(n=n, rows_per_col=rpc, w=w, dtype=np.float64)
    D = bd.column_norms(d["start"], d["vals"], n)
    A, rhs, s2, v2 = damped_dense(d["start"], d["vals"], d["b"], n, d["lam"], D)
    x, Rw, c, res_sq, _ = bd.damped_solve(d["start"], d["vals"], d["b"], n, d["lam"], D, group)
    x_np = np.linalg.lstsq(A, rhs, rcond=None)[0]
    np.testing.assert_allclose(x, x_np, rtol=1e-10, atol=1e-12)
    R = bd.dense_R_from_windows(Rw)
    R_ref = hh.qr(A).R
    np.testing.assert_allclose(hh.normalise_row_signs(R), hh.normalise_row_signs(R_ref), atol=1e-11)
    # residual norm from the fronts equals the true residual
    r = rhs - A @ x
    assert res_sq == pytest.approx(float(r @ r), rel=1e-9)


def test_group_size_does_not_change_solution():
    d = banded_problem(n=50, rows_per_col=4, w=8, dtype=np.float64)
    xs = [bd.damped_solve(d["start"], d["vals"], d["b"], 50, d["lam"], group=g)[0] for g in (1, 5, 8, 32)]
    for x in xs[1:]:
        np.testing.assert_allclose(x, xs[0], rtol=1e-11, atol=1e-13)


def test_householder_vectors_are_short():
    """Every front (Householder vector length) is bounded by the band, not by M (Sec. 4.4)."""
    n, rpc, w, g = 400, 4, 8, 8
    d = banded_problem(n=n, rows_per_col=rpc, w=w, dtype=np.float64)
    D = bd.column_norms(d["start"], d["vals"], n)
    s2, v2, r2, _ = bd.with_damping(d["start"], d["vals"], d["b"], n, d["lam"], D)
    _, _, _, fronts = bd.qr_fronts(s2, v2, r2, n, g)
    assert max(fr[1] for fr in fronts) <= (w - 1) + (rpc + 1) * g
    assert len(fronts) == n // g


def test_optimality_identity_at_larger_size():
    n = 3000
    d = banded_problem(n=n, rows_per_col=4, w=8, dtype=np.float64)
    x, Rw, c, res_sq, D = bd.damped_solve(d["start"], d["vals"], d["b"], n, d["lam"])
    r = d["b"] - bd.matvec(d["start"], d["vals"], x)
    g = bd.rmatvec(d["start"], d["vals"], r, n) - d["lam"] * D * D * x
    scale = np.linalg.norm(d["vals"]) ** 2 * np.linalg.norm(x)
    assert np.linalg.norm(g) / scale < 1e-14


def test_planted_mistake_dropped_carry_is_caught(monkeypatch):
    """Throwing away the carried rows between fronts changes R and the solution."""
    n = 24
    d = banded_problem(n=n, rows_per_col=4, w=8, dtype=np.float64)
    D = bd.column_norms(d["start"], d["vals"], n)
    A, rhs, _, _ = damped_dense(d["start"], d["vals"], d["b"], n, d["lam"], D)
    x_np = np.linalg.lstsq(A, rhs, rcond=None)[0]
    real = bd._reduce_front

    def bad(F, f_rhs):
        Rf, q = real(F, f_rhs)
        return Rf[: min(Rf.shape[0], 8)], q
    monkeypatch.setattr(bd, "_reduce_front", bad)
    try:
        x, *_ = bd.damped_solve(d["start"], d["vals"], d["b"], n, d["lam"], D, 8)
        assert np.linalg.norm(x - x_np) > 1e-6 * np.linalg.norm(x_np)
    except ValueError:
        pass
