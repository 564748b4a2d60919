"""Pins of the curve-fit model and the Nielsen-rule LM oracle (Sec. 2, Sec. 5.2)."""
import numpy as np
import pytest

from oracle import curvefit as cf
from oracle import lm
from oracle import structured as st
from workloads import curvefit_problem


def test_basis_partition_of_unity_and_derivative():
    u = np.linspace(0, 1, 11)
    np.testing.assert_allclose(cf.basis(u).sum(axis=1), 1.0, atol=1e-15)
    np.testing.assert_allclose(cf.dbasis(u).sum(axis=1), 0.0, atol=1e-15)
    h = 1e-6
    np.testing.assert_allclose(cf.dbasis(u), (cf.basis(u + h) - cf.basis(u - h)) / (2 * h), atol=1e-9)


def test_curve_reproduces_line():
    """Control points P_k = (k, 2k): the uniform cubic B-spline is the line (t + 1, 2 (t + 1))."""
    Kc = 12
    P = np.stack([np.arange(Kc), 2 * np.arange(Kc)], axis=1).astype(np.float64)
    t = np.linspace(0, Kc - 3, 37)
    np.testing.assert_allclose(cf.curve(t, P), np.stack([t + 1, 2 * (t + 1)], axis=1), atol=1e-13)
    np.testing.assert_allclose(cf.dcurve(t, P), np.tile([1.0, 2.0], (37, 1)), atol=1e-13)


def test_jacobian_matches_finite_differences():
    draw = curvefit_problem(npoints=15, Kc=10)
    data, x0 = cf.make_data(draw)
    J = cf.jacobian_dense(x0, data)
    h = 1e-6
    Jfd = np.zeros_like(J)
    for j in range(x0.shape[0]):
        e = np.zeros_like(x0)
        e[j] = h
        Jfd[:, j] = (cf.residual(x0 + e, data) - cf.residual(x0 - e, data)) / (2 * h)
    np.testing.assert_allclose(J, Jfd, atol=1e-7)


def test_nielsen_closed_form():
    assert lm.nielsen(1.0, 2.0, 1.0) == (pytest.approx(1 / 3), 2.0, True)
    assert lm.nielsen(1.0, 8.0, 0.5) == (pytest.approx(1.0), 2.0, True)
    assert lm.nielsen(2.0, 2.0, 0.75) == (pytest.approx(2 * 0.875), 2.0, True)
    assert lm.nielsen(2.0, 4.0, -0.1) == (8.0, 8.0, False)


def test_lm_monotone_and_converges():
    draw = curvefit_problem(npoints=60, Kc=12, sigma=0.0)
    data, x0 = cf.make_data(draw)
    s = lm.lm_run(x0, data, lam0=1e-3, max_iter=60)
    acc = [h[0] for h in s.history if h[3]]
    assert all(a >= b for a, b in zip(acc, acc[1:]))
    # noise-free data: the exact minimiser has zero cost
    assert s.cost < 1e-16
    again = lm.lm_run(x0, data, lam0=1e-3, max_iter=60)
    assert again.cost == s.cost and np.array_equal(again.x, s.x)


def test_lm_system_matches_dense_and_banded():
    draw = curvefit_problem(npoints=40, Kc=10)
    data, x0 = cf.make_data(draw)
    P, f = lm.curvefit_system(x0, data, 1e-2)
    p_band = lm.solve_system(P, banded_reduced=True)
    p_dense = lm.solve_system(P, banded_reduced=False)
    np.testing.assert_allclose(p_band, p_dense, rtol=1e-10, atol=1e-12)
    J = cf.jacobian_dense(x0, data)
    np.testing.assert_allclose(J, st.assemble_J(P), atol=0)


def test_library_nielsen_update_equals_the_oracle():
    """The host entry point qrkit_nielsen_update against the oracle's rule, including the
    clamp at 1/3, rho = 0 (rejected) and a negative rho."""
    from paper_1802_03773_gb300 import build as b
    b.build()
    from paper_1802_03773_gb300 import qrkit
    for lam, nu, rho in [(1.0, 2.0, 1.0), (1.0, 8.0, 0.5), (2.0, 2.0, 0.75), (2.0, 4.0, -0.1), (3e-4, 16.0, 0.0),
                         (5.0, 2.0, 0.999), (1e-8, 2.0, 0.01)]:
        got = qrkit.nielsen_update(rho, lam, nu)
        ref = lm.nielsen(lam, nu, rho)
        assert got[2] == ref[2]
        assert got[0] == pytest.approx(ref[0], rel=1e-15) and got[1] == ref[1]
    with pytest.raises(qrkit.QRKitError):
        qrkit.nielsen_update(0.5, 0.0, 2.0)
