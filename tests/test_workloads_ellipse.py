"""The ellipse-fit system (the surface fitting benchmark of Sec. 6, composed as in Sec. 4.2):
its Jacobian is the derivative of its residual, and the oracle's damped step from it lowers
the fitting cost.  CPU only."""
import numpy as np

from oracle import structured as st
from workloads import ellipse_system


def residual(t, x, y):
    """r_i = E(t_i) - y_i for the ellipse E(t) = c + Rot(phi) (a cos t, b sin t)."""
    rot = np.array([[np.cos(x[4]), -np.sin(x[4])], [np.sin(x[4]), np.cos(x[4])]])
    e = np.stack([x[2] * np.cos(t), x[3] * np.sin(t)], axis=0)
    return (x[:2, None] + rot @ e).T - y


def test_jacobian_matches_central_differences():
    d = ellipse_system(N=300)
    t0, x0, y = d["t0"], d["x0"], d["y"]
    r0 = residual(t0, x0, y)
    np.testing.assert_allclose(d["b"], -r0.reshape(-1), rtol=0, atol=1e-14)
    h = 1e-6
    # latent column of every block at once (each point's residual depends on its own t only)
    dr = (residual(t0 + h, x0, y) - residual(t0 - h, x0, y)) / (2 * h)
    np.testing.assert_allclose(d["blocks"][:, :, 0], dr, rtol=1e-7, atol=1e-8)
    S = d["S"].reshape(-1, 2, 5)
    for k in range(5):
        e = np.zeros(5)
        e[k] = h
        dr = (residual(t0, x0 + e, y) - residual(t0, x0 - e, y)) / (2 * h)
        np.testing.assert_allclose(S[:, :, k], dr, rtol=1e-7, atol=1e-8)


def test_float32_is_the_rounded_float64_system():
    d64 = ellipse_system(N=50)
    d32 = ellipse_system(N=50, dtype=np.float32)
    for key in ("blocks", "S", "b"):
        assert d32[key].dtype == np.float32
        np.testing.assert_array_equal(d32[key], d64[key].astype(np.float32))


def test_oracle_step_lowers_the_cost():
    d = ellipse_system(N=400)
    K = d["K"]
    P = st.BlockProblem(blocks=[d["blocks"][i] for i in range(K)],
                        coupled=[d["S"][2 * i:2 * i + 2] for i in range(K)], s=5, b=d["b"],
                        lam=d["lam"])
    p, _ = st.factor_and_solve(P)
    t1, x1 = d["t0"] + p[:K], d["x0"] + p[K:]
    c0 = 0.5 * np.sum(residual(d["t0"], d["x0"], d["y"]) ** 2)
    c1 = 0.5 * np.sum(residual(t1, x1, d["y"]) ** 2)
    assert c1 < 0.5 * c0
