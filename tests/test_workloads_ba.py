"""The BA-shaped workload generator (bundle adjustment, Sec. 6.2) checked on the CPU: the
camera model against hand-worked projections, the Jacobian against the model by a
first-order Taylor test (errors quadratic in the step), and the block-sparse structure of the
camera part."""
import numpy as np

from workloads import ba_project, ba_system


def test_projection_hand_worked():
    # identity rotation, camera 5 units behind the origin along z, f = 1, no distortion:
    # X = (1, 2, 0) -> X_c = (1, 2, -5) -> p = -(1, 2) / (-5) = (0.2, 0.4)
    cam = np.array([0.0, 0.0, 0.0, 0.0, 0.0, -5.0, 1.0, 0.0, 0.0])
    np.testing.assert_allclose(ba_project(cam, np.array([1.0, 2.0, 0.0])), [0.2, 0.4], rtol=1e-15)
    # radial terms: |p|^2 = 0.2, factor 1 + 0.5 * 0.2 + 0.25 * 0.04 = 1.11; focal length 2
    cam2 = cam.copy()
    cam2[6:9] = [2.0, 0.5, 0.25]
    np.testing.assert_allclose(ba_project(cam2, np.array([1.0, 2.0, 0.0])), [2 * 1.11 * 0.2, 2 * 1.11 * 0.4],
                               rtol=1e-14)
    # a quarter turn about z maps x to y: X = (1, 0, 0) -> R X = (0, 1, 0), X_c = (0, 1, -5)
    cam3 = cam.copy()
    cam3[:3] = [0.0, 0.0, np.pi / 2]
    np.testing.assert_allclose(ba_project(cam3, np.array([1.0, 0.0, 0.0])), [0.0, 0.2], atol=1e-15)


def jacobian_times(d, dX, dC):
    """J [dX; dC] from the generator's blocks and camera part (rows in observation order)."""
    rows = []
    for i, blk in enumerate(d["blocks"]):
        rows.append(blk @ dX[i])
    return np.concatenate(rows) + d["S"][:, :dC.size] @ dC.reshape(-1)


def test_jacobian_first_order():
    d = ba_system(P=120, C=6, obs_hi=5, seed_offset=3)
    g = np.random.default_rng(4)
    dX = g.standard_normal(d["X0"].shape)
    dC = g.standard_normal(d["cams0"].shape) * np.array([1e-3] * 3 + [1e-2] * 3 + [1.0, 1e-3, 1e-3])
    r0 = ba_project(d["cams0"][d["cam"]], d["X0"][d["point"]]).reshape(-1)
    errs = []
    for eps in (1e-3, 5e-4):
        r1 = ba_project((d["cams0"] + eps * dC)[d["cam"]], (d["X0"] + eps * dX)[d["point"]]).reshape(-1)
        lin = eps * jacobian_times(d, dX, dC)
        errs.append((np.linalg.norm(r1 - r0 - lin), np.linalg.norm(lin)))
    assert errs[0][0] < 1e-2 * errs[0][1]            # the linear part dominates
    assert 3.5 < errs[0][0] / errs[1][0] < 4.5     # second order: halving the step quarters the rest


def test_structure_and_rhs():
    d = ba_system(P=80, C=6, obs_lo=2, obs_hi=5, s_pad=64, seed_offset=5)
    S, cam, pt = d["S"], d["cam"], d["point"]
    assert S.shape == (2 * cam.size, 64) and d["s"] == 64
    for o in range(cam.size):
        nz = np.nonzero(np.any(S[2 * o:2 * o + 2] != 0.0, axis=0))[0]
        assert set(nz.tolist()) <= set(range(9 * cam[o], 9 * cam[o] + 9))
    assert np.all(S[:, 54:] == 0.0)                 # padding columns
    starts = np.concatenate([[0], np.cumsum(d["n"] // 2)])
    for i in range(d["K"]):
        cs = cam[starts[i]:starts[i + 1]]
        assert np.all(np.diff(cs) > 0) and 2 <= cs.size <= 5
        assert np.all(pt[starts[i]:starts[i + 1]] == i)
        assert d["blocks"][i].shape == (2 * cs.size, 3)
    r = ba_project(d["cams0"][cam], d["X0"][pt]) - d["obs"]
    np.testing.assert_allclose(d["b"], -r.reshape(-1), rtol=0, atol=0)
