"""Generators for the synthetic workloads (no arithmetic of the method here).

Workloads (shapes follow the paper's problem classes: block-angular Jacobians of
latent-variable fits, Sec. 4.2 / Sec. 6.2, and banded matrices, Sec. 4.4):

  block_angular_dense  J = [blkdiag(J_1..J_K) | S]: K blocks n x m, S dense (K n) x s,
                       N(0,1) entries, global column j scaled by 10^(3 j / (N-1)),
                       b ~ N(0,1).  Default K=200, n=4, m=2, s=30.
  batched_blocks       K independent blocks, n ~ U{2..16}, m ~ U{1..min(n,6)}, N(0,1),
                       one rhs per block; packed column-major per block.
  curvefit_problem     points on an open uniform cubic B-spline with Kc control
                       points plus N(0, sigma^2) noise, and a perturbed start.
  banded_problem       J of (rows_per_col * n) x n, row i touches columns
                       floor(i / rows_per_col) .. + w - 1 (truncated at n - 1), N(0,1).
  mlp_init             initial weights of the damping-policy MLP (He-normal, zero biases).
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 20180209


def rng_for(workload: int, seed_offset: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(SEED_BASE + workload + 1000003 * seed_offset))


def _f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def block_angular_dense(K=200, n=4, m=2, s=30, seed_offset=0, scale_decades=3.0,
                        dtype=np.float64):
    """Block-angular J = [blkdiag(J_i) | S] with geometric column scaling.

    Returns dict(blocks (K, n, m), S (K n, s), b (K n), lam).  Global column order is
    block columns first (block i owns columns i m .. i m + m - 1), then the s shared columns.
    """
    g = rng_for(1, seed_offset)
    N = K * m + s
    scale = 10.0 ** (scale_decades * np.arange(N) / max(N - 1, 1))
    blocks = g.standard_normal((K, n, m))
    S = g.standard_normal((K * n, s))
    b = g.standard_normal(K * n)
    blocks = blocks * scale[:K * m].reshape(K, 1, m)
    S = S * scale[K * m:][None, :]
    if dtype == np.float32:
        blocks, S, b = _f32(blocks), _f32(S), _f32(b)
    return dict(blocks=blocks, S=S, b=b, lam=1e-2, K=K, n=n, m=m, s=s)


def batched_blocks(K=1_000_000, n_lo=2, n_hi=16, m_hi=6, seed_offset=0, dtype=np.float32):
    """K independent blocks, n ~ U{n_lo..n_hi}, m ~ U{1..min(n, m_hi)}, N(0,1) entries.

    Returns dict(n (uint8 K), m (uint8 K), vals (packed column-major per block),
    b (packed per block), val_off (int64 K+1), row_off (int64 K+1), col_off (int64 K+1)).
    """
    g = rng_for(2, seed_offset)
    n = g.integers(n_lo, n_hi + 1, size=K)
    m = (g.random(K) * np.minimum(n, m_hi)).astype(np.int64) + 1
    m = np.minimum(m, np.minimum(n, m_hi))
    nm = n * m
    val_off = np.concatenate([[0], np.cumsum(nm)]).astype(np.int64)
    row_off = np.concatenate([[0], np.cumsum(n)]).astype(np.int64)
    col_off = np.concatenate([[0], np.cumsum(m)]).astype(np.int64)
    vals = g.standard_normal(int(val_off[-1]))
    b = g.standard_normal(int(row_off[-1]))
    if dtype == np.float32:
        vals, b = _f32(vals), _f32(b)
    return dict(n=n.astype(np.uint8), m=m.astype(np.uint8), vals=vals, b=b,
                val_off=val_off, row_off=row_off, col_off=col_off, K=K)


def curvefit_problem(npoints=200_000, Kc=2048, sigma=0.01, start_sigma_t=0.05,
                     start_sigma_p=0.01, radius_jitter=0.1, seed_offset=0, workload=3):
    """Data for fitting an open uniform cubic B-spline (Kc control points) to 2-D points.

    Control points P_k = (cos th_k, sin th_k) (1 + radius_jitter N(0,1)), th_k = 2 pi k / Kc.
    Parameters t_i ~ U[0, Kc - 3).  The curve itself is evaluated by the model code of
    each side; this returns only the random draws: control points, t_true, the noise to
    add to curve(t_true), and the start perturbations.
    """
    g = rng_for(workload, seed_offset)
    th = 2.0 * np.pi * np.arange(Kc) / Kc
    rad = 1.0 + radius_jitter * g.standard_normal(Kc)
    P_true = np.stack([np.cos(th) * rad, np.sin(th) * rad], axis=1)
    t_true = g.random(npoints) * (Kc - 3)
    noise = sigma * g.standard_normal((npoints, 2))
    dt = start_sigma_t * g.standard_normal(npoints)
    dP = start_sigma_p * g.standard_normal((Kc, 2))
    return dict(P_true=P_true, t_true=t_true, noise=noise, dt=dt, dP=dP, Kc=Kc,
                npoints=npoints)


def ellipse_system(N=500_000, sigma=0.01, start_sigma_t=0.05, start_sigma_p=0.02, lam=1e-3,
                   seed_offset=0, dtype=np.float64, workload=6):
    """The linear system of one LM step of fitting an ellipse to N 2-D points (the surface
    fitting benchmark of Sec. 6: one latent angle per point, five shared ellipse parameters,
    J a horizontal concatenation of a block diagonal and a dense part, Sec. 4.2).

    Ellipse E(t) = c + Rot(phi) (a cos t, b sin t) with c ~ N(0, 0.5^2 I), a ~ U[1.5, 2.5),
    b = a U[0.3, 0.8), phi ~ U[0, pi); points y_i = E(t_i) + N(0, sigma^2 I), t_i ~ U[0, 2 pi).
    The system is taken at a perturbed start (t_i + N(0, start_sigma_t^2), every parameter
    + N(0, start_sigma_p^2)): residual r_i = E(t_i) - y_i (2 rows per point), block i = dr_i/dt_i
    (2 x 1), S rows 2i, 2i + 1 = dr_i/d(c_x, c_y, a, b, phi) (2 x 5), right-hand side -r.  The
    ellipse model is evaluated here, once, to lay out the input; neither side of the solve
    evaluates it.  Returns dict(blocks (N, 2, 1), S (2N, 5), b (2N), lam, K, n, m, s, and the
    start t0 (N), x0 (5) and points y (N, 2) the system was taken at).
    """
    g = rng_for(workload, seed_offset)
    c = 0.5 * g.standard_normal(2)
    a = 1.5 + g.random()
    bb = a * (0.3 + 0.5 * g.random())
    phi = np.pi * g.random()
    t = 2.0 * np.pi * g.random(N)
    noise = sigma * g.standard_normal((N, 2))
    t0 = t + start_sigma_t * g.standard_normal(N)
    x0 = np.array([c[0], c[1], a, bb, phi]) + start_sigma_p * g.standard_normal(5)

    def curve(tt, x):
        cs, sn = np.cos(x[4]), np.sin(x[4])
        u, v = x[2] * np.cos(tt), x[3] * np.sin(tt)
        return np.stack([x[0] + cs * u - sn * v, x[1] + sn * u + cs * v], axis=1)

    y = curve(t, np.array([c[0], c[1], a, bb, phi])) + noise
    r = curve(t0, x0) - y
    cs, sn = np.cos(x0[4]), np.sin(x0[4])
    ct, st = np.cos(t0), np.sin(t0)
    u, v = x0[2] * ct, x0[3] * st
    du, dv = -x0[2] * st, x0[3] * ct
    blocks = np.stack([cs * du - sn * dv, sn * du + cs * dv], axis=1).reshape(N, 2, 1)
    S = np.zeros((N, 2, 5))
    S[:, 0, 0] = 1.0
    S[:, 1, 1] = 1.0
    S[:, 0, 2], S[:, 1, 2] = cs * ct, sn * ct
    S[:, 0, 3], S[:, 1, 3] = -sn * st, cs * st
    S[:, 0, 4], S[:, 1, 4] = -sn * u - cs * v, cs * u - sn * v
    S = S.reshape(2 * N, 5)
    b = -r.reshape(2 * N)
    if dtype == np.float32:
        blocks, S, b = _f32(blocks), _f32(S), _f32(b)
    return dict(blocks=blocks, S=S, b=b, lam=lam, K=N, n=2, m=1, s=5, t0=t0, x0=x0, y=y)


def _rodrigues(w):
    """Rotation matrices of angle-axis vectors w (..., 3)."""
    th = np.linalg.norm(w, axis=-1)[..., None, None]
    k = w / np.maximum(np.linalg.norm(w, axis=-1, keepdims=True), 1e-300)
    K = np.zeros(w.shape[:-1] + (3, 3))
    K[..., 0, 1], K[..., 0, 2] = -k[..., 2], k[..., 1]
    K[..., 1, 0], K[..., 1, 2] = k[..., 2], -k[..., 0]
    K[..., 2, 0], K[..., 2, 1] = -k[..., 1], k[..., 0]
    I = np.broadcast_to(np.eye(3), K.shape)
    return I + np.sin(th) * K + (1.0 - np.cos(th)) * (K @ K)


def ba_project(cam, X):
    """Projection of points X (..., 3) by cameras cam (..., 9) = [angle-axis (3), translation
    (3), focal length, radial k1, k2]: X_c = R X + t, p = -X_c[:2] / X_c[2],
    u = f (1 + k1 |p|^2 + k2 |p|^4) p (the camera model of the public bundle-adjustment
    problem sets)."""
    R = _rodrigues(cam[..., :3])
    Xc = np.einsum("...ij,...j->...i", R, X) + cam[..., 3:6]
    pxy = -Xc[..., :2] / Xc[..., 2:3]
    r2 = np.sum(pxy * pxy, axis=-1, keepdims=True)
    return cam[..., 6:7] * (1.0 + cam[..., 7:8] * r2 + cam[..., 8:9] * r2 * r2) * pxy


def ba_system(P=2000, C=7, obs_lo=2, obs_hi=6, s_pad=None, sigma=0.5, lam=1e-3, seed_offset=0,
              dtype=np.float64, workload=7):
    """The linear system of one LM step of a bundle adjustment (the BA experiments of Sec. 6.2:
    3 unknowns per point, 9 per camera; an observation gives two rows that touch its point and
    one camera): J = [blkdiag(point blocks) | camera part] (Sec. 4.2), the camera part block-
    sparse and stored dense with s = 9 C shared columns (zero-padded to s_pad when given).

    Scene: points uniform in the unit ball; C cameras on a circle of radius 4 around the y
    axis, looking at the origin; f ~ U[500, 800), k1 ~ N(0, 0.05^2), k2 ~ N(0, 0.01^2).  Each
    point is observed by k ~ U{obs_lo..obs_hi} distinct cameras (its rows in camera order);
    observations = projections + N(0, sigma^2) pixels.  The system is taken at a start with
    points + N(0, 0.01^2), angle-axis + N(0, 0.001^2), translations + N(0, 0.01^2),
    f (1 + N(0, 0.005^2)), k1, k2 + N(0, 0.001^2): rows r = projection - observation, J by
    central differences of ba_project (steps 1e-6 relative), right-hand side -r.  The camera
    model is evaluated here to lay out the input; neither side of the solve evaluates it.
    Returns dict(blocks (list of (2 k_i, 3)), n (K), m = 3, S (rows, s), b, lam, K = P, s,
    cam (rows / 2: camera of each observation), point (rows / 2), X0, cams0, obs).
    """
    if not (1 <= obs_lo <= obs_hi <= C):
        raise ValueError("need 1 <= obs_lo <= obs_hi <= C")
    g = rng_for(workload, seed_offset)
    X = g.standard_normal((P, 3))
    X *= (g.random(P) ** (1.0 / 3.0) / np.linalg.norm(X, axis=1))[:, None]
    th = 2.0 * np.pi * (np.arange(C) + 0.5 * g.random(C)) / C
    centers = 4.0 * np.stack([np.sin(th), 0.2 * g.standard_normal(C), np.cos(th)], axis=1)
    cams = np.zeros((C, 9))
    for c in range(C):
        z = centers[c] / np.linalg.norm(centers[c])      # camera z axis in world (looks along -z)
        x = np.cross([0.0, 1.0, 0.0], z)
        x /= np.linalg.norm(x)
        y = np.cross(z, x)
        R = np.stack([x, y, z])
        ang = np.arccos(np.clip((np.trace(R) - 1.0) / 2.0, -1.0, 1.0))
        axis = np.array([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]])
        nrm = np.linalg.norm(axis)
        cams[c, :3] = ang * axis / nrm if nrm > 1e-12 else 0.0
        cams[c, 3:6] = -R @ centers[c]
    cams[:, 6] = 500.0 + 300.0 * g.random(C)
    cams[:, 7] = 0.05 * g.standard_normal(C)
    cams[:, 8] = 0.01 * g.standard_normal(C)
    k = g.integers(obs_lo, obs_hi + 1, size=P)
    cam_of = np.concatenate([np.sort(g.choice(C, size=int(ki), replace=False)) for ki in k])
    pt_of = np.repeat(np.arange(P), k)
    obs = ba_project(cams[cam_of], X[pt_of]) + sigma * g.standard_normal((pt_of.size, 2))
    X0 = X + 0.01 * g.standard_normal(X.shape)
    cams0 = cams.copy()
    cams0[:, :3] += 0.001 * g.standard_normal((C, 3))
    cams0[:, 3:6] += 0.01 * g.standard_normal((C, 3))
    cams0[:, 6] *= 1.0 + 0.005 * g.standard_normal(C)
    cams0[:, 7:9] += 0.001 * g.standard_normal((C, 2))
    r = ba_project(cams0[cam_of], X0[pt_of]) - obs                 # (nobs, 2)
    nobs = pt_of.size
    Jp = np.zeros((nobs, 2, 3))
    Jc = np.zeros((nobs, 2, 9))
    for j in range(3):
        h = 1e-6 * max(1.0, float(np.max(np.abs(X0[:, j]))))
        d = np.zeros(3)
        d[j] = h
        Jp[:, :, j] = (ba_project(cams0[cam_of], X0[pt_of] + d) - ba_project(cams0[cam_of], X0[pt_of] - d)) / (2 * h)
    for j in range(9):
        h = 1e-6 * max(1.0, float(np.max(np.abs(cams0[:, j]))))
        d = np.zeros(9)
        d[j] = h
        Jc[:, :, j] = (ba_project(cams0[cam_of] + d, X0[pt_of]) - ba_project(cams0[cam_of] - d, X0[pt_of])) / (2 * h)
    s = 9 * C if s_pad is None else int(s_pad)
    if s < 9 * C:
        raise ValueError("s_pad below 9 C")
    rows = 2 * nobs
    S = np.zeros((nobs, 2, s))
    cols = 9 * cam_of[:, None] + np.arange(9)[None, :]
    S[np.arange(nobs)[:, None, None], np.arange(2)[None, :, None], cols[:, None, :]] = Jc
    S = S.reshape(rows, s)
    starts = np.concatenate([[0], np.cumsum(k)])
    blocks = [Jp[starts[i]:starts[i + 1]].reshape(-1, 3) for i in range(P)]
    b = -r.reshape(rows)
    if dtype == np.float32:
        blocks, S, b = [_f32(x) for x in blocks], _f32(S), _f32(b)
    return dict(blocks=blocks, n=(2 * k).astype(np.int64), m=3, S=S, b=b, lam=lam, K=P, s=s,
                cam=cam_of, point=pt_of, X0=X0, cams0=cams0, obs=obs)


def banded_problem(n=1_000_000, rows_per_col=4, w=8, seed_offset=0, dtype=np.float32,
                   workload=4):
    """Banded J: row i starts at column floor(i / rows_per_col), w values, N(0,1).

    Entries that would fall at columns >= n are zero (truncated band end).
    Returns dict(start int64 (M,), vals (M, w), b (M,), n, lam).
    """
    g = rng_for(workload, seed_offset)
    M = rows_per_col * n
    start = (np.arange(M, dtype=np.int64) // rows_per_col)
    vals = g.standard_normal((M, w))
    cols = start[:, None] + np.arange(w)[None, :]
    vals[cols >= n] = 0.0
    b = g.standard_normal(M)
    if dtype == np.float32:
        vals, b = _f32(vals), _f32(b)
    return dict(start=start, vals=vals, b=b, n=n, lam=1e-3, w=w, rows_per_col=rows_per_col)


def banded_batch_shapes(count=4096, n_lo=1000, n_hi=100_000, seed_offset=0):
    """Column counts of a batch of independent banded instances, n ~ U{n_lo..n_hi}."""
    g = rng_for(5, seed_offset)
    return g.integers(n_lo, n_hi + 1, size=count).astype(np.int64)


def mlp_init(seed_offset=0, F=16, H=64, C=8):
    """Initial parameters of the damping-policy MLP (flat float32 vector, He-normal weights,
    zero biases), [W1 (H x F) | b1 | W2 (H x H) | b2 | W3 (C x H) | b3]."""
    g = rng_for(6, seed_offset)
    W1 = g.standard_normal((H, F)) * np.sqrt(2.0 / F)
    W2 = g.standard_normal((H, H)) * np.sqrt(2.0 / H)
    W3 = g.standard_normal((C, H)) * np.sqrt(1.0 / H)
    parts = [W1.reshape(-1), np.zeros(H), W2.reshape(-1), np.zeros(H), W3.reshape(-1), np.zeros(C)]
    return np.concatenate(parts).astype(np.float32)
