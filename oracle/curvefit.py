"""Curve-fit model for the LM workloads: points on an open uniform cubic B-spline.

Test infrastructure only.  A simplification of the surface-fitting problems of Sec. 6.2
(ellipse fitting there; a closed B-spline-like curve here): each data point has one
latent curve parameter t_i and the control points are shared, so the Jacobian is
block-angular, [blkdiag(2x1 blocks) | S] (Sec. 4.2, Fig. 5a's shape).

Model (reading: the paper gives no curve-fit generator; this one is ours):
  x = (t_1 .. t_P, P_0x, P_0y, P_1x, P_1y, ...)       (control points interleaved)
  seg(t) = clip(floor(t), 0, Kc - 4),  u = t - seg    (end segments extrapolate)
  curve(t) = sum_{k=0..3} B_k(u) P_{seg + k}
  B_0 = (1-u)^3/6, B_1 = (3u^3 - 6u^2 + 4)/6, B_2 = (-3u^3 + 3u^2 + 3u + 1)/6, B_3 = u^3/6
  residual f_i = curve(t_i) - data_i  (2 rows per point; cost = 1/2 ||f||^2)
  J block i (2x1) = curve'(t_i);  S rows of point i: window of 8 shared columns
  starting at 2 seg(t_i): x-row = (B_0,0,B_1,0,B_2,0,B_3,0), y-row = (0,B_0,0,B_1,...).

Pins (tests/test_oracle_lm.py): the B-spline basis is a partition of unity, reproduces
a straight line from collinear control points, and J matches central finite differences
of f.
"""
from __future__ import annotations

import numpy as np


def basis(u):
    u = np.asarray(u, dtype=np.float64)
    v = 1.0 - u
    return np.stack([v ** 3 / 6.0,
                     (3.0 * u ** 3 - 6.0 * u ** 2 + 4.0) / 6.0,
                     (-3.0 * u ** 3 + 3.0 * u ** 2 + 3.0 * u + 1.0) / 6.0,
                     u ** 3 / 6.0], axis=-1)


def dbasis(u):
    u = np.asarray(u, dtype=np.float64)
    v = 1.0 - u
    return np.stack([-0.5 * v ** 2,
                     (9.0 * u ** 2 - 12.0 * u) / 6.0,
                     (-9.0 * u ** 2 + 6.0 * u + 3.0) / 6.0,
                     0.5 * u ** 2], axis=-1)


def segment(t, Kc):
    t = np.asarray(t, dtype=np.float64)
    seg = np.clip(np.floor(t), 0, Kc - 4).astype(np.int64)
    return seg, t - seg


def curve(t, P):
    P = np.asarray(P, dtype=np.float64)
    seg, u = segment(t, P.shape[0])
    B = basis(u)
    idx = seg[:, None] + np.arange(4)[None, :]
    return np.einsum("ik,ikd->id", B, P[idx])


def dcurve(t, P):
    P = np.asarray(P, dtype=np.float64)
    seg, u = segment(t, P.shape[0])
    dB = dbasis(u)
    idx = seg[:, None] + np.arange(4)[None, :]
    return np.einsum("ik,ikd->id", dB, P[idx])


def make_data(draw):
    """Data points and start point from a workloads.curvefit_problem draw."""
    data = curve(draw["t_true"], draw["P_true"]) + draw["noise"]
    t0 = draw["t_true"] + draw["dt"]
    P0 = draw["P_true"] + draw["dP"]
    return data, pack(t0, P0)


def pack(t, P):
    return np.concatenate([np.asarray(t, dtype=np.float64), np.asarray(P, dtype=np.float64).reshape(-1)])


def unpack(x, npoints):
    return x[:npoints], x[npoints:].reshape(-1, 2)


def residual(x, data):
    t, P = unpack(x, data.shape[0])
    return (curve(t, P) - data).reshape(-1)


def jacobian_parts(x, data):
    """(blocks (P, 2, 1), coupled (P, 2, 8), start (P,)) of J at x."""
    npts = data.shape[0]
    t, P = unpack(x, npts)
    seg, u = segment(t, P.shape[0])
    B = basis(u)
    blocks = dcurve(t, P)[:, :, None]
    coupled = np.zeros((npts, 2, 8))
    coupled[:, 0, 0::2] = B
    coupled[:, 1, 1::2] = B
    return blocks, coupled, 2 * seg


def jacobian_dense(x, data):
    """Dense J (small problems), columns ordered (t..., control points interleaved)."""
    npts = data.shape[0]
    t, P = unpack(x, npts)
    Kc = P.shape[0]
    blocks, coupled, start = jacobian_parts(x, data)
    J = np.zeros((2 * npts, npts + 2 * Kc))
    for i in range(npts):
        J[2 * i:2 * i + 2, i] = blocks[i, :, 0]
        J[2 * i:2 * i + 2, npts + start[i]:npts + start[i] + 8] = coupled[i]
    return J
