"""Learned damping for the device LM: data collection, training and policy runs.

Orchestration only: every LM step, feature, forward/backward pass and Adam update runs in
the library's kernels (qrkit_lm_step, qrkit_lm_features, qrkit_mlp_train_step); this module
lays out batches, moves state between calls and picks labels.

Training data come from trajectories of the plain solver (Nielsen's rule), optionally
followed by rounds on the trajectories of the trained policy itself (DAgger).  After every
accepted step of a trajectory the features of the step history are recorded together with
a label: the same state is continued for a few steps, the first with lambda times each
multiplier of the policy's grid and the rest with Nielsen's rule (all multipliers and
problems in one batched LM call per step), and the label is the multiplier whose rollout
reaches the lowest cost (the largest multiplier when no rollout step is accepted).
"""
from __future__ import annotations

import numpy as np

from .qrkit import MLP_FEATURES, MLP_MULTIPLIERS, Context


class Batch:
    """Several curve-fit problems in the library's layout: x = [all t | all control points]."""

    def __init__(self, problems):
        """problems: list of (data (P, 2) float64, x0 (P + 2 Kc,) float64) host arrays."""
        self.npts = [int(d.shape[0]) for d, _ in problems]
        self.kcs = [int((x0.shape[0] - d.shape[0]) // 2) for d, x0 in problems]
        ts = [x0[:n] for (_, x0), n in zip(problems, self.npts)]
        cs = [x0[n:] for (_, x0), n in zip(problems, self.npts)]
        self.x0 = np.concatenate(ts + cs).astype(np.float64)
        self.data = np.concatenate([d for d, _ in problems]).astype(np.float64)
        self.NP = sum(self.npts)
        self.p0 = np.concatenate([[0], np.cumsum(self.npts)]).astype(np.int64)
        self.c0 = np.concatenate([[0], np.cumsum([2 * k for k in self.kcs])]).astype(np.int64)

    @property
    def B(self):
        return len(self.npts)

    def split(self, x):
        """Per-problem x vectors (t then control points) from a packed host array."""
        return [np.concatenate([x[self.p0[k]:self.p0[k + 1]], x[self.NP + self.c0[k]:self.NP + self.c0[k + 1]]])
                for k in range(self.B)]

    def replica_index(self, reps):
        """Index into x of `reps` copies of every problem (copy-major) in the packed layout."""
        t = [np.arange(self.p0[k], self.p0[k + 1]) for _ in range(reps) for k in range(self.B)]
        c = [self.NP + np.arange(self.c0[k], self.c0[k + 1]) for _ in range(reps) for k in range(self.B)]
        return np.concatenate(t + c).astype(np.int64)


def _states_to_arrays(states):
    return dict(lam=np.array([s.lambda_ for s in states]), cost=np.array([s.cost for s in states]),
                cost_new=np.array([s.cost_new for s in states]), acc=np.array([s.accepted for s in states]),
                it=np.array([s.iteration for s in states]))


def collect(batch: Batch, iters=25, lam0=1e-3, precision="fp32_refined", refine_steps=1, horizon=1,
            policy_params=None, device=0):
    """(features float32 (n, 16), labels int32 (n,)) from LM trajectories of the batch.

    The trajectories follow Nielsen's rule, or the MLP policy `policy_params` (to label the
    states a trained policy visits, DAgger-style).  horizon: steps of each lookahead rollout
    (the first with lambda times the multiplier, the rest with Nielsen's rule); the label is
    the multiplier with the lowest cost reached."""
    import torch
    R = len(MLP_MULTIPLIERS)
    stream = torch.cuda.Stream(device)
    plain = Context(device, stream=stream, precision=precision)
    look = Context(device, stream=stream, precision=precision)
    dev = plain.device
    with torch.cuda.stream(stream):
        data = torch.from_numpy(batch.data).to(dev)
        x = torch.from_numpy(batch.x0).to(dev)
        rep = torch.from_numpy(batch.replica_index(R)).to(dev)
        data_rep = torch.from_numpy(np.concatenate([batch.data] * R)).to(dev)
        x_rep = torch.empty(rep.shape[0], dtype=torch.float64, device=dev)
        feats = torch.empty((batch.B, MLP_FEATURES), dtype=torch.float32, device=dev)
    plain.lm_plan(batch.npts, batch.kcs, data)
    look.lm_plan(batch.npts * R, batch.kcs * R, data_rep)
    if policy_params is not None:
        plain.mlp_init(policy_params)
        plain.lm_set_policy(True)
    st = plain.lm_states(lam0)
    Xs, ys = [], []
    for _ in range(iters):
        lam_used = np.array([s.lambda_ for s in st])
        done_before = np.array([s.done for s in st])
        plain.lm_step(x, st, refine_steps=refine_steps)
        a = _states_to_arrays(st)
        take = (a["acc"] == 1) & (done_before == 0)
        if not take.any():
            continue
        plain.lm_features(feats)
        with torch.cuda.stream(stream):
            torch.index_select(x, 0, rep, out=x_rep)
        lst = look.lm_states([lam_used[k] * m for m in MLP_MULTIPLIERS for k in range(batch.B)])
        reached = np.full(R * batch.B, np.inf)
        for _ in range(horizon):
            look.lm_step(x_rep, lst, refine_steps=refine_steps)
            la = _states_to_arrays(lst)
            reached = np.minimum(reached, np.where(la["acc"] == 1, la["cost_new"], np.inf))
        score = reached.reshape(R, batch.B)
        ok = np.isfinite(score)
        lab = np.where(ok.any(axis=0), np.argmin(score, axis=0), R - 1)
        stream.synchronize()
        f = feats.cpu().numpy()
        Xs.append(f[take])
        ys.append(lab[take])
    plain.close()
    look.close()
    X = np.concatenate(Xs).astype(np.float32) if Xs else np.zeros((0, MLP_FEATURES), np.float32)
    y = np.concatenate(ys).astype(np.int32) if ys else np.zeros(0, np.int32)
    return X, y


def train(X, y, init_params, steps=400, lr=3e-3, batch=256, seed=0, device=0):
    """Adam on the softmax cross-entropy; returns (params float32, loss history)."""
    import torch
    ctx = Context(device, precision="fp32")
    ctx.mlp_init(init_params)
    dev = ctx.device
    tX = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(dev)
    ty = torch.from_numpy(np.ascontiguousarray(y, dtype=np.int32)).to(dev)
    rng = np.random.default_rng(seed)
    n = X.shape[0]
    losses = []
    for _ in range(steps):
        if n > batch:
            idx = torch.from_numpy(rng.choice(n, size=batch, replace=False)).to(dev)
            bx, by = tX.index_select(0, idx).contiguous(), ty.index_select(0, idx).contiguous()
        else:
            bx, by = tX, ty
        losses.append(ctx.mlp_train_step(bx, by, lr))
    params = ctx.mlp_params()
    ctx.close()
    return params, losses


def train_policy(batch: Batch, init_params, horizon=6, dagger_rounds=2, iters=60, steps=800, lr=3e-3,
                 precision="fp32_refined", device=0):
    """Labels from Nielsen trajectories, then `dagger_rounds` rounds that add the states the
    current policy visits (labels by the same rollouts); retrains from init_params each round.
    Returns (params, number of samples, final loss)."""
    X, y = collect(batch, iters=iters, horizon=horizon, precision=precision, device=device)
    params, losses = train(X, y, init_params, steps=steps, lr=lr, device=device)
    for _ in range(dagger_rounds):
        X2, y2 = collect(batch, iters=iters, horizon=horizon, precision=precision, policy_params=params,
                         device=device)
        X, y = np.concatenate([X, X2]), np.concatenate([y, y2])
        params, losses = train(X, y, init_params, steps=steps, lr=lr, device=device)
    return params, X.shape[0], losses[-1]


def run(batch: Batch, iters=60, lam0=1e-3, params=None, precision="fp32_refined", refine_steps=1, device=0,
        x0=None, with_times=False):
    """LM with Nielsen's rule (params None) or the MLP policy, from batch.x0 (or the packed x0
    given); returns (best cost so far per iteration (iters, B), final x per problem) and, with
    with_times, the wall-clock milliseconds from the start to the end of every iteration
    (each iteration returns its states to the host, so the clock reads completed work)."""
    import time

    import torch
    stream = torch.cuda.Stream(device)
    ctx = Context(device, stream=stream, precision=precision)
    dev = ctx.device
    with torch.cuda.stream(stream):
        data = torch.from_numpy(batch.data).to(dev)
        x = torch.from_numpy(batch.x0 if x0 is None else np.asarray(x0, np.float64)).to(dev)
    ctx.lm_plan(batch.npts, batch.kcs, data)
    if params is not None:
        ctx.mlp_init(params)
        ctx.lm_set_policy(True)
    st = ctx.lm_states(lam0)
    best = np.full(batch.B, np.inf)
    hist, times = [], []
    stream.synchronize()
    t0 = time.perf_counter()
    for _ in range(iters):
        ctx.lm_step(x, st, refine_steps=refine_steps)
        a = _states_to_arrays(st)
        times.append(1000.0 * (time.perf_counter() - t0))
        now = np.where(a["acc"] == 1, a["cost_new"], a["cost"])
        best = np.minimum(best, now)
        hist.append(best.copy())
    stream.synchronize()
    xp = x.cpu().numpy()
    xs = batch.split(xp)
    ctx.close()
    if with_times:
        return np.array(hist), xs, np.array(times), xp
    return np.array(hist), xs


def iterations_to(hist, target):
    """First iteration (1-based) whose best cost is within target per problem (inf if never)."""
    hit = hist <= target[None, :]
    first = np.where(hit.any(axis=0), hit.argmax(axis=0) + 1, np.inf)
    return first
