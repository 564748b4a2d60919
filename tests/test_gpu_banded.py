"""GPU parity of the batched block-banded QR solve (Sec. 4.4, damping rows per Sec. 4.5 / 5.2)."""
import numpy as np
import pytest

from oracle import banded as bd
from oracle import householder as hh
from tests.gpu_common import assert_close, cuda_or_skip
from workloads import banded_problem

pytestmark = pytest.mark.gpu


def batch(cols, rpc, w, dtype, seed=0):
    """Concatenated instances (same generator, one seed offset per instance)."""
    inst = [banded_problem(n=int(n), rows_per_col=rpc, w=w, seed_offset=seed + k, dtype=dtype)
            for k, n in enumerate(cols)]
    vals = np.concatenate([d["vals"] for d in inst])
    b = np.concatenate([d["b"] for d in inst])
    return inst, vals, b


SOLVER = {"sweep": 1, "parallel": 2}


def run(cols, rpc, w, precision, lam, refine_steps=1, D=None, seed=0, solver="sweep"):
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context
    dtype = np.float64 if precision == "fp64" else np.float32
    inst, vals, b = batch(cols, rpc, w, dtype, seed)
    ctx = Context(0, precision=precision)
    ctx.plan_banded(cols, rows_per_col=rpc, window=w, solver=SOLVER[solver])
    tJ = torch.from_numpy(np.ascontiguousarray(vals.reshape(-1))).cuda()
    tb = torch.from_numpy(b).cuda()
    tD = None if D is None else torch.from_numpy(D.astype(dtype)).cuda()
    N = int(np.sum(cols))
    p = torch.empty(N, device="cuda", dtype=ctx.dtype)
    ctx.factor_solve(tJ, tb, p, None, D=tD, lam=lam, refine_steps=refine_steps)
    ctx.sync_status()
    Rw = torch.empty(N * w, device="cuda", dtype=ctx.dtype) if solver == "sweep" else None
    res2 = np.zeros(len(cols))
    ctx.get_band_factor(Rw, None, res2)
    out = dict(p=p.cpu().numpy().astype(np.float64), res2=res2, inst=inst,
               Rw=None if Rw is None else Rw.cpu().numpy().astype(np.float64).reshape(N, w))
    ctx.close()
    return out


def oracle_solutions(inst, lam, D=None):
    xs, Rs, r2 = [], [], []
    off = 0
    for d in inst:
        n = d["n"]
        Dn = None if D is None else D[off:off + n]
        x, Rw, c, res_sq, _ = bd.damped_solve(d["start"], d["vals"], d["b"], n, lam, Dn)
        xs.append(x)
        Rs.append(Rw)
        r2.append(res_sq)
        off += n
    return np.concatenate(xs), np.vstack(Rs), np.array(r2)


@pytest.mark.parametrize("cols,rpc,w", [([1, 7, 8, 9, 50, 333], 4, 8), ([40, 3, 17], 2, 3),
                                        ([100], 4, 16), ([64] * 9, 1, 5)])
def test_banded_fp64_matches_oracle(cols, rpc, w):
    out = run(cols, rpc, w, "fp64", lam=1e-3)
    x, Rw, r2 = oracle_solutions(out["inst"], 1e-3)
    np.testing.assert_allclose(out["p"], x, rtol=1e-12, atol=1e-12 * np.abs(x).max())
    # R up to row signs, window by window
    s = np.sign(out["Rw"][:, :1]) * np.sign(Rw[:, :1])
    np.testing.assert_allclose(out["Rw"] * s, Rw, atol=1e-11 * np.abs(Rw).max())
    np.testing.assert_allclose(out["res2"], r2, rtol=1e-9)


@pytest.mark.parametrize("cols,rpc,w", [([1, 7, 8, 9, 50, 333], 4, 8), ([40, 3, 17], 2, 3),
                                        ([64] * 9, 1, 5), ([1000], 4, 8)])
def test_banded_parallel_fp64_matches_oracle(cols, rpc, w):
    out = run(cols, rpc, w, "fp64", lam=1e-3, solver="parallel")
    x, _, r2 = oracle_solutions(out["inst"], 1e-3)
    np.testing.assert_allclose(out["p"], x, rtol=1e-12, atol=1e-12 * np.abs(x).max())
    np.testing.assert_allclose(out["res2"], r2, rtol=1e-9)


@pytest.mark.parametrize("solver", ["sweep", "parallel"])
def test_banded_fp32_refined_matches_oracle(solver):
    cols = [500, 1200, 77]
    out = run(cols, 4, 8, "fp32_refined", lam=1e-3, refine_steps=2, solver=solver)
    x, _, _ = oracle_solutions(out["inst"], 1e-3)
    assert_close(out["p"], x, 1e-5)


@pytest.mark.parametrize("solver", ["sweep", "parallel"])
def test_banded_given_D_and_no_damping(solver):
    cols = [30, 41]
    g = np.random.default_rng(3)
    D = np.abs(g.standard_normal(sum(cols))) + 0.5
    out = run(cols, 4, 8, "fp64", lam=0.2, D=D, solver=solver)
    x, _, _ = oracle_solutions(out["inst"], 0.2, D)
    np.testing.assert_allclose(out["p"], x, rtol=1e-11, atol=1e-12)
    out0 = run(cols, 4, 8, "fp64", lam=0.0, solver=solver)
    x0, _, _ = oracle_solutions(out0["inst"], 0.0, np.ones(sum(cols)))
    np.testing.assert_allclose(out0["p"], x0, rtol=1e-10, atol=1e-11)


@pytest.mark.parametrize("solver", ["sweep", "parallel"])
def test_banded_batch_scaled_sampled(solver):
    """A batch of 256 instances with n ~ U{1000..4000}: every instance's solution satisfies the
    optimality identity; 4 sampled instances match the oracle."""
    g = np.random.default_rng(1)
    cols = g.integers(1000, 4001, size=256)
    out = run(list(cols), 4, 8, "fp32_refined", lam=1e-3, refine_steps=2, solver=solver)
    off = 0
    worst = 0.0
    for k, d in enumerate(out["inst"]):
        n = d["n"]
        x = out["p"][off:off + n]
        start, vals = d["start"], d["vals"].astype(np.float64)
        D = bd.column_norms(start, vals, n)
        r = d["b"].astype(np.float64) - bd.matvec(start, vals, x)
        gr = bd.rmatvec(start, vals, r, n) - 1e-3 * D * D * x
        worst = max(worst, np.linalg.norm(gr) / (np.linalg.norm(vals) ** 2 * np.linalg.norm(x)))
        off += n
    assert worst < 1e-6
    sel = [0, 77, 200, 255]
    off = np.concatenate([[0], np.cumsum(cols)])
    for k in sel:
        d = out["inst"][k]
        x, *_ = bd.damped_solve(d["start"], d["vals"], d["b"], d["n"], 1e-3)
        got = out["p"][off[k]:off[k + 1]]
        assert_close(got, x, 1e-5)


def test_banded_parallel_large_instance():
    """One instance of 100,000 columns (400,000 rows): matches the oracle to 1e-5."""
    out = run([100000], 4, 8, "fp32_refined", lam=1e-3, refine_steps=2, solver="parallel", seed=9)
    x, _, _ = oracle_solutions(out["inst"], 1e-3)
    assert_close(out["p"], x, 1e-5)


@pytest.mark.slow
def test_banded_parallel_full_size_optimality():
    """n = 1,000,000 columns, 4,000,000 rows, lambda = 1e-3: the first-order condition
    J^T (b - J x) = lambda D^2 x holds to float accuracy after refinement."""
    out = run([1000000], 4, 8, "fp32_refined", lam=1e-3, refine_steps=2, solver="parallel", seed=4)
    d = out["inst"][0]
    x = out["p"]
    start, vals = d["start"], d["vals"].astype(np.float64)
    D = bd.column_norms(start, vals, d["n"])
    r = d["b"].astype(np.float64) - bd.matvec(start, vals, x)
    gr = bd.rmatvec(start, vals, r, d["n"]) - 1e-3 * D * D * x
    assert np.linalg.norm(gr) / (np.linalg.norm(vals) ** 2 * np.linalg.norm(x)) < 1e-7


def banded_batch_optimality(d, p, lam, chunk=256):
    """Worst instance of ||J^T (b - J x) - lambda D^2 x|| / (||J||_F^2 ||x||) over a batch held
    on the device (workloads.device layout), computed on the device with plain PyTorch ops in
    double, a chunk of instances at a time."""
    import torch
    vals, b = d["vals"], d["b"]
    cols, row0, col0 = d["cols"], d["row0"], d["col0"]
    w, rpc = d["w"], d["rows_per_col"]
    dev = vals.device
    x = p.double()
    worst = 0.0
    for k0 in range(0, cols.size, chunk):
        k1 = min(cols.size, k0 + chunk)
        R0, R1, C0, C1 = int(row0[k0]), int(row0[k1]), int(col0[k0]), int(col0[k1])
        nk = k1 - k0
        inst = torch.repeat_interleave(torch.arange(nk, device=dev), torch.from_numpy(rpc * cols[k0:k1]).to(dev))
        rloc = torch.arange(R1 - R0, device=dev) - torch.from_numpy(row0[k0:k1] - R0).to(dev)[inst]
        base = torch.from_numpy(col0[k0:k1] - C0).to(dev)[inst] + rloc // rpc
        idx = base[:, None] + torch.arange(w, device=dev)[None, :]
        end = torch.from_numpy(col0[k0 + 1:k1 + 1] - C0).to(dev)[inst][:, None]
        idx = torch.where(idx < end, idx, torch.zeros_like(idx))   # truncated band ends hold zeros
        V = vals[R0:R1].double()
        xc = x[C0:C1]
        r = b[R0:R1].double() - (V * xc[idx]).sum(1)
        flat = idx.reshape(-1)
        g = torch.zeros(C1 - C0, dtype=torch.float64, device=dev).index_add_(0, flat, (V * r[:, None]).reshape(-1))
        D2 = torch.zeros(C1 - C0, dtype=torch.float64, device=dev).index_add_(0, flat, (V * V).reshape(-1))
        D2 = torch.where(D2 > 0, D2, torch.ones_like(D2))
        g -= lam * D2 * xc
        cinst = torch.repeat_interleave(torch.arange(nk, device=dev), torch.from_numpy(cols[k0:k1]).to(dev))
        g2 = torch.zeros(nk, dtype=torch.float64, device=dev).index_add_(0, cinst, g * g)
        x2 = torch.zeros(nk, dtype=torch.float64, device=dev).index_add_(0, cinst, xc * xc)
        J2 = torch.zeros(nk, dtype=torch.float64, device=dev).index_add_(0, inst, (V * V).sum(1))
        worst = max(worst, float((g2.sqrt() / (J2 * x2.sqrt())).max()))
        del inst, rloc, base, idx, end, V, r, flat, g, D2, cinst
    return worst


@pytest.mark.slow
def test_banded_batch_full_size_4096_instances():
    """The 4096-instance batch of workload 4 at full size (n ~ U{1000..100000}, 4n rows each:
    about 2e8 columns and 8e8 rows, drawn on the device), parallel solver, FP32 refined: every
    instance satisfies the first-order condition J^T (b - J x) = lambda D^2 x to float accuracy
    (checked on the device); the smallest and the largest instance, copied to the host, match
    the oracle to 1e-5."""
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context
    from workloads import banded_batch_shapes
    from workloads.device import banded_batch_device
    cols = banded_batch_shapes()
    d = banded_batch_device(cols, seed_offset=0)
    ctx = Context(0, precision="fp32_refined")
    ctx.plan_banded(list(cols), rows_per_col=4, window=8, solver=SOLVER["parallel"])
    N = int(cols.sum())
    p = torch.empty(N, device="cuda", dtype=torch.float32)
    ctx.factor_solve(d["vals"].reshape(-1), d["b"], p, None, lam=1e-3, refine_steps=2)
    ctx.sync_status()
    ctx.close()
    assert banded_batch_optimality(d, p, 1e-3) < 1e-6
    for k in (int(np.argmin(cols)), int(np.argmax(cols))):
        r0, r1, c0, n = int(d["row0"][k]), int(d["row0"][k + 1]), int(d["col0"][k]), int(cols[k])
        vals = d["vals"][r0:r1].cpu().numpy()
        b = d["b"][r0:r1].cpu().numpy()
        start = np.arange(r1 - r0, dtype=np.int64) // 4
        x, *_ = bd.damped_solve(start, vals, b, n, 1e-3)
        got = p[c0:c0 + n].cpu().numpy().astype(np.float64)
        assert_close(got, x, 1e-5)


def test_banded_batch_solve_replays_in_cuda_graph():
    """The parallel banded factor + solve with refinement, captured once in a CUDA graph after a
    warm-up call and replayed on new J and b, gives the eager result bit for bit."""
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context
    from workloads.device import banded_batch_device
    cols = np.array([1500, 3000, 2200, 4100], dtype=np.int64)
    d0 = banded_batch_device(cols, seed_offset=1)
    d1 = banded_batch_device(cols, seed_offset=2)
    stream = torch.cuda.Stream()
    ctx = Context(0, stream=stream, precision="fp32_refined")
    ctx.plan_banded(list(cols), rows_per_col=4, window=8, solver=SOLVER["parallel"])
    J, b = d0["vals"].reshape(-1).clone(), d0["b"].clone()
    p = torch.empty(int(cols.sum()), device="cuda", dtype=torch.float32)
    torch.cuda.synchronize()
    solve = lambda: ctx.factor_solve(J, b, p, None, lam=1e-3, refine_steps=2)
    with torch.cuda.stream(stream):
        solve()
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        solve()
    with torch.cuda.stream(stream):
        J.copy_(d1["vals"].reshape(-1))
        b.copy_(d1["b"])
        graph.replay()
    stream.synchronize()
    replayed = p.clone()
    with torch.cuda.stream(stream):
        solve()
    stream.synchronize()
    ctx.sync_status()
    assert torch.equal(replayed, p)
    assert banded_batch_optimality(d1, p, 1e-3) < 1e-6
    ctx.close()
