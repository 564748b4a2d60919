"""GPU test of the autotuner: a choice is made for a block plan and a banded plan, written to
the cache, reused by a fresh context, and the tuned configuration still solves to the oracle's
accuracy."""
import numpy as np
import pytest

from oracle import banded as bd
from tests.gpu_common import cuda_or_skip, oracle_block
from workloads import banded_problem, batched_blocks

pytestmark = pytest.mark.gpu


def test_autotune_blocks_and_cache(tmp_path):
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context
    d = batched_blocks(K=100_000, seed_offset=21)
    J = torch.from_numpy(d["vals"]).cuda()
    b = torch.from_numpy(d["b"]).cuda()
    p = torch.empty(int(d["col_off"][-1]), device="cuda", dtype=torch.float32)
    cache = str(tmp_path / "tune.txt")
    ctx = Context(0, precision="fp32_refined")
    ctx.plan_blocks(d["n"], d["m"])
    choice = ctx.autotune(J, b, p, refine_steps=2, cache_path=cache)
    assert choice.startswith("budget ") or choice.startswith("tasks ")
    lines = open(cache).read().strip().splitlines()
    assert len(lines) == 1 and lines[0].endswith(choice)
    ctx.factor_solve(J, b, p, None, refine_steps=2)
    ctx.sync_status()
    x = p.cpu().numpy().astype(np.float64)
    idx = np.random.default_rng(2).choice(100_000, 500, replace=False)
    num = den = 0.0
    for i in idx:
        xi = oracle_block(d, i)[0]
        c0, m = int(d["col_off"][i]), int(d["m"][i])
        num += float(np.sum((x[c0:c0 + m] - xi) ** 2))
        den += float(np.sum(xi ** 2))
    assert np.sqrt(num / den) <= 1e-5
    ctx.close()
    ctx2 = Context(0, precision="fp32_refined")
    ctx2.plan_blocks(d["n"], d["m"])
    assert ctx2.autotune(J, b, p, refine_steps=2, cache_path=cache) == choice
    assert len(open(cache).read().strip().splitlines()) == 1   # found, not timed again
    ctx2.close()


def test_autotune_banded(tmp_path):
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context
    q = banded_problem(n=20_000, rows_per_col=4, w=8, seed_offset=3)
    J = torch.from_numpy(np.ascontiguousarray(q["vals"].reshape(-1))).cuda()
    b = torch.from_numpy(q["b"]).cuda()
    p = torch.empty(20_000, device="cuda", dtype=torch.float32)
    ctx = Context(0, precision="fp32_refined")
    ctx.plan_banded([20_000], rows_per_col=4, window=8)
    choice = ctx.autotune(J, b, p, refine_steps=2, cache_path=str(tmp_path / "tune.txt"))
    assert choice.startswith("compress ")
    ctx.factor_solve(J, b, p, None, lam=1e-3, refine_steps=2)
    ctx.sync_status()
    x, *_ = bd.damped_solve(q["start"], q["vals"], q["b"], 20_000, 1e-3)
    assert np.linalg.norm(p.cpu().numpy() - x) / np.linalg.norm(x) <= 1e-5
    ctx.close()
