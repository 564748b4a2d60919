"""The allocation-free block solve gives the same solution as the context-based one.

qrkit_block_solve_noalloc serves callers that cannot call cudaMalloc (a framework that owns
all device memory, a fixed memory budget): it keeps every intermediate in one static device
array.  It runs the tile kernel of the fused solve, so this test pins the context to the same
tile mapping, calls the allocation-free entry point through the C-ABI twice in a row (the array
keeps the previous call's contents) and compares each result with qrkit_factor_solve's and,
block by block, with the FP64 oracle's.  It lives in its own file so that pytest collects it
last.
"""
import numpy as np
import pytest

from tests.gpu_common import U32, U64, assert_blocks_within, cuda_or_skip
from workloads import batched_blocks

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [("fp32_refined", 1e-5), ("fp32", 1e-4), ("fp64", 1e-12)])
def test_noalloc_matches_context_solve_twice(precision, tol):
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context, qrkit
    dtype = np.float64 if precision == "fp64" else np.float32
    d = batched_blocks(K=20000, seed_offset=21, dtype=dtype)
    tdt = torch.float64 if precision == "fp64" else torch.float32
    J = torch.from_numpy(np.asarray(d["vals"])).cuda().to(tdt)
    b = torch.from_numpy(np.asarray(d["b"])).cuda().to(tdt)
    ncols = int(d["col_off"][-1])
    ctx = Context(0, precision=precision)
    ctx.plan_blocks(d["n"], d["m"])
    ctx.apply_tuning("budget 256 1536 512 256 2048" if precision == "fp64" else "budget 256 3072 1024 512 4096")
    p_ref = torch.empty(ncols, device="cuda", dtype=tdt)
    ctx.factor_solve(J, b, p_ref, None, refine_steps=2)
    ctx.sync_status()
    ref = p_ref.cpu().numpy().astype(np.float64)
    ctx.close()
    for call in range(2):
        p = torch.full((ncols,), float("nan"), device="cuda", dtype=tdt)
        qrkit.block_solve_noalloc(d["n"], d["m"], J, b, p, precision=precision, refine_steps=2)
        got = p.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got)), f"call {call}: non-finite output"
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= tol, f"call {call}: relative difference {err:.3e}"
        # against the oracle, per block: the mode's target (FP32 plain: the float error bound)
        target, u = {"fp32_refined": (1e-5, U64), "fp64": (1e-12, U64), "fp32": (1e-6, U32)}[precision]
        assert_blocks_within(d, got, None, target, u, c=8.0 if u == U32 else None, what=f"call {call}: ")


def test_noalloc_restores_the_current_device():
    """The call makes its device current only while it runs."""
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import qrkit
    d = batched_blocks(K=500, seed_offset=22)
    J = torch.from_numpy(d["vals"]).cuda()
    b = torch.from_numpy(d["b"]).cuda()
    p = torch.empty(int(d["col_off"][-1]), device="cuda")
    before = torch.cuda.current_device()
    qrkit.block_solve_noalloc(d["n"], d["m"], J, b, p)
    assert torch.cuda.current_device() == before


def test_noalloc_rejects_oversized_problem():
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import qrkit
    d = batched_blocks(K=400_000)   # about 12 million values: more than the array holds
    J = torch.from_numpy(d["vals"]).cuda()
    b = torch.from_numpy(d["b"]).cuda()
    p = torch.empty(int(d["col_off"][-1]), device="cuda")
    with pytest.raises(qrkit.QRKitError) as e:
        qrkit.block_solve_noalloc(d["n"], d["m"], J, b, p)
    assert e.value.status == 8
