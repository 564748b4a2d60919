"""The distributed dense-S solve on CPU: two gloo ranks run the driver of
paper_1802_03773_gb300/distributed.py (column sums all-reduced, local factorizations, the
ranks' triangles all-gathered and solved again, local back-substitution) with the float64
oracle standing in for the library's local steps; the assembled solution equals the
single-process solve of the whole problem (Sec. 4.2 with the reduced block by TSQR)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, lam, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1802_03773_gb300.distributed import TorchComm, tsqr_solve
    from paper_1802_03773_gb300.replicas import share
    from tests.distributed_common import OracleOps, part, problem
    d = problem()
    lo, hi = share(d["K"], rank, world)
    blocks, S, b = part(d, lo, hi)
    ops = OracleOps(blocks, S, b, d["s"])
    p = tsqr_solve(TorchComm(), ops, None, None, None, lam, ops.nb, d["s"])
    parts = [None] * world
    dist.all_gather_object(parts, p.numpy())
    if rank == 0:
        out.put(parts)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,lam", [(2, 1e-2), (3, 0.0)])
def test_gloo_ranks_reproduce_the_single_process_solve(world, lam):
    from tests.distributed_common import problem, reference
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, lam, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    d = problem()
    s = d["s"]
    ref = reference(d, lam)
    # every rank has the same shared unknowns
    for x in parts[1:]:
        np.testing.assert_allclose(x[-s:], parts[0][-s:], rtol=1e-14, atol=1e-15)
    got = np.concatenate([x[:-s] for x in parts] + [parts[0][-s:]])
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
