"""The multi-rank path on CPU: two gloo ranks each solve their own share of independent blocks
with the float64 oracle; together they reproduce the single-process result, and the combined
timing is the maximum over the ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1802_03773_gb300.replicas import max_over_ranks, share  # noqa: E402


def test_share_covers_every_unit_once():
    for total in (0, 1, 7, 1000, 1_000_003):
        for world in (1, 2, 3, 8):
            spans = [share(total, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == total
            for (a, b), (c, d) in zip(spans, spans[1:]):
                assert b == c
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        share(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import householder as hh
    from workloads import batched_blocks
    d = batched_blocks(K=400, seed_offset=3)
    lo, hi = share(d["K"], rank, world)
    xs = []
    for i in range(lo, hi):
        n, m = int(d["n"][i]), int(d["m"][i])
        v0, r0 = int(d["val_off"][i]), int(d["row_off"][i])
        A = np.asarray(d["vals"][v0:v0 + n * m], dtype=np.float64).reshape(m, n).T
        xs.append(hh.lstsq(A, np.asarray(d["b"][r0:r0 + n], dtype=np.float64))[0])
    x = np.concatenate(xs)
    parts = [None] * world
    dist.all_gather_object(parts, x)
    t = max_over_ranks(10.0 * (rank + 1))
    if rank == 0:
        out.put((np.concatenate(parts), t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_single_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    x, t = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from oracle import householder as hh
    from workloads import batched_blocks
    d = batched_blocks(K=400, seed_offset=3)
    ref = []
    for i in range(d["K"]):
        n, m = int(d["n"][i]), int(d["m"][i])
        v0, r0 = int(d["val_off"][i]), int(d["row_off"][i])
        A = np.asarray(d["vals"][v0:v0 + n * m], dtype=np.float64).reshape(m, n).T
        ref.append(hh.lstsq(A, np.asarray(d["b"][r0:r0 + n], dtype=np.float64))[0])
    np.testing.assert_array_equal(x, np.concatenate(ref))
    assert t == 20.0
