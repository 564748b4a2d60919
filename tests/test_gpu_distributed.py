"""The distributed dense-S solve through the library: ranks emulated by threads in one process,
each with a context of its own on the one GPU (their kernels never wait on one another; the
exchanges are host-side), against the oracle's single-process solve (Sec. 4.2, reduced block by
TSQR across ranks)."""
import threading

import numpy as np
import pytest

from tests.distributed_common import part, problem, reference
from tests.gpu_common import assert_close, cuda_or_skip

pytestmark = pytest.mark.gpu


class ThreadComm:
    def __init__(self, rank, shared):
        self.rank, self.shared = rank, shared
        self.world_size = len(shared["slots"])

    def _swap(self, t):
        sh = self.shared
        sh["slots"][self.rank] = t.clone()
        sh["barrier"].wait()
        vals = [x.clone() for x in sh["slots"]]
        sh["barrier"].wait()
        return vals

    def all_reduce_sum(self, t):
        vals = self._swap(t)
        tot = vals[0]
        for v in vals[1:]:
            tot = tot + v
        t.copy_(tot)
        return t

    def all_gather(self, t):
        return self._swap(t)


@pytest.mark.parametrize("world,precision,tol", [(2, "fp64", 1e-10), (3, "fp64", 1e-10), (2, "fp32", 2e-3)])
def test_threads_as_ranks_equal_the_oracle(world, precision, tol):
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context, qrkit
    from paper_1802_03773_gb300.distributed import LibraryOps, tsqr_solve
    from paper_1802_03773_gb300.replicas import share
    d = problem(K=300, s=24, seed=5)
    lam, s, n, m = 1e-2, d["s"], d["n"], d["m"]
    dt = torch.float64 if precision == "fp64" else torch.float32
    shared = {"slots": [None] * world, "barrier": threading.Barrier(world)}
    results, errors = [None] * world, []

    def rank_main(r):
        try:
            lo, hi = share(d["K"], r, world)
            blocks, S, b = part(d, lo, hi)
            ctx = Context(0, precision=precision)
            K = hi - lo
            ctx.plan_blocks(np.full(K, n), np.full(K, m), qrkit.COUPLED_DENSE, shared_cols=s)
            J = torch.from_numpy(np.concatenate([blk.T.reshape(-1) for blk in blocks])).cuda().to(dt)
            St = torch.from_numpy(np.ascontiguousarray(S.T).reshape(-1)).cuda().to(dt)
            bt = torch.from_numpy(b).cuda().to(dt)
            p = tsqr_solve(ThreadComm(r, shared), LibraryOps(ctx, K * m, s), J, St, bt, lam, K * m, s)
            ctx.sync_status()
            results[r] = p.cpu().numpy().astype(np.float64)
            ctx.close()
        except Exception as ex:   # pragma: no cover - reported below
            errors.append(ex)
            shared["barrier"].abort()

    threads = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not errors, errors
    for x in results[1:]:
        np.testing.assert_allclose(x[-s:], results[0][-s:], rtol=1e-12, atol=1e-14)
    got = np.concatenate([x[:-s] for x in results] + [results[0][-s:]])
    assert_close(got, reference(d, lam), tol, floor=1e-2)


def test_dense_lstsq_equals_the_oracle():
    torch = cuda_or_skip()
    from oracle import householder as hh
    from paper_1802_03773_gb300 import Context
    g = np.random.default_rng(17)
    for M, N in ((300, 40), (1152, 128), (64, 64)):
        A = g.standard_normal((M, N)) * 10.0 ** g.uniform(-1, 1, size=N)
        b = g.standard_normal(M)
        ctx = Context(0, precision="fp64")
        At = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
        x = torch.empty(N, dtype=torch.float64, device="cuda")
        r2 = ctx.dense_lstsq(At, torch.from_numpy(b).cuda(), x)
        ctx.sync_status()
        ref, f, qtb = hh.lstsq(A, b)
        assert_close(x.cpu().numpy(), ref, 1e-11)
        assert r2 == pytest.approx(float(qtb[N:] @ qtb[N:]), rel=1e-9)
        ctx.close()
