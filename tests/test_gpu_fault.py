"""Failure detection without a GPU fault: a bounded device wait that runs out.

The tile mapping of the block solve waits for its bulk copies on an mbarrier with a poll
limit.  With the limit set to zero every such wait gives up at once: the kernel records
QRKIT_ETIMEOUT in the device status word, waits (with a limit of its own) for its copies in
flight and returns; nothing traps or hangs.  The context then solves correctly again once the
limit is restored.
"""
import numpy as np
import pytest

from tests.gpu_common import U64, assert_blocks_within, cuda_or_skip
from workloads import batched_blocks

pytestmark = pytest.mark.gpu


def test_zero_poll_limit_reports_timeout_and_context_recovers():
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context, QRKitError
    d = batched_blocks(K=5000, seed_offset=31)
    ctx = Context(0, precision="fp32_refined")
    ctx.plan_blocks(d["n"], d["m"])
    ctx.apply_tuning("budget 256 3072 1024 512 4096")   # the tile mapping (bounded mbarrier waits)
    J = torch.from_numpy(d["vals"]).cuda()
    b = torch.from_numpy(d["b"]).cuda()
    p = torch.empty(int(d["col_off"][-1]), device="cuda")
    ctx.set_wait_limit(0)
    ctx.factor_solve(J, b, p, None, refine_steps=2)
    with pytest.raises(QRKitError) as e:
        ctx.sync_status()
    assert e.value.status == 6   # QRKIT_ETIMEOUT
    ctx.sync_status()            # read and cleared
    ctx.set_wait_limit(1 << 26)
    ctx.factor_solve(J, b, p, None, refine_steps=2)
    ctx.sync_status()
    assert_blocks_within(d, p.cpu().numpy(), None, 1e-5, U64)
    ctx.close()


def test_negative_poll_limit_rejected():
    cuda_or_skip()
    from paper_1802_03773_gb300 import Context, QRKitError
    ctx = Context(0, precision="fp32")
    with pytest.raises(QRKitError) as e:
        ctx.set_wait_limit(-1)
    assert e.value.status == 1
    ctx.close()
