"""GPU parity of Moré's two-factorization LM step (Sec. 5.2, Eq. LMTwoStep) on block-diagonal J.

Stage 1 is the undamped fused block QR (its Q^T b kept); stage 2, once per damping value,
factors [R_i; lambda^(1/2) D_i] per block.  The result must be the damped least-squares
solution of every block: the oracle's two-factorization step (oracle/more.py), and the
oracle's single Householder factorization of the augmented block [J_i; lambda^(1/2) D_i].
"""
import numpy as np
import pytest

from oracle import more
from oracle import structured as st
from tests.gpu_common import U32, U64, assert_blocks_within, assert_close, cuda_or_skip
from workloads import batched_blocks

pytestmark = pytest.mark.gpu


def blocks_problem(d):
    blocks, rhs = [], []
    for i in range(d["K"]):
        n, m = int(d["n"][i]), int(d["m"][i])
        v0, r0 = int(d["val_off"][i]), int(d["row_off"][i])
        blocks.append(np.asarray(d["vals"][v0:v0 + n * m], dtype=np.float64).reshape(m, n).T)
        rhs.append(np.asarray(d["b"][r0:r0 + n], dtype=np.float64))
    return st.BlockProblem(blocks=blocks, b=np.concatenate(rhs))


def augmented(d, Dv, lam):
    """The blocks [J_i; lambda^(1/2) D_i] with rhs [b_i; 0], in the workload's packing."""
    K = d["K"]
    n = d["n"].astype(np.int64)
    m = d["m"].astype(np.int64)
    vals, b = [], []
    for i in range(K):
        v0, r0, c0 = int(d["val_off"][i]), int(d["row_off"][i]), int(d["col_off"][i])
        A = np.asarray(d["vals"][v0:v0 + n[i] * m[i]], dtype=np.float64).reshape(m[i], n[i]).T
        Aa = np.vstack([A, np.sqrt(lam) * np.diag(Dv[c0:c0 + m[i]])])
        vals.append(Aa.T.reshape(-1))
        b.append(np.concatenate([np.asarray(d["b"][r0:r0 + n[i]], dtype=np.float64), np.zeros(m[i])]))
    na = n + m
    return dict(n=na.astype(np.uint8), m=m.astype(np.uint8), vals=np.concatenate(vals), b=np.concatenate(b), K=K,
                val_off=np.concatenate([[0], np.cumsum(na * m)]).astype(np.int64),
                row_off=np.concatenate([[0], np.cumsum(na)]).astype(np.int64),
                col_off=d["col_off"])


def stage1(torch, ctx, d):
    J = torch.from_numpy(np.asarray(d["vals"])).cuda().to(ctx.dtype)
    b = torch.from_numpy(np.asarray(d["b"])).cuda().to(ctx.dtype)
    p0 = torch.empty(int(d["col_off"][-1]), device="cuda", dtype=ctx.dtype)
    qtb = torch.empty(int(d["row_off"][-1]), device="cuda", dtype=ctx.dtype)
    ctx.plan_blocks(d["n"], d["m"])
    ctx.factor_solve(J, b, p0, qtb, refine_steps=0)
    return J, b, p0, qtb


@pytest.mark.parametrize("mapping", [None, "budget 256 1536 512 256 2048"])
def test_more_fp64_equals_oracle_for_several_lambdas(mapping):
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context
    d = batched_blocks(K=3000, seed_offset=41, dtype=np.float64)
    P = blocks_problem(d)
    Dv = st.column_norms(P)
    ctx = Context(0, precision="fp64")
    if mapping:
        ctx.plan_blocks(d["n"], d["m"])
        ctx.apply_tuning(mapping)
        J = torch.from_numpy(d["vals"]).cuda()
        b = torch.from_numpy(d["b"]).cuda()
        p0 = torch.empty(int(d["col_off"][-1]), device="cuda", dtype=torch.float64)
        qtb = torch.empty(int(d["row_off"][-1]), device="cuda", dtype=torch.float64)
        ctx.factor_solve(J, b, p0, qtb, refine_steps=0)
    else:
        J, b, p0, qtb = stage1(torch, ctx, d)
    p = torch.empty_like(p0)
    for lam in (1e-3, 0.5, 10.0):
        ctx.more_solve(qtb, p, None, lam)   # D = column norms of J
        ctx.sync_status()
        got = p.cpu().numpy()
        ref = more.block_steps(P.blocks, P.b, Dv, lam)
        assert_close(got, ref, 1e-12, what=f"lambda {lam}: ")
        assert_blocks_within(augmented(d, Dv, lam), got, None, 1e-12, U64, what=f"lambda {lam}: ")
    # lambda = 0: the undamped solution of stage 1 again
    ctx.more_solve(qtb, p, None, 0.0)
    ctx.sync_status()
    assert_close(p.cpu().numpy(), p0.cpu().numpy(), 1e-12)
    ctx.close()


def test_more_given_D_and_the_damped_fused_call():
    """An explicit D, and qrkit_factor_solve with lambda > 0 (stage 1 + stage 2 in one call)
    against the oracle's single factorization of the augmented blocks."""
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context
    d = batched_blocks(K=2000, seed_offset=42, dtype=np.float64)
    Dv = np.random.default_rng(3).uniform(0.5, 2.0, size=int(d["col_off"][-1]))
    lam = 0.2
    ctx = Context(0, precision="fp64")
    J, b, p0, qtb = stage1(torch, ctx, d)
    tD = torch.from_numpy(Dv).cuda()
    p = torch.empty_like(p0)
    ctx.more_solve(qtb, p, tD, lam)
    ctx.sync_status()
    aug = augmented(d, Dv, lam)
    assert_blocks_within(aug, p.cpu().numpy(), None, 1e-12, U64)
    p2 = torch.empty_like(p0)
    ctx.factor_solve(J, b, p2, None, tD, lam, refine_steps=0)
    ctx.sync_status()
    assert_blocks_within(aug, p2.cpu().numpy(), None, 1e-12, U64)
    ctx.close()


def test_more_fp32_within_float_bound():
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context
    d = batched_blocks(K=3000, seed_offset=43)
    P = blocks_problem(d)
    Dv = st.column_norms(P)
    ctx = Context(0, precision="fp32")
    J, b, p0, qtb = stage1(torch, ctx, d)
    p = torch.empty_like(p0)
    lam = 1e-2
    ctx.more_solve(qtb, p, None, lam)
    ctx.sync_status()
    assert_blocks_within(augmented(d, Dv, lam), p.cpu().numpy(), None, 1e-6, U32, c=16.0)
    ctx.close()


def test_more_needs_a_factor():
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context, QRKitError
    d = batched_blocks(K=10, seed_offset=44, dtype=np.float64)
    ctx = Context(0, precision="fp64")
    ctx.plan_blocks(d["n"], d["m"])
    q = torch.zeros(int(d["row_off"][-1]), device="cuda", dtype=torch.float64)
    p = torch.zeros(int(d["col_off"][-1]), device="cuda", dtype=torch.float64)
    with pytest.raises(QRKitError) as e:
        ctx.more_solve(q, p, None, 1.0)
    assert e.value.status == 9
    ctx.close()


def oracle_blocks_and_d(d):
    P = blocks_problem(d)
    dcol = np.concatenate([np.sqrt(np.sum(B * B, axis=0)) for B in P.blocks])
    dcol[dcol == 0.0] = 1.0
    return P, dcol


@pytest.mark.parametrize("precision,mapping", [("fp64", None), ("fp64", "budget 256 1536 512 256 2048"),
                                               ("fp32", None)])
def test_trust_region_lambda_equals_oracle(precision, mapping):
    """Moré's trust-region lambda (qrkit_more_trust_region) against the oracle's iteration on the
    same blocks: lambda to the iteration's rounding, the step as the damped solution there, and
    the scaled length within sigma of the radius."""
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context
    d = batched_blocks(K=3000, seed_offset=31, dtype=np.float64 if precision == "fp64" else np.float32)
    P, dcol = oracle_blocks_and_d(d)
    p_gn = np.concatenate([np.linalg.lstsq(B, P.b[int(d["row_off"][i]):int(d["row_off"][i + 1])], rcond=None)[0]
                           for i, B in enumerate(P.blocks)])
    gn_len = float(np.linalg.norm(dcol * p_gn))
    ctx = Context(0, precision=precision)
    J, b, p0, qtb = stage1(torch, ctx, d)
    if mapping:
        ctx.apply_tuning(mapping)
        ctx.factor_solve(J, b, p0, qtb, refine_steps=0)
    p = torch.empty_like(p0)
    for frac in (0.02, 0.3):
        delta = frac * gn_len
        lam, it = ctx.more_trust_region(qtb, p, delta, sigma=0.1)
        ctx.sync_status()
        lam_o, p_o, it_o = more.trust_region_lambda(P.blocks, P.b, dcol, delta, sigma=0.1)
        pg = p.cpu().numpy().astype(np.float64)
        length = float(np.linalg.norm(dcol * pg))
        assert abs(length - delta) <= 0.1 * delta * (1 + 1e-3)
        if precision == "fp64":
            assert it == it_o
            assert lam == pytest.approx(lam_o, rel=1e-8)
            assert_close(pg, p_o, 1e-10)
        else:
            # float stage 2: the same iteration on slightly different sums
            assert lam == pytest.approx(lam_o, rel=1e-3)
            p_ref = more.block_steps(P.blocks, P.b, dcol, lam)
            assert_close(pg, p_ref, 2e-4)
    # a radius the undamped step already fits: lambda = 0 and the undamped step
    lam, it = ctx.more_trust_region(qtb, p, 2.0 * gn_len)
    assert lam == 0.0 and it == 0
    if precision == "fp64":
        assert_close(p.cpu().numpy().astype(np.float64), p_gn, 1e-10)
    else:   # the same back-substitution as stage 1's
        assert_close(p.cpu().numpy().astype(np.float64), p0.cpu().numpy().astype(np.float64), 1e-5)
    ctx.close()


def test_trust_region_rejects_bad_arguments():
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context, qrkit
    d = batched_blocks(K=100, seed_offset=32, dtype=np.float64)
    ctx = Context(0, precision="fp64")
    J, b, p0, qtb = stage1(torch, ctx, d)
    for delta, sigma, iters in ((0.0, 0.1, 10), (1.0, 0.0, 10), (1.0, 1.0, 10), (1.0, 0.1, 0)):
        with pytest.raises(qrkit.QRKitError):
            ctx.more_trust_region(qtb, p0, delta, sigma=sigma, max_iter=iters)
    ctx.close()
