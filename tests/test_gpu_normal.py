"""GPU parity of the normal-equations comparison path (Eq. 1 by Cholesky with the Schur
complement onto the shared block; Sec. 1 / Sec. 6.1): the float64 variant against the oracle's
Cholesky of the assembled J^T J + lambda D^2, and the float32 variant's error growing with
cond(A)^2 where the QR path's does not."""
import numpy as np
import pytest

from oracle import curvefit as cf
from oracle import lm
from oracle import normal as nrm
from oracle import structured as st
from tests.gpu_common import assert_close, cuda_or_skip
from tests.test_gpu_composed import packed, problem_from, rel
from workloads import block_angular_dense, curvefit_problem

pytestmark = pytest.mark.gpu


def normal_gpu(precision, plan, J, S, b, N, lam, D=None):
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context
    ctx = Context(0, precision=precision)
    plan(ctx)
    dt = torch.float64 if precision == "fp64" else torch.float32
    tJ = torch.from_numpy(J).cuda()
    tS = None if S is None else torch.from_numpy(S).cuda()
    tb = torch.from_numpy(b).cuda()
    tD = None if D is None else torch.from_numpy(D).to(dt).cuda()
    p = torch.empty(N, device="cuda", dtype=dt)
    ctx.normal_solve(tJ, tS, tb, p, D=tD, lam=lam)
    ctx.sync_status()
    out = p.cpu().numpy().astype(np.float64)
    ctx.close()
    return out


def dense_case(K, s, decades, dtype):
    from paper_1802_03773_gb300 import qrkit
    d = block_angular_dense(K=K, n=4, m=2, s=s, scale_decades=decades)
    P = problem_from(d)
    J, S, b = packed(d, dtype)
    plan = lambda ctx: ctx.plan_blocks(np.full(K, 4), np.full(K, 2), qrkit.COUPLED_DENSE, shared_cols=s)
    return P, J, S, b, plan


def test_normal_dense_fp64_matches_oracle_cholesky():
    P, J, S, b, plan = dense_case(60, 12, 1.0, np.float64)
    p = normal_gpu("fp64", plan, J, S, b, P.N, P.lam)
    Jd = st.assemble_J(P)
    p_ref = nrm.solve(Jd, np.asarray(P.b), st.damping(P), P.lam)
    assert_close(p, p_ref, 1e-10)


def test_normal_window_fp64_matches_oracle_cholesky():
    from paper_1802_03773_gb300 import qrkit
    draw = curvefit_problem(npoints=400, Kc=12, seed_offset=3)
    data, x0 = cf.make_data(draw)
    Pb, _ = lm.curvefit_system(x0, data, 1e-2)
    K = Pb.K
    J = np.concatenate([blk.T.reshape(-1) for blk in Pb.blocks])
    S = np.concatenate([c.T.reshape(-1) for c in Pb.coupled])
    plan = lambda ctx: ctx.plan_blocks(np.full(K, 2), np.full(K, 1), qrkit.COUPLED_WINDOW, shared_cols=Pb.s,
                                       window=8, window_start=np.asarray(Pb.start, dtype=np.int32))
    p = normal_gpu("fp64", plan, J, S, np.asarray(Pb.b), Pb.N, Pb.lam)
    p_ref = nrm.solve(st.assemble_J(Pb), np.asarray(Pb.b), st.damping(Pb), Pb.lam)
    assert_close(p, p_ref, 1e-9)


def test_normal_blocks_only_fp64():
    from paper_1802_03773_gb300 import qrkit
    g = np.random.default_rng(4)
    K = 300
    n = g.integers(1, 9, size=K)
    m = np.minimum(g.integers(1, 5, size=K), 8)
    blocks = [g.standard_normal((int(n[i]), int(m[i]))) for i in range(K)]
    b = g.standard_normal(int(n.sum()))
    P = st.BlockProblem(blocks=blocks, b=b, lam=0.3)
    J = np.concatenate([x.T.reshape(-1) for x in blocks])
    plan = lambda ctx: ctx.plan_blocks(n, m)
    p = normal_gpu("fp64", plan, J, None, b, P.N, P.lam)
    p_ref = nrm.solve(st.assemble_J(P), b, st.damping(P), P.lam)
    assert_close(p, p_ref, 1e-10)


def test_normal_fp32_loses_cond_squared():
    """cond(A) ~ 1e3 (columns scaled over 3 decades): float Cholesky of the normal equations
    misses by ~cond^2 u while float QR with refinement stays within 1e-5 of the float64 QR."""
    torch = cuda_or_skip()
    P, J, S, b, plan = dense_case(100, 20, 3.0, np.float32)
    # the float64 oracle solves the float-rounded values
    Pr = st.BlockProblem(blocks=[x.astype(np.float32).astype(np.float64) for x in P.blocks],
                         coupled=[x.astype(np.float32).astype(np.float64) for x in P.coupled],
                         s=P.s, b=np.asarray(P.b, np.float32).astype(np.float64), lam=P.lam)
    p_ref, _ = st.factor_and_solve(Pr)
    A, _ = st.assemble_augmented(Pr)
    sv = np.linalg.svd(A, compute_uv=False)
    kappa = sv[0] / sv[-1]
    p_chol = normal_gpu("fp32_refined", plan, J, S, b, P.N, P.lam)
    e_chol = rel(p_chol, p_ref)
    from tests.test_gpu_composed import run as qr_run
    d = block_angular_dense(K=100, n=4, m=2, s=20, scale_decades=3.0)
    e_qr = rel(qr_run(d, "fp32_refined", refine_steps=2)["p"], p_ref)
    print(f"cond(A) = {kappa:.3g}: float Cholesky error {e_chol:.3g}, float QR + refinement {e_qr:.3g}")
    assert e_qr <= 1e-5
    assert e_chol <= 50.0 * kappa ** 2 * 2.0 ** -24
    assert e_chol > 10.0 * e_qr
