"""GPU parity of the windowed block-angular solve: J = [blkdiag(2x1 latent blocks) | S] with
each point's rows touching 8 consecutive shared columns (cubic B-spline curve fit), damping rows
interleaved (Secs. 4.1, 4.2, 4.4, 4.5, 5.2)."""
import numpy as np
import pytest

from oracle import curvefit as cf
from oracle import lm
from oracle import structured as st
from tests.gpu_common import assert_close, cuda_or_skip
from workloads import curvefit_problem

pytestmark = pytest.mark.gpu


def sorted_system(npoints, Kc, lam, seed=0, round32=False):
    """The damped LM system at the start point, points sorted by segment (the row permutation);
    round32: J, S and b rounded once to float32 (the system a float factorization is given)."""
    draw = curvefit_problem(npoints=npoints, Kc=Kc, seed_offset=seed)
    data, x0 = cf.make_data(draw)
    t, P = cf.unpack(x0, npoints)
    seg, _ = cf.segment(t, Kc)
    order = np.argsort(seg, kind="stable")
    data = data[order]
    x0 = cf.pack(t[order], P)
    Pb, f = lm.curvefit_system(x0, data, lam, round32=round32)
    return Pb, f


def run(Pb, precision, refine_steps=2):
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context, qrkit
    dt = np.float64 if precision == "fp64" else np.float32
    K = Pb.K
    J = np.concatenate([blk.T.reshape(-1) for blk in Pb.blocks]).astype(dt)
    S = np.concatenate([c.T.reshape(-1) for c in Pb.coupled]).astype(dt)
    b = np.asarray(Pb.b).astype(dt)
    ctx = Context(0, precision=precision)
    ctx.plan_blocks(np.full(K, 2), np.full(K, 1), qrkit.COUPLED_WINDOW, shared_cols=Pb.s, window=8,
                    window_start=np.asarray(Pb.start, dtype=np.int32))
    tJ, tS, tb = (torch.from_numpy(a).cuda() for a in (J, S, b))
    ctx.factor(tJ, tS, None, Pb.lam)
    p = torch.empty(Pb.N, device="cuda", dtype=ctx.dtype)
    ctx.solve(tb, p, refine_steps=refine_steps)
    ctx.sync_status()
    out = p.cpu().numpy().astype(np.float64)
    ctx.close()
    return out


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("npoints,Kc", [(300, 12), (2000, 64)])
def test_window_fp64_matches_oracle(npoints, Kc):
    Pb, _ = sorted_system(npoints, Kc, 1e-2)
    p_ref, _ = st.factor_and_solve(Pb, reduced_solver=st.banded_reduced_solver())
    p = run(Pb, "fp64", refine_steps=0)
    assert_close(p, p_ref, 1e-12)


def test_window_fp32_refined_matches_oracle():
    """The oracle solves the float-rounded system in float64 (the system the float solve is
    given): every component within 1e-5 of it (componentwise, with the small components)."""
    Pb, _ = sorted_system(4000, 128, 1e-3, seed=2, round32=True)
    p_ref, _ = st.factor_and_solve(Pb, reduced_solver=st.banded_reduced_solver())
    p = run(Pb, "fp32_refined", refine_steps=2)
    assert_close(p, p_ref, 1e-5)


def shuffled(Pb, seed):
    """The same problem with its blocks in a random order (the P_r sort must undo it)."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(Pb.K)
    ro = Pb.row_offsets()
    b = np.concatenate([np.asarray(Pb.b)[ro[i]:ro[i + 1]] for i in perm])
    return st.BlockProblem(blocks=[Pb.blocks[i] for i in perm], coupled=[Pb.coupled[i] for i in perm],
                           start=np.asarray(Pb.start)[perm], s=Pb.s, b=b, lam=Pb.lam)


def test_window_unsorted_starts_and_row_order():
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context, qrkit
    Pb = shuffled(sorted_system(900, 24, 1e-2, seed=5)[0], 7)
    p_ref, _ = st.factor_and_solve(Pb, reduced_solver=st.banded_reduced_solver())
    p = run(Pb, "fp64", refine_steps=0)
    assert_close(p, p_ref, 1e-12)
    # P_r of the reduced block: rows (2 per block with damping) sorted by (start, row index)
    K = Pb.K
    J = np.concatenate([blk.T.reshape(-1) for blk in Pb.blocks])
    S = np.concatenate([c.T.reshape(-1) for c in Pb.coupled])
    ctx = Context(0, precision="fp64")
    ctx.plan_blocks(np.full(K, 2), np.full(K, 1), qrkit.COUPLED_WINDOW, shared_cols=Pb.s, window=8,
                    window_start=np.asarray(Pb.start, dtype=np.int32))
    tJ, tS = torch.from_numpy(J).cuda(), torch.from_numpy(S).cuda()
    ctx.factor(tJ, tS, None, Pb.lam)
    order = torch.empty(2 * K, dtype=torch.int64, device="cuda")
    ctx.get_row_order(order)
    ctx.sync_status()
    row_start = np.repeat(np.asarray(Pb.start, dtype=np.int64), 2)
    expect = np.lexsort((np.arange(2 * K), row_start))
    assert np.array_equal(order.cpu().numpy(), expect)
    ctx.close()


def test_window_set_start_on_device():
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context, qrkit
    Pb = shuffled(sorted_system(500, 16, 1e-3, seed=6)[0], 8)
    p_ref, _ = st.factor_and_solve(Pb, reduced_solver=st.banded_reduced_solver())
    K = Pb.K
    ctx = Context(0, precision="fp32_refined")
    ctx.plan_blocks(np.full(K, 2), np.full(K, 1), qrkit.COUPLED_WINDOW, shared_cols=Pb.s, window=8,
                    window_start=np.zeros(K, dtype=np.int32))
    ctx.set_window_start(torch.from_numpy(np.asarray(Pb.start, dtype=np.int32)).cuda())
    J = np.concatenate([blk.T.reshape(-1) for blk in Pb.blocks]).astype(np.float32)
    S = np.concatenate([c.T.reshape(-1) for c in Pb.coupled]).astype(np.float32)
    tJ, tS, tb = (torch.from_numpy(a).cuda() for a in (J, S, np.asarray(Pb.b, dtype=np.float32)))
    ctx.factor(tJ, tS, None, Pb.lam)
    p = torch.empty(Pb.N, device="cuda", dtype=torch.float32)
    ctx.solve(tb, p, refine_steps=2)
    ctx.sync_status()
    # the oracle solves the float-rounded values in float64
    Pr = st.BlockProblem(blocks=[b.astype(np.float32).astype(np.float64) for b in Pb.blocks],
                         coupled=[c.astype(np.float32).astype(np.float64) for c in Pb.coupled],
                         start=Pb.start, s=Pb.s, b=np.asarray(Pb.b, np.float32).astype(np.float64), lam=Pb.lam)
    p_ref, _ = st.factor_and_solve(Pr, reduced_solver=st.banded_reduced_solver())
    assert_close(p.cpu().numpy().astype(np.float64), p_ref, 1e-5)
    ctx.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32_refined", 1e-5)])
def test_window_segments(precision, tol):
    """Three independent curve-fit systems as one structure with three segments of S."""
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context, qrkit
    parts = [sorted_system(n, kc, 1e-2, seed=sd)[0] for n, kc, sd in ((300, 12, 1), (700, 20, 2), (200, 8, 3))]
    blocks, coupled, start, b = [], [], [], []
    c0 = 0
    for Pk in parts:
        blocks += Pk.blocks
        coupled += Pk.coupled
        start.append(np.asarray(Pk.start) + c0)
        b.append(np.asarray(Pk.b))
        c0 += Pk.s
    dt = np.float64 if precision == "fp64" else np.float32
    r = (lambda a: a) if precision == "fp64" else (lambda a: np.asarray(a, np.float32).astype(np.float64))
    Pall = st.BlockProblem(blocks=[r(x) for x in blocks], coupled=[r(x) for x in coupled],
                           start=np.concatenate(start), s=c0, b=r(np.concatenate(b)), lam=1e-2)
    p_ref, _ = st.factor_and_solve(Pall, reduced_solver=st.banded_reduced_solver())
    K = Pall.K
    ctx = Context(0, precision=precision)
    ctx.plan_blocks(np.full(K, 2), np.full(K, 1), qrkit.COUPLED_WINDOW, shared_cols=c0, window=8,
                    window_start=np.asarray(Pall.start, dtype=np.int32),
                    segment_cols=[Pk.s for Pk in parts], segment_blocks=[Pk.K for Pk in parts])
    J = np.concatenate([x.T.reshape(-1) for x in Pall.blocks]).astype(dt)
    S = np.concatenate([x.T.reshape(-1) for x in Pall.coupled]).astype(dt)
    tJ, tS, tb = (torch.from_numpy(a).cuda() for a in (J, S, np.asarray(Pall.b).astype(dt)))
    ctx.factor(tJ, tS, None, Pall.lam)
    p = torch.empty(Pall.N, device="cuda", dtype=ctx.dtype)
    ctx.solve(tb, p, refine_steps=2)
    ctx.sync_status()
    assert_close(p.cpu().numpy().astype(np.float64), p_ref, tol)
    ctx.close()
