"""GPU parity of the windowed block-angular solve: J = [blkdiag(2x1 latent blocks) | S] with
each point's rows touching 8 consecutive shared columns (cubic B-spline curve fit), damping rows
interleaved (Secs. 4.1, 4.2, 4.4, 4.5, 5.2)."""
import numpy as np
import pytest

from oracle import curvefit as cf
from oracle import lm
from oracle import structured as st
from tests.gpu_common import cuda_or_skip
from workloads import curvefit_problem

pytestmark = pytest.mark.gpu


def sorted_system(npoints, Kc, lam, seed=0):
    """The damped LM system at the start point, points sorted by segment (the row permutation)."""
    draw = curvefit_problem(npoints=npoints, Kc=Kc, seed_offset=seed)
    data, x0 = cf.make_data(draw)
    t, P = cf.unpack(x0, npoints)
    seg, _ = cf.segment(t, Kc)
    order = np.argsort(seg, kind="stable")
    data = data[order]
    x0 = cf.pack(t[order], P)
    Pb, f = lm.curvefit_system(x0, data, lam)
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
    assert rel(p, p_ref) <= 1e-12


def test_window_fp32_refined_matches_oracle():
    Pb, _ = sorted_system(4000, 128, 1e-3, seed=2)
    p_ref, _ = st.factor_and_solve(Pb, reduced_solver=st.banded_reduced_solver())
    p = run(Pb, "fp32_refined", refine_steps=2)
    assert rel(p, p_ref) <= 1e-5
