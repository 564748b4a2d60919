"""GPU parity of the LM iteration (Sec. 2, Backtrack LM of Sec. 5.2) on the curve-fit model:
one step and short runs against the float64 oracle, single and batched problems, with and
without CUDA-graph replay."""
import numpy as np
import pytest

from oracle import curvefit as cf
from oracle import lm
from tests.gpu_common import cuda_or_skip
from workloads import curvefit_problem

pytestmark = pytest.mark.gpu


def problem(npoints, Kc, seed):
    draw = curvefit_problem(npoints=npoints, Kc=Kc, seed_offset=seed)
    data, x0 = cf.make_data(draw)
    return data, x0


def gpu_ctx(precision):
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context
    stream = torch.cuda.Stream()
    return torch, Context(0, stream=stream, precision=precision)


def pack_batch(problems):
    """x and data of several problems in the library's layout (all t, then all control points)."""
    ts, Ps, datas = [], [], []
    for data, x0 in problems:
        t, P = cf.unpack(x0, data.shape[0])
        ts.append(t)
        Ps.append(P.reshape(-1))
        datas.append(data)
    return np.concatenate(ts + Ps), np.concatenate(datas)


def unpack_batch(x, problems):
    npts = [d.shape[0] for d, _ in problems]
    kcs = [(x0.shape[0] - d.shape[0]) // 2 for d, x0 in problems]
    NP = sum(npts)
    out, p0, c0 = [], 0, NP
    for n, kc in zip(npts, kcs):
        out.append(np.concatenate([x[p0:p0 + n], x[c0:c0 + 2 * kc]]))
        p0 += n
        c0 += 2 * kc
    return out


def run_steps(precision, problems, lams, steps, refine=2):
    torch, ctx = gpu_ctx(precision)
    xh, dh = pack_batch(problems)
    with torch.cuda.stream(ctx.stream):
        data = torch.from_numpy(dh).cuda()
        x = torch.from_numpy(xh).cuda()
    ctx.lm_plan([d.shape[0] for d, _ in problems], [(x0.shape[0] - d.shape[0]) // 2 for d, x0 in problems], data)
    st = ctx.lm_states(lams)
    hist = []
    for _ in range(steps):
        ctx.lm_step(x, st, refine_steps=refine)
        hist.append([(s.cost, s.cost_new, s.pred, s.rho, s.accepted, s.lambda_, s.nu) for s in st])
    ctx.stream.synchronize()
    xs = unpack_batch(x.cpu().numpy(), problems)
    ctx.close()
    return xs, hist


def oracle_steps(data, x0, lam, steps, round32=False):
    s = lm.LMState(x=np.array(x0), lam=lam)
    hist = []
    for _ in range(steps):
        s, acc, c, cn = lm.lm_step(s, data, round32=round32)
        hist.append((c, cn, s.history[-1][2], acc, s.lam, s.nu))
    return s.x, hist


def test_lm_step_fp64_matches_oracle():
    data, x0 = problem(600, 16, 11)
    xs, hist = run_steps("fp64", [(data, x0)], 1e-3, 1, refine=0)
    xo, ho = oracle_steps(data, x0, 1e-3, 1)
    c, cn, pred, rho, acc, lam, nu = hist[0][0]
    oc, ocn, orho, oacc, olam, onu = ho[0]
    assert c == pytest.approx(oc, rel=1e-12)
    assert cn == pytest.approx(ocn, rel=1e-9)
    assert rho == pytest.approx(orho, rel=1e-7, abs=1e-9)
    assert bool(acc) == oacc
    assert lam == pytest.approx(olam, rel=1e-7) and nu == onu
    assert np.linalg.norm(xs[0] - xo) <= 1e-10 * np.linalg.norm(xo)


def test_lm_step_fp32_refined_matches_rounded_oracle():
    data, x0 = problem(1500, 32, 12)
    xs, hist = run_steps("fp32_refined", [(data, x0)], 1e-2, 1, refine=2)
    s = lm.LMState(x=np.array(x0), lam=1e-2)
    s, acc, c, cn = lm.lm_step(s, data, round32=True)
    assert hist[0][0][0] == pytest.approx(c, rel=1e-12)          # cost at x: double on both sides
    p_gpu = xs[0] - x0
    assert acc and hist[0][0][4] == 1
    assert np.linalg.norm(p_gpu - s.last_p) <= 1e-5 * np.linalg.norm(s.last_p)
    assert hist[0][0][1] == pytest.approx(cn, rel=1e-6)


def test_lm_batched_problems_fp64():
    probs = [problem(300, 12, 21), problem(800, 20, 22), problem(450, 8, 23)]
    lams = [1e-3, 1e-1, 10.0]
    xs, hist = run_steps("fp64", probs, lams, 3, refine=0)
    for k, ((data, x0), lam0) in enumerate(zip(probs, lams)):
        xo, ho = oracle_steps(data, x0, lam0, 3)
        for it in range(3):
            c, cn, pred, rho, acc, lam, nu = hist[it][k]
            oc, ocn, orho, oacc, olam, onu = ho[it]
            assert c == pytest.approx(oc, rel=1e-10)
            assert bool(acc) == oacc
            assert lam == pytest.approx(olam, rel=1e-6)
        assert np.linalg.norm(xs[k] - xo) <= 1e-9 * np.linalg.norm(xo)


@pytest.mark.parametrize("use_graph", [False, True])
def test_lm_run_matches_oracle_run(use_graph):
    torch, ctx = gpu_ctx("fp64")
    data, x0 = problem(400, 12, 31)
    with torch.cuda.stream(ctx.stream):
        d = torch.from_numpy(data).cuda()
        x = torch.from_numpy(x0.copy()).cuda()
    ctx.lm_plan([400], [12], d)
    st = ctx.lm_states(1e-3)
    ctx.lm_run(x, st, max_iter=40, ftol=1e-10, refine_steps=0, use_graph=use_graph)
    ctx.stream.synchronize()
    xg = x.cpu().numpy()
    so = lm.lm_run(x0, data, lam0=1e-3, max_iter=40, ftol=1e-10)
    assert st[0].iteration == so.it
    assert st[0].lambda_ == pytest.approx(so.lam, rel=1e-6)
    assert np.linalg.norm(xg - so.x) <= 1e-8 * np.linalg.norm(so.x)
    ctx.close()


def test_lm_graph_replay_equals_eager_fp32():
    torch = cuda_or_skip()
    probs = [problem(700, 16, 41), problem(300, 10, 42)]
    xh, dh = pack_batch(probs)
    outs = []
    for use_graph in (False, True):
        _, ctx = gpu_ctx("fp32_refined")
        with torch.cuda.stream(ctx.stream):
            d = torch.from_numpy(dh).cuda()
            x = torch.from_numpy(xh.copy()).cuda()
        ctx.lm_plan([700, 300], [16, 10], d)
        st = ctx.lm_states([1e-3, 1e-2])
        ctx.lm_run(x, st, max_iter=16, ftol=0.0, refine_steps=1, use_graph=use_graph)
        ctx.stream.synchronize()
        outs.append((x.cpu().numpy(), [(s.iteration, s.lambda_, s.cost) for s in st]))
        ctx.close()
    (xa, sa), (xb, sb) = outs
    assert [s[0] for s in sa] == [s[0] for s in sb]
    assert np.linalg.norm(xa - xb) <= 1e-6 * np.linalg.norm(xa)
    for a, b in zip(sa, sb):
        assert a[2] == pytest.approx(b[2], rel=1e-6)
