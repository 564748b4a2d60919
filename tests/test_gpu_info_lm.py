"""The result record (qrkit_get_info) and an LM loop over a model of the caller's own
(qrkit_lm_trial + qrkit_nielsen_update), against the oracle (Eq. 1, Eq. 2, Sec. 2, Sec. 5.2)."""
import numpy as np
import pytest

from oracle import curvefit as cf
from oracle import lm
from oracle import structured as st
from tests.gpu_common import cuda_or_skip
from workloads import batched_blocks, curvefit_problem

pytestmark = pytest.mark.gpu


def host_norms(d, p, lam=0.0, Dv=None):
    r2 = g2 = 0.0
    for i in range(d["K"]):
        n, m = int(d["n"][i]), int(d["m"][i])
        v0, r0, c0 = int(d["val_off"][i]), int(d["row_off"][i]), int(d["col_off"][i])
        A = np.asarray(d["vals"][v0:v0 + n * m], dtype=np.float64).reshape(m, n).T
        x = np.asarray(p[c0:c0 + m], dtype=np.float64)
        r = np.asarray(d["b"][r0:r0 + n], dtype=np.float64) - A @ x
        Di = np.linalg.norm(A, axis=0) if Dv is None else Dv[c0:c0 + m]
        g = A.T @ r - lam * Di * Di * x
        r2 += r @ r
        g2 += g @ g
    return np.sqrt(r2), np.sqrt(g2)


@pytest.mark.parametrize("precision", ["fp64", "fp32_refined"])
def test_info_of_a_block_solve(precision):
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context
    dt = np.float64 if precision == "fp64" else np.float32
    d = batched_blocks(K=20000, seed_offset=51, dtype=dt)
    ctx = Context(0, precision=precision)
    ctx.plan_blocks(d["n"], d["m"])
    J = torch.from_numpy(d["vals"]).cuda()
    b = torch.from_numpy(d["b"]).cuda()
    p = torch.empty(int(d["col_off"][-1]), device="cuda", dtype=ctx.dtype)
    ctx.factor_solve(J, b, p, None, refine_steps=2)
    info = ctx.info(J, b, p)
    ctx.close()
    rn, gn = host_norms(d, p.cpu().numpy())
    assert info["residual_norm"] == pytest.approx(rn, rel=1e-12)
    assert info["optimality_norm"] == pytest.approx(gn, rel=1e-9, abs=1e-12 * info["optimality_scale"])
    if precision == "fp64":
        assert info["optimality_norm"] <= 1e-14 * info["optimality_scale"]
        assert info["refined_blocks"] == -1 and info["refine_steps_max"] == -1
    else:
        assert info["optimality_norm"] <= 1e-7 * info["optimality_scale"]
        assert 0 < info["refined_blocks"] < d["K"] // 2
        assert info["refine_steps_max"] in (1, 2)


def test_lm_loop_over_a_caller_model_matches_the_oracle():
    """A curve fit whose residual and Jacobian the caller evaluates (here with the oracle's model
    code, as a user's own model would be): J, S and b go to qrkit_lm_trial, the gain ratio is
    formed by the caller and the damping updated by qrkit_nielsen_update.  In FP64 the run
    follows the oracle's LM (oracle/lm.py) step for step."""
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context, qrkit
    draw = curvefit_problem(npoints=300, Kc=14, seed_offset=4)
    data, x0 = cf.make_data(draw)
    ref = lm.lm_run(x0, data, lam0=1e-3, max_iter=12, ftol=0.0)
    ctx = Context(0, precision="fp64")
    x = np.array(x0)
    lam, nu = 1e-3, 2.0
    hist = []
    for it in range(len(ref.history)):
        P, f = lm.curvefit_system(x, data, lam)
        if it == 0:
            ctx.plan_blocks(np.full(P.K, 2), np.full(P.K, 1), qrkit.COUPLED_WINDOW, shared_cols=P.s, window=8,
                            window_start=np.asarray(P.start, dtype=np.int32))
        else:
            ctx.set_window_start(torch.from_numpy(np.asarray(P.start, dtype=np.int32)).cuda())
        J = torch.from_numpy(np.concatenate([blk.T.reshape(-1) for blk in P.blocks])).cuda()
        S = torch.from_numpy(np.concatenate([c.T.reshape(-1) for c in P.coupled])).cuda()
        b = torch.from_numpy(np.asarray(P.b)).cuda()
        p = torch.empty(P.N, device="cuda", dtype=torch.float64)
        pred = ctx.lm_trial(J, S, b, p, None, lam, refine_steps=0)
        pv = p.cpu().numpy()
        assert pred == pytest.approx(lm.predicted_decrease(P, pv), rel=1e-10)
        cost = 0.5 * float(f @ f)
        fn = cf.residual(x + pv, data)
        cost_new = 0.5 * float(fn @ fn)
        rho = (cost - cost_new) / pred if pred > 0 else -1.0
        hist.append((cost, lam, rho))
        lam, nu, acc = qrkit.nielsen_update(rho, lam, nu)
        assert acc == ref.history[it][3], it
        if acc:
            x = x + pv
    ctx.close()
    for (c, l, r), (rc, rl, rr, _) in zip(hist, ref.history):
        assert c == pytest.approx(rc, rel=1e-10) and l == pytest.approx(rl, rel=1e-10)
    assert 0.5 * float(cf.residual(x, data) @ cf.residual(x, data)) == pytest.approx(ref.cost, rel=1e-9)
