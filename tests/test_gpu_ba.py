"""GPU parity of the composed solve on the BA-shaped system (bundle adjustment, Sec. 6.2):
point blocks of 2 k_i x 3 (k_i observations) horizontally concatenated with the cameras' 9
columns each (Sec. 4.2), damped (Sec. 4.5), against the FP64 oracle."""
import numpy as np
import pytest

from oracle import structured as st
from tests.gpu_common import assert_close, cuda_or_skip
from workloads import ba_system

pytestmark = pytest.mark.gpu


def problem_from(d, dtype=np.float64):
    starts = np.concatenate([[0], np.cumsum(d["n"])])
    blocks = [np.asarray(b, dtype=np.float64) for b in d["blocks"]]
    coupled = [np.asarray(d["S"][starts[i]:starts[i + 1]], dtype=np.float64) for i in range(d["K"])]
    return st.BlockProblem(blocks=blocks, coupled=coupled, s=d["s"], b=np.asarray(d["b"], np.float64),
                           lam=d["lam"])


def run(d, precision, refine_steps):
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context, qrkit
    dt = np.float64 if precision == "fp64" else np.float32
    J = np.concatenate([np.asarray(b).T.reshape(-1) for b in d["blocks"]]).astype(dt)   # col-major
    S = np.asarray(d["S"]).T.reshape(-1).astype(dt)                                      # col-major
    b = np.asarray(d["b"]).astype(dt)
    ctx = Context(0, precision=precision)
    K, s = d["K"], d["s"]
    ctx.plan_blocks(d["n"], np.full(K, 3), qrkit.COUPLED_DENSE, shared_cols=s)
    ctx.factor(torch.from_numpy(J).cuda(), torch.from_numpy(S).cuda(), None, d["lam"])
    p = torch.empty(3 * K + s, device="cuda", dtype=ctx.dtype)
    ctx.solve(torch.from_numpy(b).cuda(), p, refine_steps=refine_steps)
    ctx.sync_status()
    out = p.cpu().numpy().astype(np.float64)
    ctx.close()
    return out


@pytest.mark.parametrize("P,C,s_pad,precision,steps,tol", [
    (300, 7, None, "fp64", 0, 1e-10),          # 63 camera columns, CUDA-core TSQR tiles
    (1500, 14, 128, "fp32_refined", 2, 1e-5),  # 126 camera columns padded to 128: column panels
    (800, 10, 96, "fp32_refined", 2, 1e-5),
    (1200, 30, 288, "fp32_refined", 2, 1e-5),  # 270 camera columns: nine panels of 32
])
def test_ba_system_matches_oracle(P, C, s_pad, precision, steps, tol):
    d = ba_system(P=P, C=C, s_pad=s_pad, dtype=np.float64 if precision == "fp64" else np.float32)
    p_ref, _ = st.factor_and_solve(problem_from(d))
    p = run(d, precision, steps)
    assert_close(p, p_ref, tol)
    # padding columns (zero in S) get a zero step
    if s_pad is not None:
        np.testing.assert_array_equal(p[3 * P + 9 * C:], 0.0)
