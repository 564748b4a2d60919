"""GPU parity of the composed solve on the ellipse-fit system (the surface fitting benchmark
of Sec. 6: 2 x 1 latent blocks horizontally concatenated with 5 dense shared columns,
Sec. 4.1 / 4.2 / 4.5) against the FP64 oracle."""
import numpy as np
import pytest

from oracle import structured as st
from tests.gpu_common import assert_close
from tests.test_gpu_composed import problem_from, rel, run
from workloads import ellipse_system

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,precision,steps,tol", [
    (500, "fp64", 0, 1e-12),
    (2000, "fp32_refined", 2, 1e-5),
    (6000, "fp64", 0, 1e-11),         # a reduced block of 12,005 rows
])
def test_ellipse_system_matches_oracle(N, precision, steps, tol):
    d = ellipse_system(N=N, dtype=np.float64 if precision == "fp64" else np.float32)
    p_ref, _ = st.factor_and_solve(problem_from(d))
    out = run(d, precision, refine_steps=steps)
    assert_close(out["p"], p_ref, tol)
    if precision == "fp32_refined":
        assert rel(out["p"], p_ref) < rel(out["p_norefine"], p_ref)


def test_ellipse_system_full_size_optimality():
    """N = 500,000 points (the largest size of the paper's sweep), FP64: the solution satisfies
    the normal equations J^T (b - J p) = lambda D^2 p, D = column norms, to rounding."""
    N = 500_000
    d = ellipse_system(N=N)
    out = run(d, "fp64", refine_steps=0)
    p = out["p"]
    A = d["blocks"][:, :, 0]                  # (N, 2)
    S = d["S"]                                # (2N, 5)
    r = d["b"] - (A * p[:N, None]).reshape(-1) - S @ p[N:]
    Dt2 = np.sum(A * A, axis=1)
    Ds2 = np.sum(S * S, axis=0)
    g = np.concatenate([np.sum(A * r.reshape(N, 2), axis=1) - d["lam"] * Dt2 * p[:N],
                        S.T @ r - d["lam"] * Ds2 * p[N:]])
    nJ = np.sqrt(np.sum(A * A) + np.sum(S * S))
    assert np.linalg.norm(g) / (nJ * nJ * np.linalg.norm(p) + nJ * np.linalg.norm(d["b"])) <= 1e-13
