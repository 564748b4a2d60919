"""Levenberg-Marquardt with the Nielsen damping rule, float64 (test infrastructure only).

Follows Sec. 2 (LM for F(x) = sum of squares, J the Jacobian of f, b = -f) and the
"Backtrack" variant of Sec. 5.2: one QR per iteration of P_r [J; lambda^(1/2) D] with
D = diag(J^T J)^(1/2), damping controlled directly (the paper adapts Lourakis' scheme).

Readings (the paper prints no lambda formula, stopping rule or cost scale):
  * cost = 1/2 ||f||^2 (the paper's F has an inconsistent 1/2).
  * gain ratio rho = (cost(x) - cost(x + p)) / (1/2 p^T (lambda D^2 p + J^T b)).
  * Nielsen rule: accept if rho > 0, then lambda *= max(1/3, 1 - (2 rho - 1)^3), nu = 2;
    reject: lambda *= nu, nu *= 2.
  * stop: accepted step with relative cost decrease < ftol, or ||J^T f||_inf <= gtol,
    or lambda > 1e16, or max_iter iterations.
Pins (tests/test_oracle_lm.py): closed-form Nielsen values, monotone accepted costs,
convergence on a problem with a known exact minimiser, determinism.  predicted_decrease
(tests/test_oracle_damping_pins.py): equals L(0) - L(p*) of the undamped linear model
L(p) = 1/2 ||b - J p||^2 at the damped minimiser, computed from J p alone; the gain ratio of
a residual that is linear in x is exactly 1; a dropped 1/2, lambda D for lambda D^2 and a
wrong sign of J^T b fail.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import curvefit
from . import structured


def nielsen(lam, nu, rho):
    """Returns (lam, nu, accepted) after a step with gain ratio rho."""
    if rho > 0.0:
        return lam * max(1.0 / 3.0, 1.0 - (2.0 * rho - 1.0) ** 3), 2.0, True
    return lam * nu, nu * 2.0, False


def curvefit_system(x, data, lam, round32=False):
    """BlockProblem of the damped LM system at x (b = -f).

    round32: J, S and b rounded once to float32 (the system a float factorization is given);
    the oracle still solves it in float64.  D then follows from the rounded J.
    """
    npts = data.shape[0]
    f = curvefit.residual(x, data)
    blocks, coupled, start = curvefit.jacobian_parts(x, data)
    b = -f
    if round32:
        blocks = blocks.astype(np.float32).astype(np.float64)
        coupled = coupled.astype(np.float32).astype(np.float64)
        b = b.astype(np.float32).astype(np.float64)
    Kc = (x.shape[0] - npts) // 2
    P = structured.BlockProblem(blocks=list(blocks), coupled=list(coupled), start=start,
                                s=2 * Kc, b=b, lam=lam)
    return P, f


def solve_system(P, banded_reduced=True):
    solver = structured.banded_reduced_solver() if banded_reduced else None
    p, _ = structured.factor_and_solve(P, reduced_solver=solver)
    return p


def predicted_decrease(P, p, f=None):
    """1/2 p^T (lambda D^2 p + J^T b) with the system's b (= -f) (the model decrease, Sec. 2)."""
    D = structured.damping(P)
    b = np.asarray(P.b, dtype=np.float64) if f is None else -f
    J = structured.assemble_J(P) if P.M * P.N <= 4_000_000 else None
    if J is not None:
        jtb = J.T @ b
    else:
        jtb = _jt_vec(P, b)
    return 0.5 * float(np.dot(p, P.lam * D * D * p + jtb))


def _jt_vec(P, r):
    co, ro = P.col_offsets(), P.row_offsets()
    nb = P.n_block_cols
    out = np.zeros(P.N)
    for i, blk in enumerate(P.blocks):
        ri = r[ro[i]:ro[i + 1]]
        out[co[i]:co[i + 1]] += blk.T @ ri
        if P.coupled is not None and P.s > 0:
            w = P.coupled[i].shape[1]
            st = 0 if P.start is None else int(P.start[i])
            out[nb + st:nb + st + w] += P.coupled[i].T @ ri
    return out


@dataclass
class LMState:
    x: np.ndarray
    lam: float = 1e-3
    nu: float = 2.0
    cost: float = float("nan")
    it: int = 0
    history: list = field(default_factory=list)   # (cost, lam, rho, accepted)
    last_p: np.ndarray = None


def lm_step(state: LMState, data, banded_reduced=True, round32=False):
    P, f = curvefit_system(state.x, data, state.lam, round32)
    cost = 0.5 * float(np.dot(f, f))
    p = solve_system(P, banded_reduced)
    state.last_p = p
    x_new = state.x + p
    f_new = curvefit.residual(x_new, data)
    cost_new = 0.5 * float(np.dot(f_new, f_new))
    pred = predicted_decrease(P, p)
    rho = (cost - cost_new) / pred if pred > 0 else -1.0
    lam, nu, acc = nielsen(state.lam, state.nu, rho)
    state.history.append((cost, state.lam, rho, acc))
    if acc:
        state.x = x_new
        state.cost = cost_new
    else:
        state.cost = cost
    state.lam, state.nu = lam, nu
    state.it += 1
    return state, acc, cost, cost_new


def lm_run(x0, data, lam0=1e-3, max_iter=200, ftol=1e-12, banded_reduced=True):
    st = LMState(x=np.array(x0, dtype=np.float64), lam=lam0)
    for _ in range(max_iter):
        st, acc, c_old, c_new = lm_step(st, data, banded_reduced)
        if acc and (c_old - c_new) <= ftol * c_old:
            break
        if st.lam > 1e16:
            break
    return st
