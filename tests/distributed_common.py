"""Inputs and a float64 stand-in of the local steps for the distributed dense-S solve tests."""
import numpy as np

from oracle import householder as hh
from oracle import structured as st
from workloads import block_angular_dense


def problem(K=40, s=6, seed=3):
    d = block_angular_dense(K=K, n=4, m=2, s=s, seed_offset=seed, scale_decades=1.0)
    return d


def part(d, lo, hi):
    """Blocks lo .. hi - 1 with their rows of S and b."""
    n = d["n"]
    blocks = [np.asarray(d["blocks"][i], dtype=np.float64) for i in range(lo, hi)]
    S = np.asarray(d["S"], dtype=np.float64)[lo * n:hi * n]
    b = np.asarray(d["b"], dtype=np.float64)[lo * n:hi * n]
    return blocks, S, b


class OracleOps:
    """The local steps of the driver computed by the float64 oracle (Secs. 4.1, 4.2, 4.5), on
    CPU tensors: lets the gloo test check the exchanges and the assembly on CPU."""

    def __init__(self, blocks, S, b, s):
        import torch
        self.torch = torch
        self.blocks, self.S, self.b, self.s = blocks, S, b, s
        n = blocks[0].shape[0]
        self.coupled = [S[i * n:(i + 1) * n] for i in range(len(blocks))]
        self.nb = sum(blk.shape[1] for blk in blocks)

    def column_sumsq(self, J, S):
        P = st.BlockProblem(blocks=self.blocks, coupled=self.coupled, s=self.s, b=self.b)
        A = st.assemble_J(P)
        return self.torch.from_numpy((A * A).sum(axis=0))

    def norms(self, sq):
        d = np.sqrt(sq.numpy())
        d[d == 0.0] = 1.0
        return self.torch.from_numpy(d)

    def factor(self, J, S, D, lam):
        P = st.BlockProblem(blocks=self.blocks, coupled=self.coupled, s=self.s, b=self.b, lam=lam,
                            D=D.numpy().copy())
        with np.errstate(divide="ignore", invalid="ignore"):   # the local triangle may be singular
            _, self.F = st.factor_and_solve(P)

    def summary(self, b):
        F = self.F
        R = self.torch.from_numpy(np.ascontiguousarray(F.reduced_factor.R.T).reshape(-1))
        qtb = self.torch.from_numpy(np.concatenate(F.c_blocks + [F.c_S]))
        return R, self.torch.from_numpy(F.c_S.copy()), qtb

    def merge(self, stack, rhs):
        A = stack.numpy().T          # (G s) x s
        return self.torch.from_numpy(hh.lstsq(A, rhs.numpy())[0])

    def finish(self, qtb, p_S):
        F = self.F
        ps = p_S.numpy()
        out = [hh.back_substitute(f.R[:f.R.shape[1]], c - R12 @ ps)
               for f, c, R12 in zip(F.block_factors, F.c_blocks, F.R12)]
        return self.torch.from_numpy(np.concatenate(out + [ps]))


def reference(d, lam):
    blocks, S, b = part(d, 0, d["K"])
    n = d["n"]
    P = st.BlockProblem(blocks=blocks, coupled=[S[i * n:(i + 1) * n] for i in range(d["K"])], s=d["s"], b=b,
                        lam=lam)
    return st.factor_and_solve(P)[0]
