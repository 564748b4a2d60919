"""A block-angular solve with a dense S whose blocks (and rows of S) are split over ranks, one GPU
each: the horizontal concatenation of Sec. 4.2 with the reduced shared block factored by TSQR
across GPUs (Sec. 2 QR of stacked triangles).

Every rank holds a contiguous range of blocks and the rows of S they own.  The steps:

  1. squared column sums of the local J (library); the shared columns' sums are added over the
     ranks (all-reduce), so that D = diag(J^T J)^(1/2) is the global column norm (Sec. 5.2);
  2. the local composed factorization of P_r [J_g; lambda^(1/2) D_g] (library), where only rank 0
     keeps the damping entries of the shared columns (the others pass zero there, so each
     shared damping row enters once);
  3. each rank's summary of its reduced shared block: the s x s triangle R_g and c_g (library);
     an all-gather brings every rank the stacked [R_1; .. ; R_G] and [c_1; .. ; c_G];
  4. the stack is solved once more by Householder QR (library, on every rank: the result is the
     same, and no broadcast is needed): p_S;
  5. every rank back-substitutes its own blocks with p_S (library).

The local steps go through an `ops` object (LibraryOps: the C-ABI on this rank's GPU) and the
exchanges through a `comm` object (TorchComm: torch.distributed, NCCL on GPUs), so the same driver
runs the library on GPUs and any other implementation of the local steps elsewhere.  This module
only moves data between those calls: the arithmetic is in the library's kernels.
"""
from __future__ import annotations


class TorchComm:
    """The two collectives of the driver over a torch.distributed process group."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world_size = dist.get_world_size(group)

    def all_reduce_sum(self, t):
        self.dist.all_reduce(t, group=self.group)
        return t

    def all_gather(self, t):
        import torch
        out = [torch.empty_like(t) for _ in range(self.world_size)]
        self.dist.all_gather(out, t.contiguous(), group=self.group)
        return out


class LibraryOps:
    """The local steps on this rank's GPU through the C-ABI (a Context planned for the local
    blocks with a dense S; device tensors in the context precision)."""

    def __init__(self, ctx, nb, s):
        self.ctx, self.nb, self.s = ctx, nb, s

    def column_sumsq(self, J, S):
        import torch
        sq = torch.empty(self.nb + self.s, dtype=torch.float64, device=self.ctx.device)
        self.ctx.column_sumsq(J, S, sq)
        return sq

    def norms(self, sq):
        import torch
        D = torch.empty(sq.numel(), dtype=self.ctx.dtype, device=self.ctx.device)
        self.ctx.norms_from_sumsq(sq, D)
        return D

    def factor(self, J, S, D, lam):
        self.ctx.factor(J, S, D, lam)

    def summary(self, b):
        import torch
        qtb = torch.empty(self.nb + self.s, dtype=self.ctx.dtype, device=self.ctx.device)
        self.ctx.apply_qt(b, qtb)
        R = torch.empty(self.s * self.s, dtype=self.ctx.dtype, device=self.ctx.device)
        self.ctx.reduced_r(R)
        return R, qtb[self.nb:].clone(), qtb

    def merge(self, stack, rhs):
        import torch
        x = torch.empty(self.s, dtype=self.ctx.dtype, device=self.ctx.device)
        self.ctx.dense_lstsq(stack, rhs, x)
        return x

    def finish(self, qtb, p_S):
        import torch
        p = torch.empty(self.nb + self.s, dtype=self.ctx.dtype, device=self.ctx.device)
        p[self.nb:].copy_(p_S)
        self.ctx.solve_blocks(qtb, p)
        return p


def tsqr_solve(comm, ops, J, S, b, lam, nb, s):
    """The damped solve of the global problem for this rank's blocks (see the module docstring).

    J, S, b: the local values (layouts of qrkit_factor / qrkit_apply_qt); nb: local block columns;
    s: shared columns.  Returns the local p: [block unknowns of this rank; p_S (the same on
    every rank)].
    """
    import torch
    sq = ops.column_sumsq(J, S)
    sq_S = comm.all_reduce_sum(sq[nb:].clone())
    sq = torch.cat([sq[:nb], sq_S])
    D = ops.norms(sq)
    if comm.rank != 0:   # the shared damping rows enter once, on rank 0
        D = D.clone()
        D[nb:] = 0
    ops.factor(J, S, D, lam)
    R, c, qtb = ops.summary(b)
    Rs = comm.all_gather(R)
    cs = comm.all_gather(c)
    # [R_1; ..; R_G] column-major: each R_g is s x s column-major, i.e. (s, s) row-major by column
    stack = torch.cat([Rg.reshape(s, s) for Rg in Rs], dim=1).contiguous()
    rhs = torch.cat(cs).contiguous()
    p_S = ops.merge(stack, rhs)
    return ops.finish(qtb, p_S)
