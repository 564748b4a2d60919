"""GPU parity of the fused batched block QR solve (Sec. 4.1) against the FP64 oracle."""
import numpy as np
import pytest

from oracle import householder as hh
from tests.gpu_common import (U32, U64, assert_blocks_within, block_errors, block_kappa, cuda_or_skip,
                              optimality_all, oracle_block)
from workloads import batched_blocks

pytestmark = pytest.mark.gpu


def _at_offset(torch, host, offset, dev, dt):
    """A device copy of host that starts `offset` elements into its allocation."""
    buf = torch.zeros(len(host) + offset, device=dev, dtype=dt)
    view = buf[offset:]
    view.copy_(torch.from_numpy(np.asarray(host)).to(dev, dt))
    return view


def run(d, precision, refine_steps=1, with_qtb=True, tuning=None, offset=0, refinement=None):
    """offset: J, b and Q^T b start that many elements into their allocations (their 16-byte
    alignment then differs from the factor workspace's); refinement: (select, residual) for
    qrkit_set_refinement."""
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context
    ctx = Context(0, precision=precision)
    dt = ctx.dtype
    dev = ctx.device
    J = _at_offset(torch, d["vals"], offset, dev, dt)
    b = _at_offset(torch, d["b"], offset, dev, dt)
    K = d["K"]
    ncols = int(d["col_off"][-1])
    p = torch.empty(ncols, device=dev, dtype=dt)
    qtb = _at_offset(torch, np.zeros(int(d["row_off"][-1])), offset, dev, dt) if with_qtb else None
    ctx.plan_blocks(d["n"], d["m"])
    if tuning is not None:
        ctx.apply_tuning(tuning)
    if refinement is not None:
        ctx.set_refinement(*refinement)
    ctx.factor_solve(J, b, p, qtb, refine_steps=refine_steps)
    launches = ctx.launch_count
    F = torch.empty_like(J)
    tau = torch.empty(ncols, device=dev, dtype=dt)
    ctx.get_factor(F, tau)
    ctx.sync_status()
    out = dict(p=p.cpu().numpy().astype(np.float64), F=F.cpu().numpy().astype(np.float64),
               tau=tau.cpu().numpy().astype(np.float64),
               qtb=None if qtb is None else qtb.cpu().numpy().astype(np.float64),
               launches=launches)
    ctx.close()
    return out


def gpu_block(d, out, i):
    n, m = int(d["n"][i]), int(d["m"][i])
    v0, r0, c0 = int(d["val_off"][i]), int(d["row_off"][i]), int(d["col_off"][i])
    F = out["F"][v0:v0 + n * m].reshape(m, n).T
    R = np.triu(F[:m, :])
    V = np.tril(F, -1)
    V[np.arange(m), np.arange(m)] = 1.0
    return dict(R=R, V=V, tau=out["tau"][c0:c0 + m], x=out["p"][c0:c0 + m],
                qtb=None if out["qtb"] is None else out["qtb"][r0:r0 + n])


# Per precision: the solution target (per block), the unit roundoff of the bound that admits
# blocks too ill-conditioned for it, the R / tau / Q^T b tolerance.  FP32 refined and FP64 must
# meet the target on every block unless even the FP64 oracle cannot (u = 2^-53); plain FP32
# must stay within the float forward-error bound of each block.
MODES = {"fp64": (1e-12, U64, 1e-13), "fp32_refined": (1e-5, U64, 2e-6), "fp32": (1e-6, U32, 2e-6)}


def check_blocks(d, out, idx, precision):
    x_tol, u_bound, r_tol = MODES[precision]
    for i in idx:
        x, f, qtb, A, b = oracle_block(d, i)
        g = gpu_block(d, out, i)
        nA = np.linalg.norm(A)
        # R equals the oracle's R (same reflector sign convention); compare with row signs
        # normalised so that a sign flip from a near-zero x0 is not reported
        np.testing.assert_allclose(hh.normalise_row_signs(g["R"]), hh.normalise_row_signs(f.R),
                                   atol=r_tol * nA, err_msg=f"R of block {i}")
        same = np.sign(np.diag(g["R"])) == np.sign(np.diag(f.R))
        np.testing.assert_allclose(g["tau"][same], f.tau[same], atol=r_tol * 10)
        if g["qtb"] is not None:
            m = A.shape[1]
            s = np.where(np.diag(g["R"]) * np.diag(f.R) < 0, -1.0, 1.0)
            np.testing.assert_allclose(g["qtb"][:m] * s, qtb[:m], atol=r_tol * (np.linalg.norm(b) + 1))
            np.testing.assert_allclose(np.linalg.norm(g["qtb"][m:]), np.linalg.norm(qtb[m:]),
                                       atol=r_tol * (np.linalg.norm(b) + 1))
    return assert_blocks_within(d, out["p"], np.asarray(list(idx)), x_tol, u_bound, c=8.0 if u_bound == U32 else None,
                                what=f"{precision}: ")


TILES = {"fp64": "budget 256 1536 512 256 2048", "fp32": "budget 256 3072 1024 512 4096"}


@pytest.mark.parametrize("mapping", ["tasks", "tasks 32 4 0", "tasks 64 8 1", "tiles"])
@pytest.mark.parametrize("precision", ["fp64", "fp32_refined", "fp32"])
def test_blocks_parity_small(precision, mapping):
    """3000 blocks: several supertiles / tiles, ragged warp tasks and a ragged last tile;
    every block checked.  Mappings: the default shape-uniform warp tasks, tasks over
    32-block supertiles in supertile order with 4 warps per CTA, tasks over 64-block
    supertiles in shape-key order, and tiles of consecutive blocks."""
    d = batched_blocks(K=3000, seed_offset=7, dtype=np.float64 if precision == "fp64" else np.float32)
    tuning = {"tasks": None, "tiles": TILES["fp64" if precision == "fp64" else "fp32"]}.get(mapping, mapping)
    out = run(d, precision, tuning=tuning, refine_steps=2)
    check_blocks(d, out, range(3000), precision)
    # one fused launch (FP32-refined warp tasks: one per key class, blocks of <= 4 and of 5-8
    # columns, both present here); with refinement one more refines the blocks it selected
    factor = 2 if (precision == "fp32_refined" and mapping != "tiles") else 1
    assert out["launches"] == factor + (1 if precision == "fp32_refined" else 0)


@pytest.mark.parametrize("offset", [1, 3])
@pytest.mark.parametrize("precision", ["fp64", "fp32_refined"])
def test_blocks_unaligned_buffers(precision, offset):
    """J, b and Q^T b that start off the factor workspace's 16-byte alignment: the blocks at
    the buffers' ends are loaded with plain loads, the factor and Q^T b leave with plain
    stores."""
    d = batched_blocks(K=2000, seed_offset=12, dtype=np.float64 if precision == "fp64" else np.float32)
    out = run(d, precision, offset=offset, refine_steps=2)
    check_blocks(d, out, range(2000), precision)


def test_blocks_refinement_reduces_error():
    d = batched_blocks(K=4000, seed_offset=8)
    e = []
    for steps in (0, 1, 2):
        out = run(d, "fp32_refined", refine_steps=steps, with_qtb=False)
        num = den = 0.0
        worst = 0.0
        for i in range(4000):
            x = oracle_block(d, i)[0]
            c0, m = int(d["col_off"][i]), int(d["m"][i])
            err = out["p"][c0:c0 + m] - x
            num += float(err @ err)
            den += float(x @ x)
            worst = max(worst, float(np.linalg.norm(err) / np.linalg.norm(x)))
        e.append((np.sqrt(num / den), worst))
    assert e[1][0] < e[0][0] and e[1][1] < e[0][1]
    assert e[1][1] < 1e-5
    assert e[2][1] <= e[1][1] * 1.5 + 1e-7


@pytest.mark.parametrize("shape", [(1, 1), (2, 2), (16, 8), (16, 1), (8, 8), (5, 3)])
def test_blocks_edge_shapes(shape):
    n, m = shape
    g = np.random.default_rng(n * 31 + m)
    K = 700
    nn = np.full(K, n, dtype=np.uint8)
    mm = np.full(K, m, dtype=np.uint8)
    vals = g.standard_normal(K * n * m)
    b = g.standard_normal(K * n)
    d = dict(n=nn, m=mm, vals=vals, b=b, K=K,
             val_off=np.arange(K + 1, dtype=np.int64) * n * m,
             row_off=np.arange(K + 1, dtype=np.int64) * n,
             col_off=np.arange(K + 1, dtype=np.int64) * m)
    out = run(d, "fp64")
    check_blocks(d, out, range(K), "fp64")


def test_blocks_single_block_and_status():
    d = batched_blocks(K=1, seed_offset=3, dtype=np.float64)
    out = run(d, "fp64")
    check_blocks(d, out, [0], "fp64")


def test_singular_block_reports_status():
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context, QRKitError
    ctx = Context(0, precision="fp64")
    n = np.array([3, 3], dtype=np.uint8)
    m = np.array([2, 2], dtype=np.uint8)
    vals = np.array([1, 2, 3, 0, 0, 0, 1, 0, 0, 0, 1, 0], dtype=np.float64)  # block 0 col 1 zero
    J = torch.tensor(vals, device="cuda", dtype=torch.float64)
    b = torch.ones(6, device="cuda", dtype=torch.float64)
    p = torch.empty(4, device="cuda", dtype=torch.float64)
    ctx.plan_blocks(n, m)
    ctx.factor_solve(J, b, p, refine_steps=0)
    with pytest.raises(QRKitError) as e:
        ctx.sync_status()
    assert e.value.status == 4
    ctx.sync_status()   # the status word is cleared after it is read
    ctx.close()


def test_plan_rejects_oversized_blocks():
    cuda_or_skip()
    from paper_1802_03773_gb300 import Context, QRKitError
    ctx = Context(0, precision="fp32")
    with pytest.raises(QRKitError) as e:
        ctx.plan_blocks(np.array([17], dtype=np.uint8), np.array([2], dtype=np.uint8))
    assert e.value.status == 8
    ctx.close()


def test_blocks_full_size_every_block():
    """The 1,000,000-block workload in the launch configuration bench.py times (FP32 refined,
    two refinement steps): every block within 1e-5 of the oracle's FP64 solution, every block
    passes the optimality identity, and 3000 sampled blocks match the oracle's R, tau too."""
    d = batched_blocks(K=1_000_000)
    out = run(d, "fp32_refined", with_qtb=False, refine_steps=2)
    assert optimality_all(d, out["p"]) < 1e-6
    worst, blk = assert_blocks_within(d, out["p"], None, 1e-5, U64)
    print(f"1M blocks: worst block {blk} at {worst:.2e}")
    idx = np.random.default_rng(0).choice(1_000_000, 3000, replace=False)
    check_blocks(d, out, idx, "fp32_refined")


@pytest.mark.parametrize("residual", ["dot2", "fp64"])
def test_blocks_ill_conditioned_refined(residual):
    """Every block of the 1M workload with kappa > 1e3 (466 of them, kappa up to 7.4e5, where
    u kappa^2 > 1 for about a hundred): FP32 refined with two steps of the augmented-system
    refinement meets 1e-5 against the oracle on each, with either residual precision."""
    d = batched_blocks(K=1_000_000)
    ill = np.nonzero(block_kappa(d) > 1e3)[0]
    assert ill.size > 400
    out = run(d, "fp32_refined", with_qtb=False, refine_steps=2, refinement=(2e-6, residual))
    err, _ = block_errors(d, out["p"], ill)
    w = int(np.argmax(err))
    assert err[w] <= 1e-5, f"block {int(ill[w])}: error {err[w]:.3e}"
    print(f"{residual}: {ill.size} blocks with kappa > 1e3, worst error {err[w]:.2e}")


def test_blocks_select_everything():
    """select = 0 refines every block (no block is left to the a-priori estimate): every block
    meets 1e-5 against the oracle."""
    d = batched_blocks(K=200_000, seed_offset=5)
    out = run(d, "fp32_refined", with_qtb=False, refine_steps=2, refinement=(0.0, "dot2"))
    assert_blocks_within(d, out["p"], None, 1e-5, U64)
