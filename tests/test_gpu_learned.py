"""GPU parity of the damping-policy MLP kernels (forward, backward, Adam, in-kernel inference)
against the float64 oracle evaluated with the same bfloat16-rounded weights, and the A/B
comparison of the trained policy with Nielsen's rule on held-out curve-fit problems."""
import numpy as np
import pytest

from oracle import curvefit as cf
from oracle import mlp
from tests.gpu_common import cuda_or_skip
from workloads import curvefit_problem, mlp_init

pytestmark = pytest.mark.gpu


def ctx_with(params):
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context
    ctx = Context(0, precision="fp32")
    ctx.mlp_init(params)
    return torch, ctx


def samples(n, seed):
    g = np.random.default_rng(seed)
    X = g.standard_normal((n, mlp.F)).astype(np.float32)
    y = g.integers(0, mlp.C, size=n).astype(np.int32)
    return X, y


def test_mlp_forward_and_gradient_match_oracle():
    theta = mlp_init(1)
    torch, ctx = ctx_with(theta)
    X, y = samples(100, 2)        # several 32-sample tiles and a ragged last one
    tX, ty = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    logits = torch.empty((100, mlp.C), dtype=torch.float32, device="cuda")
    ctx.mlp_forward(tX, logits)
    grad = torch.empty(mlp.P, dtype=torch.float32, device="cuda")
    loss = ctx.mlp_train_step(tX, ty, 0.0, grad=grad)
    p = mlp.working_weights(theta)
    z, _ = mlp.forward(p, X.astype(np.float64))
    np.testing.assert_allclose(logits.cpu().numpy(), z, rtol=1e-5, atol=1e-5)
    ref_loss, ref_g = mlp.loss_and_grad(p, X.astype(np.float64), y)
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    g = grad.cpu().numpy().astype(np.float64)
    gr = mlp.flatten(ref_g)
    assert np.linalg.norm(g - gr) <= 1e-5 * np.linalg.norm(gr)
    ctx.close()


def test_mlp_adam_steps_match_oracle():
    theta = mlp_init(3)
    torch, ctx = ctx_with(theta)
    X, y = samples(64, 4)
    tX, ty = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    th = theta.astype(np.float64)
    m = np.zeros(mlp.P)
    v = np.zeros(mlp.P)
    for t in range(1, 4):
        ctx.mlp_train_step(tX, ty, 1e-2)
        _, gr = mlp.loss_and_grad(mlp.working_weights(th.astype(np.float32)), X.astype(np.float64), y)
        th, m, v = mlp.adam_step(th, mlp.flatten(gr), m, v, t, lr=1e-2)
    got = ctx.mlp_params().astype(np.float64)
    np.testing.assert_allclose(got, th, atol=2e-5)
    ctx.close()


def problems(specs):
    out = []
    for n, kc, sd in specs:
        d, x0 = cf.make_data(curvefit_problem(npoints=n, Kc=kc, seed_offset=sd))
        out.append((d, x0))
    return out


def test_policy_inference_inside_lm_step_matches_oracle():
    """With the policy on, the lambda after an accepted step is lambda times the multiplier of
    the oracle's argmax on the features the step reports."""
    torch = cuda_or_skip()
    from paper_1802_03773_gb300 import Context, learned
    from paper_1802_03773_gb300.qrkit import MLP_MULTIPLIERS
    theta = mlp_init(5)
    b = learned.Batch(problems([(300, 12, 51), (500, 16, 52), (200, 8, 53)]))
    ctx = Context(0, precision="fp64")
    data = torch.from_numpy(b.data).cuda()
    x = torch.from_numpy(b.x0).cuda()
    ctx.lm_plan(b.npts, b.kcs, data)
    ctx.mlp_init(theta)
    ctx.lm_set_policy(True)
    st = ctx.lm_states([1e-3, 1e-2, 1e-1])
    feats = torch.empty((3, 16), dtype=torch.float32, device="cuda")
    for _ in range(3):
        lam_used = [s.lambda_ for s in st]
        ctx.lm_step(x, st, refine_steps=0)
        ctx.lm_features(feats)
        f = feats.cpu().numpy().astype(np.float64)
        z, _ = mlp.forward(mlp.working_weights(theta), f)
        for k, s in enumerate(st):
            if s.accepted:
                assert s.lambda_ == pytest.approx(lam_used[k] * MLP_MULTIPLIERS[int(np.argmax(z[k]))], rel=1e-12)
            else:
                assert s.lambda_ == pytest.approx(lam_used[k] * (s.nu / 2.0), rel=1e-12)
    ctx.close()


def test_learned_policy_against_nielsen():
    """Train on trajectories of 128 problems (rollout labels, two DAgger rounds); on 64
    held-out problems compare with Nielsen's rule: problems whose cost gets within 1e-3 of the
    best cost any run reaches in 150 iterations, the mean iterations to get there (150 + 1 when
    never), and the median remaining gap after 150 iterations."""
    cuda_or_skip()
    from paper_1802_03773_gb300 import learned
    g = np.random.default_rng(11)
    spec = lambda n, base: [(int(g.integers(500, 3001)), int(g.integers(16, 65)), base + i) for i in range(n)]
    train_b = learned.Batch(problems(spec(128, 1000)))
    test_b = learned.Batch(problems(spec(64, 5000)))
    params, nsamples, loss = learned.train_policy(train_b, mlp_init(7))
    assert nsamples > 1000
    iters = 150
    h_n, _ = learned.run(test_b, iters=iters)
    h_m, _ = learned.run(test_b, iters=iters, params=params)
    best = np.minimum(h_n[-1], h_m[-1])
    stats = {}
    for name, h in (("nielsen", h_n), ("mlp", h_m)):
        it = learned.iterations_to(h, best * (1.0 + 1e-3))
        stats[name] = (int(np.isfinite(it).sum()), float(np.where(np.isfinite(it), it, iters + 1).mean()),
                       float(np.median((h[-1] - best) / best)))
        print(f"{name}: within 1e-3 on {stats[name][0]}/64, mean iterations {stats[name][1]:.1f}, "
              f"median final gap {stats[name][2]:.2e}")
    assert stats["mlp"][0] >= stats["nielsen"][0]
    assert stats["mlp"][1] <= stats["nielsen"][1]
    assert stats["mlp"][2] <= stats["nielsen"][2]
