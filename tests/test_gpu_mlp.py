"""The learned-proposal network on the GPU against the FP64 oracle.

The kernels take bfloat16 operands and accumulate in FP32; the oracle's
``bf16=True`` path rounds the same operands the same way and accumulates in
FP64, so the two differ only by FP32 accumulation (relative ~1e-6) and the
rare operand whose bf16 rounding flips because its FP32 and FP64 values
straddle a rounding boundary (one bf16 ulp, 2^-8 relative, on one element).
The tolerances below allow for both; the comparison with the pure FP64
network shows the size of the bf16 effect itself.
"""
import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu

swig = pytest.importorskip("paper_2607_28265_gb300.swig")


@pytest.fixture(scope="module")
def ctx():
    c = swig.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def params0():
    return mlp.init_params(77)


def _inputs(n, d, seed):
    rng = np.random.default_rng(seed)
    x = np.zeros((n, mlp.D_IN))
    x[:, :d] = rng.standard_normal((n, d))
    return x


def _curved_live(n, d, seed):
    """Live-like points in the unit cube with a curved, correlated core."""
    rng = np.random.default_rng(seed)
    t = rng.random(n)
    u = np.empty((n, d))
    u[:, 0] = 0.2 + 0.6 * t
    u[:, 1] = 0.5 + 0.25 * np.sin(3 * t) + 0.02 * rng.standard_normal(n)
    for j in range(2, d):
        u[:, j] = 0.5 + 0.1 * (j % 3 - 1) * t + 0.05 * rng.standard_normal(n)
    return np.clip(u, 0.0, 1.0)


def test_init_matches_oracle(ctx, params0):
    p = ctx.mlp_init(77)
    assert p.shape == (mlp.N_PARAMS,)
    assert np.all(np.abs(p - params0) <= 1e-6 * np.abs(params0) + 1e-9)


@pytest.mark.parametrize("n,d", [(1, 13), (300, 12), (1000, 4)])
def test_forward_matches_oracle(ctx, params0, n, d):
    x = _inputs(n, d, n)
    got = ctx.mlp_forward(params0, x)
    want = mlp.forward(params0, x, bf16=True)["O"]
    scale = np.max(np.abs(want))
    assert np.max(np.abs(got - want)) <= 2e-3 * scale, np.max(np.abs(got - want)) / scale
    exact = mlp.forward(params0, x)["O"]
    assert np.max(np.abs(got - exact)) <= 5e-2 * scale


def test_loss_and_gradient_match_oracle(ctx, params0):
    n, d = 500, 12
    live = _curved_live(n, d, 3)
    tdir, tls = mlp.local_pca_targets(live)
    x = mlp.standardise(live, d)
    loss, g = ctx.mlp_loss_grad(params0, x, tdir, tls, d)
    cache = mlp.forward(params0, x, bf16=True)
    want_loss, dO = mlp.loss_and_dout(cache["O"], tdir, tls, d)
    want = mlp.backward(params0, cache, dO, bf16=True)
    assert abs(loss - want_loss) <= 1e-4 * abs(want_loss)
    offs = np.cumsum([0] + [int(np.prod(s)) for s in mlp.SHAPES])
    for a, b in zip(offs[:-1], offs[1:]):
        gs, ws = g[a:b], want[a:b]
        scale = np.max(np.abs(ws))
        assert np.max(np.abs(gs - ws)) <= 1e-2 * scale, (a, np.max(np.abs(gs - ws)) / scale)
        # overall agreement: relative L2 error of the block
        assert np.linalg.norm(gs - ws) <= 3e-3 * np.linalg.norm(ws)
    # exact zeros where the sampled dimensions end (inputs and outputs beyond d)
    W1 = g[:offs[1]].reshape(13, 256)
    assert not W1[d:].any()
    W3 = g[offs[4]:offs[5]].reshape(256, 26)
    assert not W3[:, d:13].any() and not W3[:, 13 + d:].any()


def test_targets_match_oracle(ctx):
    n, d = 600, 12
    live = _curved_live(n, d, 5)
    tdir, tls, nbr = ctx.mlp_targets(live)
    want_dir, want_ls, want_nbr, gap = mlp.local_pca_targets(live, details=True)
    assert np.array_equal(nbr, want_nbr)
    assert np.all(np.abs(tls - want_ls) <= 1e-6 * np.abs(want_ls) + 1e-6)
    ok = gap > 0.05
    assert ok.sum() > n // 2
    dots = np.abs(np.sum(tdir[ok] * want_dir[ok], axis=1))
    assert np.all(dots > 1 - 1e-5), dots.min()
    # the sign convention holds everywhere the direction is defined
    same = np.sum(tdir[ok] * want_dir[ok], axis=1) > 0
    assert same.all()


def test_training_matches_oracle_and_reduces_loss(ctx, params0):
    n, d, steps, lr = 400, 6, 3, 1e-3
    live = _curved_live(n, d, 8)
    p_gpu, out = ctx.mlp_train(live, params0, steps, lr)
    tdir, tls = mlp.local_pca_targets(live)
    x = mlp.standardise(live, d)
    p = params0.copy()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    losses = []
    for t in range(1, steps + 1):
        cache = mlp.forward(p, x, bf16=True)
        loss, dO = mlp.loss_and_dout(cache["O"], tdir, tls, d)
        losses.append(loss)
        g = mlp.backward(p, cache, dO, bf16=True)
        p, m, v = mlp.adam_update(p, g, m, v, t, lr=lr)
    # Adam moves each weight by about lr per step whatever the gradient's
    # size, so weights whose gradient is near zero may move differently;
    # all but a small fraction agree to 1 % of the total step
    dev = np.abs((p_gpu - params0) - (p - params0))
    assert np.mean(dev > 1e-2 * lr * steps) < 0.01
    assert np.max(dev) <= 2 * lr * steps + 1e-7
    want_out = mlp.forward(p, x, bf16=True)["O"]
    assert np.max(np.abs(out - want_out)) <= 1e-2 * np.max(np.abs(want_out))
    # more steps lower the loss on both sides
    p_more, _ = ctx.mlp_train(live, params0, 60, lr)
    cache = mlp.forward(p_more.astype(np.float64), x, bf16=True)
    assert mlp.loss_and_dout(cache["O"], tdir, tls, d)[0] < 0.9 * losses[0]


def test_training_is_deterministic(ctx, params0):
    live = _curved_live(300, 5, 9)
    a, oa = ctx.mlp_train(live, params0, 20)
    b, ob = ctx.mlp_train(live, params0, 20)
    assert np.array_equal(a, b) and np.array_equal(oa, ob)
