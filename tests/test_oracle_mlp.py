"""Pins of the learned-proposal oracle (oracle/mlp.py) against closed forms,
finite differences and special cases."""
import math

import numpy as np
import pytest

from oracle import mlp
from oracle.philox import philox4x32_10


def _small_params(seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal(mlp.N_PARAMS) * 0.1


def test_silu_and_derivative():
    assert mlp.silu(0.0) == 0.0 and mlp.dsilu(0.0) == 0.5
    z = np.linspace(-8, 8, 33)
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.dsilu(z))) < 1e-8
    # limits: silu(z) -> z for z >> 0 and -> 0 for z << 0
    assert abs(mlp.silu(40.0) - 40.0) < 1e-12 and abs(mlp.silu(-40.0)) < 1e-15


def test_bf16_round_closed_forms():
    assert mlp.bf16_round(1.0) == 1.0
    assert mlp.bf16_round(1.0 + 2.0 ** -8) == 1.0            # tie -> even (1.0)
    assert mlp.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6  # tie -> even (mantissa ...10)
    assert mlp.bf16_round(1.0 + 2.0 ** -7) == 1.0 + 2.0 ** -7  # representable
    assert mlp.bf16_round(-2.5) == -2.5
    x = np.random.default_rng(1).standard_normal(10000) * 100
    r = mlp.bf16_round(x)
    # unit roundoff of an 8-bit significand: 2^-8
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x) * (1 + 1e-7))


def test_gradient_against_central_differences():
    rng = np.random.default_rng(3)
    d = 5
    n = 7
    p = _small_params(3)
    xs = np.zeros((n, mlp.D_IN))
    xs[:, :d] = rng.standard_normal((n, d))
    tdir = np.zeros((n, mlp.D_IN))
    e = rng.standard_normal((n, d))
    tdir[:, :d] = e / np.linalg.norm(e, axis=1)[:, None]
    tls = np.zeros((n, mlp.D_IN))
    tls[:, :d] = rng.standard_normal((n, d))

    def f(q):
        return mlp.loss_and_dout(mlp.forward(q, xs)["O"], tdir, tls, d)[0]

    cache = mlp.forward(p, xs)
    _, dO = mlp.loss_and_dout(cache["O"], tdir, tls, d)
    g = mlp.backward(p, cache, dO)
    # every layer's weights and biases are probed
    offs = np.cumsum([0] + [int(np.prod(s)) for s in mlp.SHAPES])
    idx = np.concatenate([rng.choice(np.arange(offs[i], offs[i + 1]), 8, replace=False) for i in range(6)])
    h = 1e-6
    for i in idx:
        q = p.copy()
        q[i] += h
        fp = f(q)
        q[i] -= 2 * h
        fm = f(q)
        fd = (fp - fm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_loss_zero_at_targets_and_sign_invariant():
    d = 4
    rng = np.random.default_rng(5)
    e = rng.standard_normal(d)
    e /= np.linalg.norm(e)
    t = rng.standard_normal(d)
    O = np.zeros((2, mlp.D_OUT))
    O[0, :d] = 3.0 * e
    O[1, :d] = -0.5 * e
    O[:, mlp.D_IN:mlp.D_IN + d] = t
    tdir = np.zeros((2, mlp.D_IN))
    tdir[:, :d] = e
    tls = np.zeros((2, mlp.D_IN))
    tls[:, :d] = t
    loss, dO = mlp.loss_and_dout(O, tdir, tls, d)
    # zero up to the 1e-12 regulariser of |u| (1 - c^2 = 1e-12 / (|u|^2 + 1e-12))
    assert loss < 1e-10 and np.max(np.abs(dO)) < 1e-10
    # orthogonal direction: loss 1 per point
    O2 = O.copy()
    f = np.zeros(d)
    f[0] = 1.0
    f -= e * (f @ e)
    O2[:, :d] = f
    assert abs(mlp.loss_and_dout(O2, tdir, tls, d)[0] - 1.0) < 1e-9


def test_zero_weights_give_biases():
    parts = [np.zeros(s) for s in mlp.SHAPES]
    parts[5] = np.arange(mlp.D_OUT, dtype=float)
    p = mlp.pack(parts)
    out = mlp.forward(p, np.random.default_rng(0).standard_normal((3, mlp.D_IN)))["O"]
    assert np.array_equal(out, np.tile(np.arange(mlp.D_OUT, dtype=float), (3, 1)))


def test_adam_first_steps_closed_form():
    g = np.array([1e-3, -5.0, 2.0, -1e-2])
    p0 = np.zeros(4)
    m = np.zeros(4)
    v = np.zeros(4)
    p1, m, v = mlp.adam_update(p0, g, m, v, 1, lr=0.01)
    # bias-corrected m_hat = g, v_hat = g^2: step = -lr g / (|g| + eps)
    assert np.allclose(p1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    # a constant gradient keeps m_hat = g and v_hat = g^2 at every step
    p2, m, v = mlp.adam_update(p1, g, m, v, 2, lr=0.01)
    assert np.allclose(p2 - p1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)


def test_local_pca_on_a_line_recovers_its_direction():
    """Points on a line x = a + t v: the correlation matrix of any neighbour
    set is sign(v) sign(v)^T, so e1 = sign(v)/sqrt(d) and the block direction
    built from (e1, log sigma) is parallel to v."""
    rng = np.random.default_rng(2)
    v = np.array([0.3, -0.1, 0.05])
    a = np.array([0.2, 0.6, 0.4])
    t = rng.random(40)
    pts = a + t[:, None] * v
    tdir, tls = mlp.local_pca_targets(pts)
    for i in (0, 17, 39):
        e1 = tdir[i, :3]
        assert np.allclose(np.abs(e1), 1 / math.sqrt(3), atol=1e-9)
        row = np.concatenate([tdir[i], tls[i]])
        n = mlp.block_direction(row, [0, 1, 2])
        cosang = abs(n @ v) / (np.linalg.norm(n) * np.linalg.norm(v))
        assert cosang > 1 - 1e-9


def test_local_pca_scale_on_a_grid():
    """A regular 1-D grid of spacing h (d = 1, K = 2): an interior point's two
    neighbours sit at +-h, so sigma = h exactly."""
    h = 0.01
    pts = (0.1 + h * np.arange(30))[:, None]
    _, tls = mlp.local_pca_targets(pts)
    assert abs(tls[10, 0] - math.log(h)) < 1e-9


def test_init_params_statistics_and_counter_layout():
    p = mlp.init_params(12345)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p)
    assert not b1.any() and not b2.any() and not b3.any()
    # W2 has 65536 N(0, 1/256) draws: mean and variance within 5 sigma
    z = W2.ravel() * 16.0
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / z.size)
    # one entry recomputed from the Philox words (counter (j, i, layer, 9))
    r = philox4x32_10((7, 3, 0, 9), (12345, 0))
    u1 = ((r[0] >> 8) + 1) * 2.0 ** -24
    u2 = (r[1] >> 8) * 2.0 ** -24
    assert W1[3, 7] == pytest.approx(math.sqrt(-2 * math.log(u1)) * math.cos(2 * math.pi * u2) / math.sqrt(13),
                                     rel=1e-15)


def test_bf16_forward_close_to_fp64():
    rng = np.random.default_rng(9)
    p = mlp.init_params(1)
    xs = rng.standard_normal((20, mlp.D_IN))
    a = mlp.forward(p, xs)["O"]
    b = mlp.forward(p, xs, bf16=True)["O"]
    assert np.max(np.abs(a - b)) < 0.05 * np.max(np.abs(a))
