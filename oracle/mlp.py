"""Learned slice proposal: the network, its training targets and Adam (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper draws slice directions from the live points' covariance (Sec. 2.3,
Eq. 3; Sec. 3.2) and does not learn them.  This module defines the learned
alternative the library offers, written plainly so that the CUDA kernels can be
checked against it:

* Network (13 -> 256 -> 256 -> 26, SiLU): input a live point in standardised
  unit-cube coordinates (x - mean) / std of the live set, zero beyond the d
  sampled dimensions; output (u, s): a direction u and per-dimension
  log-widths s.
* Targets, per live point: the K = 2d nearest other live points (Euclidean in
  standardised coordinates, ties by index); their covariance C in unit-cube
  coordinates; sigma_j = sqrt(C_jj) (floored at 1e-12); t = log sigma; e1 = the
  leading eigenvector of the correlation matrix C / (sigma sigma^T), its
  largest-magnitude entry made positive.
* Loss, mean over points: 1 - (u_hat . e1)^2 + sum_{j<d} (s_j - t_j)^2 with
  u_hat = u / sqrt(|u|^2 + 1e-12), u restricted to the sampled dimensions.
* Slice direction for Gibbs block b from an output row: n_b = exp(s_b) *
  u_b / sqrt(|u_b|^2 + 1e-12), zero outside the block.  Its distribution does
  not depend on the chain's position (the row belongs to a live point drawn
  uniformly from a frozen snapshot), so the hit-and-run slice move keeps the
  constrained prior invariant.
* Mixed precision: with ``bf16=True`` every matrix-product operand (inputs,
  activations, output gradients and weights) is rounded to bfloat16 (round to
  nearest, ties to even) before the product; sums, biases, SiLU and the loss
  stay in full precision.  That is the arithmetic the GPU kernels perform with
  FP32 accumulation.
* Adam (Kingma & Ba 2015) with bias correction on FP32/FP64 master weights.
* Initial weights: N(0, 1/fan_in) from Philox-4x32-10 with the Box-Muller
  transform; biases zero.

Parameter vector layout (flat): W1 [13][256], b1 [256], W2 [256][256], b2 [256],
W3 [256][26], b3 [26] (row index = input unit).
"""
from __future__ import annotations

import math

import numpy as np

from .philox import philox4x32_10

D_IN, D_H, D_OUT = 13, 256, 26
SHAPES = [(D_IN, D_H), (D_H,), (D_H, D_H), (D_H,), (D_H, D_OUT), (D_OUT,)]
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES)
EPS_NORM = 1e-12


def unpack(flat):
    out, o = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(np.asarray(flat[o:o + n], dtype=np.float64).reshape(s))
        o += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), through float32."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def init_params(seed):
    """W[i][j] = z / sqrt(fan_in), z = Box-Muller of Philox words 0, 1 at
    counter (j, i, layer, 9) with key (seed lo, seed hi); biases 0."""
    k0, k1 = seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF
    parts = []
    for layer, s in enumerate(SHAPES):
        if len(s) == 1:
            parts.append(np.zeros(s))
            continue
        w = np.empty(s)
        for i in range(s[0]):
            for j in range(s[1]):
                r = philox4x32_10((j, i, layer, 9), (k0, k1))
                u1 = ((r[0] >> 8) + 1) * 2.0 ** -24
                u2 = (r[1] >> 8) * 2.0 ** -24
                w[i, j] = math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2) / math.sqrt(s[0])
        parts.append(w)
    return pack(parts)


def standardise(live_u, d):
    """Network inputs: (x - mean) / std per sampled dimension (std floored at
    1e-12, population form), zero-padded to 13 columns."""
    live_u = np.asarray(live_u, dtype=np.float64)
    mu = live_u.mean(axis=0)
    sd = np.maximum(live_u.std(axis=0), 1e-12)
    xs = np.zeros((live_u.shape[0], D_IN))
    xs[:, :d] = (live_u - mu) / sd
    return xs


def forward(params, xs, bf16=False):
    W1, b1, W2, b2, W3, b3 = unpack(params)
    r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    X = r(xs)
    Z1 = X @ r(W1) + b1
    H1 = silu(Z1)
    Z2 = r(H1) @ r(W2) + b2
    H2 = silu(Z2)
    O = r(H2) @ r(W3) + b3
    return {"X": X, "Z1": Z1, "H1": H1, "Z2": Z2, "H2": H2, "O": O}


def loss_and_dout(O, tdir, tlogsig, d):
    """Mean loss over the rows of O and its gradient with respect to O."""
    n = O.shape[0]
    u = np.zeros((n, D_IN))
    u[:, :d] = O[:, :d]
    s = O[:, D_IN:]
    norm = np.sqrt(np.sum(u * u, axis=1) + EPS_NORM)
    uh = u / norm[:, None]
    c = np.sum(uh * tdir, axis=1)
    diff = np.zeros((n, D_IN))
    diff[:, :d] = s[:, :d] - tlogsig[:, :d]
    loss = float(np.mean(1.0 - c * c + np.sum(diff * diff, axis=1)))
    dO = np.zeros_like(O)
    du = -2.0 * c[:, None] * (tdir - c[:, None] * uh) / norm[:, None]
    dO[:, :d] = du[:, :d] / n
    dO[:, D_IN:D_IN + d] = 2.0 * diff[:, :d] / n
    return loss, dO


def backward(params, cache, dO, bf16=False):
    """Gradients of sum(dO * O) with respect to the parameters (flat)."""
    _, _, W2, _, W3, _ = unpack(params)
    r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    dOr = r(dO)
    gW3 = r(cache["H2"]).T @ dOr
    gb3 = dO.sum(axis=0)
    dZ2 = (dOr @ r(W3).T) * dsilu(cache["Z2"])
    dZ2r = r(dZ2)
    gW2 = r(cache["H1"]).T @ dZ2r
    gb2 = dZ2.sum(axis=0)
    dZ1 = (dZ2r @ r(W2).T) * dsilu(cache["Z1"])
    gW1 = cache["X"].T @ r(dZ1)
    gb1 = dZ1.sum(axis=0)
    return pack([gW1, gb1, gW2, gb2, gW3, gb3])


def adam_update(params, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (step number t >= 1); returns (params, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def local_pca_targets(live_u, k=None, details=False):
    """Per live point: (e1 padded to 13, log sigma padded to 13); with
    details also the neighbour indices (n x k, distance order) and the
    relative eigen-gap (lambda1 - lambda2) / lambda1 of each correlation
    matrix (e1 is well defined only where it is not small)."""
    live_u = np.asarray(live_u, dtype=np.float64)
    n, d = live_u.shape
    k = 2 * d if k is None else k
    xs = standardise(live_u, d)[:, :d]
    tdir = np.zeros((n, D_IN))
    tls = np.zeros((n, D_IN))
    nbrs = np.zeros((n, k), dtype=np.int64)
    gaps = np.zeros(n)
    for i in range(n):
        d2 = np.sum((xs - xs[i]) ** 2, axis=1)
        d2[i] = np.inf
        nb = np.lexsort((np.arange(n), d2))[:k]
        Y = live_u[nb]
        C = np.cov(Y.T, bias=True).reshape(d, d)
        sig = np.maximum(np.sqrt(np.diag(C)), 1e-12)
        R = C / np.outer(sig, sig)
        w, V = np.linalg.eigh(R)
        e1 = V[:, -1]
        if e1[np.argmax(np.abs(e1))] < 0:
            e1 = -e1
        tdir[i, :d] = e1
        tls[i, :d] = np.log(sig)
        nbrs[i] = nb
        gaps[i] = (w[-1] - w[-2]) / w[-1] if d > 1 else 1.0
    if details:
        return tdir, tls, nbrs, gaps
    return tdir, tls


def block_direction(out_row, dims):
    """Slice direction of a Gibbs block (unit-cube dims) from one output row."""
    dims = np.asarray(dims)
    u = out_row[dims]
    s = out_row[D_IN + dims]
    return np.exp(s) * u / math.sqrt(float(np.sum(u * u)) + EPS_NORM)
