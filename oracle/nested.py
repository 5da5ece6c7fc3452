"""Nested sampling with batch deletion and a Slice-within-Gibbs inner kernel, FP64.

Outer loop (Sec. 2.2, Eq. 1): m live points; each iteration deletes the k with
the lowest logL, sets logL* to the lowest logL among the survivors, adds the
deleted points' volume to Z and replaces them with k draws from the constrained
prior pi* ~ pi 1[logL > logL*] made by k independent chains started at
survivors.  Deaths within a batch are treated as k successive deaths with live
counts m, m-1, ..., m-k+1, each shrinking log X by 1/n (its expected value).
Dead weights use the simple quadrature w_j = L_j (X_{j-1} - X_j).  The run
stops when log Z_live - log Z_dead < -3 (Sec. 3.2), Z_live = X * mean(L_live);
the live points are then added with weight X/m each.

Inner kernel (Sec. 2.3, Eq. 3; Sec. 3.2): for each of M sweeps and each Gibbs
block b in order, ``steps_per_dim * |b|`` hit-and-run slice updates of the
block-conditional constrained prior.  Directions are n = L_b z, z ~ N(0, I),
with L_b the Cholesky factor of the covariance of the m live points at the
start of the iteration restricted to block b.  Each update follows Neal (2003)
stepping-out and shrinkage along n with unit width and random initial offset.

Readings where the paper is silent (this module's own choices): start points are
drawn uniformly with replacement among the survivors; stepping-out and
shrinkage are capped at 100 moves (on a shrink cap the chain keeps its point);
bounded unit-cube coordinates (no wrapping for periodic angles).
"""
from __future__ import annotations

import math

import numpy as np

MAX_STEP_OUT = 100
MAX_SHRINK = 100


def block_cholesky(points, blocks, jitter=1e-12):
    """Cholesky factors of the live-point covariance restricted to each block."""
    cov = np.atleast_2d(np.cov(points, rowvar=False))
    out = []
    for b in blocks:
        c = cov[np.ix_(b, b)].copy()
        c += jitter * (np.trace(c) / len(b) + 1e-300) * np.eye(len(b))
        out.append(np.linalg.cholesky(c))
    return out


def inside_cube(x):
    return bool(np.all(x >= 0.0) and np.all(x <= 1.0))


def slice_step(x, logl_x, block, chol, logl_star, loglike, rng, counters):
    """One hit-and-run slice update of the dims in ``block`` (Neal 2003)."""
    nb = len(block)
    z = rng.standard_normal(nb)
    direction = np.zeros_like(x)
    direction[block] = chol @ z
    r = rng.random()
    lo, hi = -r, 1.0 - r

    def in_slice(t):
        y = x + t * direction
        if not inside_cube(y):
            return False, y, -np.inf
        ly = loglike(y)
        counters["evals"] += 1
        return ly > logl_star, y, ly

    n_out = 0
    while n_out < MAX_STEP_OUT:
        ok, _, _ = in_slice(lo)
        if not ok:
            break
        lo -= 1.0
        n_out += 1
    n_out = 0
    while n_out < MAX_STEP_OUT:
        ok, _, _ = in_slice(hi)
        if not ok:
            break
        hi += 1.0
        n_out += 1
    for _ in range(MAX_SHRINK):
        t = lo + (hi - lo) * rng.random()
        ok, y, ly = in_slice(t)
        if ok:
            return y, ly
        if t < 0.0:
            lo = t
        else:
            hi = t
    counters["shrink_caps"] += 1
    return x, logl_x


def run_nested(loglike, ndim, blocks, nlive, nrep, steps_per_dim=5, sweeps=1, rng=None,
               dlogz=-3.0, max_iter=100000, init_points=None):
    """Run nested sampling; returns a dict with dead points, weights and log Z.

    ``loglike`` maps a unit-cube point (ndim,) to logL (or -inf).
    """
    rng = np.random.default_rng(rng)
    if init_points is None:
        live = rng.random((nlive, ndim))
    else:
        live = np.array(init_points, dtype=np.float64)
    live_l = np.array([loglike(x) for x in live])
    counters = {"evals": nlive, "shrink_caps": 0}
    log_x = 0.0
    log_z = -np.inf
    dead_u, dead_l, dead_logw = [], [], []
    n_iter = 0
    while n_iter < max_iter:
        m = live_l.max()
        log_z_live = log_x + m + math.log(np.mean(np.exp(live_l - m)))
        if np.isfinite(log_z) and log_z_live - log_z < dlogz:
            break
        order = np.argsort(live_l, kind="stable")
        worst, survivors = order[:nrep], order[nrep:]
        logl_star = live_l[survivors[0]]
        for j, idx in enumerate(worst):
            n = nlive - j
            log_x_new = log_x - 1.0 / n
            logw = live_l[idx] + log_x + math.log1p(-math.exp(-1.0 / n))
            dead_u.append(live[idx].copy())
            dead_l.append(live_l[idx])
            dead_logw.append(logw)
            log_z = np.logaddexp(log_z, logw)
            log_x = log_x_new
        chol = block_cholesky(live, blocks)
        starts = survivors[rng.integers(0, survivors.size, size=nrep)]
        new_u = np.empty((nrep, ndim))
        new_l = np.empty(nrep)
        for c in range(nrep):
            x = live[starts[c]].copy()
            lx = live_l[starts[c]]
            for _ in range(sweeps):
                for bi, b in enumerate(blocks):
                    for _ in range(steps_per_dim * len(b)):
                        x, lx = slice_step(x, lx, b, chol[bi], logl_star, loglike, rng, counters)
            new_u[c], new_l[c] = x, lx
        live[worst] = new_u
        live_l[worst] = new_l
        n_iter += 1
    # add the remaining live points, X/m each
    for idx in np.argsort(live_l, kind="stable"):
        logw = live_l[idx] + log_x - math.log(nlive)
        dead_u.append(live[idx].copy())
        dead_l.append(live_l[idx])
        dead_logw.append(logw)
        log_z = np.logaddexp(log_z, logw)
    dead_logw = np.array(dead_logw)
    dead_l = np.array(dead_l)
    p = np.exp(dead_logw - log_z)
    h_info = float(np.sum(p * (dead_l - log_z)))
    return {
        "u": np.array(dead_u), "logl": dead_l, "logw": dead_logw, "logz": float(log_z),
        "logz_err": math.sqrt(max(h_info, 0.0) / nlive), "info": h_info,
        "n_iter": n_iter, "n_evals": counters["evals"], "shrink_caps": counters["shrink_caps"],
        "ess": float(1.0 / np.sum(p**2)),
    }
