"""Pins of the oracle nested sampler: closed-form evidence, the prior-volume
shrinkage law, invariance of the constrained slice kernel, p-p calibration."""
import math

import numpy as np
import pytest
from scipy import special, stats

from oracle import nested, pp
from oracle.philox import philox4x32_10


def gaussian_problem(mu, sigma):
    mu = np.asarray(mu, dtype=np.float64)
    d = mu.size

    def loglike(u):
        if np.any(u < 0) or np.any(u > 1):
            return -np.inf
        r2 = np.sum((u - mu) ** 2)
        return -0.5 * r2 / sigma**2 - d * math.log(sigma * math.sqrt(2 * math.pi))

    # closed form: prod_j [Phi((1-mu_j)/s) - Phi(-mu_j/s)]
    logz = float(np.sum(np.log(special.ndtr((1 - mu) / sigma) - special.ndtr(-mu / sigma))))
    return loglike, logz


@pytest.mark.parametrize("d,sigma,blocks", [(2, 0.05, [[0, 1]]), (4, 0.08, [[0, 1], [2], [3]])])
def test_gaussian_evidence_closed_form(d, sigma, blocks):
    rng = np.random.default_rng(10 + d)
    mu = rng.uniform(0.3, 0.7, d)
    ll, logz = gaussian_problem(mu, sigma)
    res = nested.run_nested(ll, d, blocks, nlive=200, nrep=20, steps_per_dim=5, rng=11 + d)
    assert abs(res["logz"] - logz) < 4 * res["logz_err"] + 0.05
    # posterior mean recovers mu
    w = np.exp(res["logw"] - res["logz"])
    mean = np.sum(w[:, None] * res["u"], axis=0)
    assert np.allclose(mean, mu, atol=4 * sigma / math.sqrt(res["ess"]) + 2e-3)


def test_prior_volume_shrinkage_law():
    """On L = -|u - 1/2| the true enclosed volume is the d-ball, X = V_d r^d,
    while the run assigns log X_j = -sum 1/n.  Their difference at each death
    has mean 0 and variance sum 1/n^2 (Skilling 2006)."""
    d = 3
    ll = lambda u: -float(np.linalg.norm(u - 0.5)) if np.all((u >= 0) & (u <= 1)) else -np.inf
    vd = math.pi ** (d / 2) / special.gamma(d / 2 + 1)
    diffs = []
    for seed in range(4):
        res = nested.run_nested(ll, d, [[0, 1, 2]], nlive=100, nrep=10, rng=100 + seed, dlogz=-1e9, max_iter=60)
        n = 100
        logx, expect, var = 0.0, [], []
        for j, l in enumerate(res["logl"][: 60 * 10]):
            nj = n - (j % 10)
            logx -= 1.0 / nj
            r = -l
            if r < 0.5:
                expect.append(logx - (math.log(vd) + d * math.log(r)))
                var.append(sum(1.0 / (n - (i % 10)) ** 2 for i in range(j + 1)))
        diffs.append(expect[-1] / math.sqrt(var[-1]))
    assert abs(np.mean(diffs)) < 3.0 / math.sqrt(len(diffs)) + 0.5


def test_run_assigns_the_true_enclosed_volume():
    """The prior volume a run assigns to its deaths, read from its own
    weights (X_j = sum over later dead points of exp(logw - logL), the final
    live points included), against the true enclosed volume of the d-ball on
    L = -|u - 1/2|.  log X_run - log X_true has mean 0 and variance
    sum 1/n^2 over the deaths (Skilling 2006); after 200 iterations of
    k = 10 deaths from m = 100 a per-death shrinkage of 1/m instead of
    1/(m - j) would sit ~2.3 standard deviations off."""
    d, m, k, iters = 3, 100, 10, 200
    ll = lambda u: -float(np.linalg.norm(u - 0.5)) if np.all((u >= 0) & (u <= 1)) else -np.inf
    vd = math.pi ** (d / 2) / special.gamma(d / 2 + 1)
    var = sum(1.0 / (m - (i % k)) ** 2 for i in range(iters * k))
    zs = []
    for seed in range(8):
        res = nested.run_nested(ll, d, [[0, 1, 2]], nlive=m, nrep=k, rng=300 + seed, dlogz=-1e9, max_iter=iters)
        inc = np.exp(res["logw"] - res["logl"])  # X_{j-1} - X_j of each dead point
        j = iters * k - 1  # the last death before the final live points
        log_x_run = math.log(float(np.sum(inc[j + 1:])))
        log_x_true = math.log(vd) + d * math.log(-res["logl"][j])
        zs.append((log_x_run - log_x_true) / math.sqrt(var))
    assert abs(np.mean(zs)) < 3.0 / math.sqrt(len(zs)) + 0.3, zs


def test_slice_kernel_leaves_constrained_uniform_invariant():
    """Chains started from the constrained prior (uniform in a ball of radius
    r* inside the cube) stay uniform: r^d / r*^d ~ U(0, 1)."""
    d, rstar = 3, 0.3
    ll = lambda u: -float(np.linalg.norm(u - 0.5))
    rng = np.random.default_rng(7)
    pts = []
    while len(pts) < 400:
        x = rng.random(d)
        if np.linalg.norm(x - 0.5) < rstar:
            pts.append(x)
    pts = np.array(pts)
    chol = nested.block_cholesky(pts, [[0, 1, 2]])
    cnt = {"evals": 0, "shrink_caps": 0}
    out = []
    for x in pts:
        lx = ll(x)
        for _ in range(5):
            x, lx = nested.slice_step(x, lx, [0, 1, 2], chol[0], -rstar, ll, rng, cnt)
        out.append(np.linalg.norm(x - 0.5))
    out = np.array(out)
    assert np.all(out < rstar)
    assert stats.kstest((out / rstar) ** d, "uniform").pvalue > 0.01


def test_one_slice_step_from_a_fixed_point_is_uniform_on_the_slice():
    """On a one-dimensional slice (the interval L > L* = (0.3, 0.7)) one
    stepping-out and shrinkage step from a fixed start lands uniformly on the
    slice (Neal 2003): shrinkage only removes ground outside it.  20,000
    independent steps from x0 = 0.32 near the edge: KS against U(0.3, 0.7),
    and no step may stay at x0."""
    ll = lambda u: -abs(float(u[0]) - 0.5)
    chol = np.array([[0.15]])
    rng = np.random.default_rng(12)
    cnt = {"evals": 0, "shrink_caps": 0}
    x0 = np.array([0.32])
    out = np.array([nested.slice_step(x0, ll(x0), [0], chol, -0.2, ll, rng, cnt)[0][0] for _ in range(20000)])
    assert cnt["shrink_caps"] == 0 and not np.any(out == x0[0])
    assert np.all((out > 0.3) & (out < 0.7))
    assert stats.kstest((out - 0.3) / 0.4, "uniform").pvalue > 1e-3


def test_pp_calibration_on_gaussian_toys():
    rng = np.random.default_rng(21)
    levels = []
    for i in range(40):
        truth = rng.uniform(0.2, 0.8, 2)
        sigma = 0.05
        obs = truth + rng.normal(0, sigma, 2)
        ll = lambda u, o=obs: -0.5 * np.sum((u - o) ** 2) / sigma**2 if np.all((u >= 0) & (u <= 1)) else -np.inf
        res = nested.run_nested(ll, 2, [[0], [1]], nlive=60, nrep=6, rng=500 + i)
        levels.append(pp.credible_level(res["u"][:, 0], res["logw"], truth[0]))
    assert pp.ks_uniform_pvalue(levels) > 0.01


def test_pp_tools():
    assert pp.binomial_band(0.5, 100) == pytest.approx(0.05)
    assert pp.binomial_band(0.5, 1000) == pytest.approx(0.0158, rel=1e-2)
    assert pp.fisher_combined([1.0, 1.0]) == pytest.approx(1.0)
    assert pp.fisher_combined([0.5]) == pytest.approx(0.5)


def test_philox_known_answers():
    here = __file__.rsplit("/", 1)[0]
    rows = [l.split() for l in open(f"{here}/golden/philox4x32_10_kat.txt") if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert philox4x32_10(v[0:4], v[4:6]) == tuple(v[6:10])
