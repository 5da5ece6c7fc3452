"""Calibration tools of Sec. 5.1 and App. B: weighted credible levels, KS,
Fisher combination and binomial bands."""
from __future__ import annotations

import math

import numpy as np
from scipy import stats


def credible_level(samples, log_weights, truth):
    """q = sum_j w_j 1(theta_j < theta_true) with normalised NS weights."""
    w = np.exp(np.asarray(log_weights) - np.max(log_weights))
    w /= w.sum()
    return float(np.sum(w * (np.asarray(samples) < truth)))


def ks_uniform_pvalue(levels):
    return float(stats.kstest(np.asarray(levels), "uniform").pvalue)


def fisher_combined(pvalues):
    """Fisher's method: -2 sum log p ~ chi^2 with 2n degrees of freedom."""
    p = np.clip(np.asarray(pvalues, dtype=np.float64), 1e-300, 1.0)
    return float(stats.chi2.sf(-2.0 * np.sum(np.log(p)), 2 * p.size))


def binomial_band(p, n):
    """One-sigma width sqrt(p (1 - p) / N) of the empirical CDF at level p."""
    return math.sqrt(p * (1.0 - p) / n)


def weighted_ks_2samp(x1, w1, x2, w2):
    """Two-sample KS distance between weighted samples, with Kish effective sizes.

    Returns (D, p) where p uses the asymptotic Kolmogorov distribution with
    n_eff = n1 n2 / (n1 + n2) built from each sample's Kish ESS.
    """
    x1, x2 = np.asarray(x1), np.asarray(x2)
    w1 = np.asarray(w1, dtype=np.float64) / np.sum(w1)
    w2 = np.asarray(w2, dtype=np.float64) / np.sum(w2)
    grid = np.sort(np.concatenate([x1, x2]))
    o1, o2 = np.argsort(x1), np.argsort(x2)
    c1 = np.concatenate([[0.0], np.cumsum(w1[o1])])
    c2 = np.concatenate([[0.0], np.cumsum(w2[o2])])
    f1 = c1[np.searchsorted(x1[o1], grid, side="right")]
    f2 = c2[np.searchsorted(x2[o2], grid, side="right")]
    d = float(np.max(np.abs(f1 - f2)))
    n1, n2 = 1.0 / np.sum(w1**2), 1.0 / np.sum(w2**2)
    ne = n1 * n2 / (n1 + n2)
    return d, float(stats.kstwobign.sf(d * math.sqrt(ne)))
