"""Write the exact evidence of the 4 s single-detector workload by importance
sampling of the FP64 oracle likelihood (tests/golden/cfg1_is_evidence.txt),
and the importance-weighted draws themselves as the reference posterior
(tests/golden/cfg1_is_posterior.csv: independent draws, each with its exact
weight L pi / q, so the only error is the Monte Carlo one of the weights).

Proposal: a multivariate t (5 degrees of freedom) fitted to the oracle's own
nested-sampling posterior (tests/golden/cfg1_oracle_posterior.csv), with its
covariance inflated x4, in (Mc, q, d_L, t_c); Z = mean of L pi / q over the
draws, with its Monte Carlo standard error.  Calls only oracle/ and
swig_inputs.  Run from the repository root.
"""
import math
import os
import sys

import numpy as np
from scipy import stats

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import swig_inputs as si  # noqa: E402
from oracle import events  # noqa: E402
from oracle import likelihood as L  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
N, SEED = 20000, 2


def main():
    wl = si.config1()
    ev, th = events.build_event(wl)
    path = os.path.join(HERE, "cfg1_oracle_posterior.csv")
    head = open(path).readlines()[1]
    lz = float(head.split("logz=")[1].split()[0])
    ref = np.loadtxt(path, delimiter=",", comments="#", skiprows=3)
    w = np.exp(ref[:, -1] - lz)
    w /= w.sum()
    X = ref[:, :4]
    mu = np.sum(w[:, None] * X, axis=0)
    C = np.cov(X.T, aweights=w)
    sd = np.sqrt(np.diag(C))
    prop = stats.multivariate_t(loc=np.zeros(4), shape=4 * C / np.outer(sd, sd), df=5, seed=SEED)
    S = mu + prop.rvs(N) * sd
    slots = [si.IDX[n] for n in ("mc", "q", "dl", "tc")]
    lo = np.array([wl.params[s].lo for s in slots])
    hi = np.array([wl.params[s].hi for s in slots])
    logprior = -np.sum(np.log(hi - lo))
    lw = np.full(N, -np.inf)
    for i in range(N):
        if np.all((S[i] >= lo) & (S[i] <= hi)):
            t = th.copy()
            t[slots] = S[i]
            lw[i] = L.loglike(ev, t) + logprior - (prop.logpdf((S[i] - mu) / sd) - np.sum(np.log(sd)))
    m = lw.max()
    r = np.exp(lw - m)
    logz = m + math.log(r.mean())
    err = r.std(ddof=1) / math.sqrt(N) / r.mean()
    ok = np.isfinite(lw)
    ess = 1.0 / np.sum((r[ok] / r[ok].sum()) ** 2)
    # draws below 1e-4 of the largest weight carry 3e-5 of the mass: not kept
    ok &= r >= 1e-4
    lwn = lw[ok] - math.log(N)  # normalised: logsumexp = log Z (up to the dropped mass)
    with open(os.path.join(HERE, "cfg1_is_posterior.csv"), "w") as f:
        f.write("# importance-sampled posterior, config 1 (H1, 4 s), oracle likelihood\n")
        f.write(f"# logz={logz:.6f} logz_err={err:.6f} ess={ess:.1f} n_draws={N} kept={int(ok.sum())}\n")
        f.write("mc,q,dl,tc,logl,logw\n")
        for x, l in zip(S[ok], lwn):
            t = th.copy()
            t[slots] = x
            f.write(",".join(f"{v:.10g}" for v in list(x) + [L.loglike(ev, t), l]) + "\n")
    with open(os.path.join(HERE, "cfg1_is_evidence.txt"), "w") as f:
        f.write("# exact log-evidence of config 1 (H1, 4 s) by importance sampling of the FP64 oracle\n")
        f.write(f"# draws={N} seed={SEED} proposal=multivariate-t(df=5, 4x posterior covariance)\n")
        f.write(f"{logz:.6f} {err:.6f}\n")
    print(logz, err)


if __name__ == "__main__":
    main()
