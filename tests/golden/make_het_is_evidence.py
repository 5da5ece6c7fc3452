"""Write the exact evidence of the heterodyned likelihood on the 4 s
single-detector workload (tests/golden/cfg3_het_is_evidence.txt).

Heterodyned likelihood (Sec. 3.4) of the FP64 oracle: fiducial = injection,
450 bins with geometric spacing and 450 bins of equal maximum phase change.
Importance sampling with the same proposal as make_is_evidence.py (a
multivariate t, 5 degrees of freedom, fitted to the oracle's nested-sampling
posterior in (Mc, q, d_L, t_c), covariance inflated x4); the full-grid
evidence of the same draws is written beside it, so the file also records
how far the approximation moves log Z.  Calls only oracle/ and swig_inputs.
Run from the repository root.
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
N, SEED, NB = 20000, 3, 450


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
    hets = {"geometric": L.het_setup(ev, th, NB, spacing="geometric"), "phase": L.het_setup(ev, th, NB)}
    lws = {k: np.full(N, -np.inf) for k in ("geometric", "phase", "full")}
    for i in range(N):
        if np.all((S[i] >= lo) & (S[i] <= hi)):
            t = th.copy()
            t[slots] = S[i]
            lq = logprior - (prop.logpdf((S[i] - mu) / sd) - np.sum(np.log(sd)))
            for k, h in hets.items():
                lws[k][i] = L.het_loglike(ev, h, t) + lq
            lws["full"][i] = L.loglike(ev, t) + lq
    out = {}
    for k, lw in lws.items():
        m = lw.max()
        r = np.exp(lw - m)
        out[k] = (m + math.log(r.mean()), r.std(ddof=1) / math.sqrt(N) / r.mean())
    with open(os.path.join(HERE, "cfg3_het_is_evidence.txt"), "w") as f:
        f.write("# exact log-evidence of the heterodyned likelihood on config 1 (H1, 4 s) by importance sampling\n")
        f.write(f"# of the FP64 oracle: fiducial = injection, {NB} bins; draws={N} seed={SEED}\n")
        f.write("# spacing logz err\n")
        for k in ("geometric", "phase", "full"):
            f.write(f"{k} {out[k][0]:.6f} {out[k][1]:.6f}\n")
    print(out)


if __name__ == "__main__":
    main()
