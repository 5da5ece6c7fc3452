"""Write the oracle's nested-sampling posterior for the 4 s single-detector
workload (tests/golden/cfg1_oracle_posterior.csv).

Calls only the FP64 oracle (oracle/) and the seeded inputs (swig_inputs).
Run from the repository root:  python tests/golden/make_ns_reference.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import swig_inputs as si  # noqa: E402
from oracle import events, nested, physics  # noqa: E402
from oracle import likelihood as L  # noqa: E402

NLIVE, NREP, SEED = 400, 40, 4242


def main():
    wl = si.config1()
    ev, th = events.build_event(wl)
    ns = len(wl.sampled())
    blocks = {}
    for j, slot in enumerate(wl.sampled()):
        blocks.setdefault(wl.params[slot].block, []).append(j)
    blocks = [blocks[b] for b in sorted(blocks)]
    res = nested.run_nested(lambda u: L.loglike_u(ev, u), ns, blocks, NLIVE, NREP, steps_per_dim=5, rng=SEED)
    theta = physics.prior_transform(res["u"], wl.params)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cfg1_oracle_posterior.csv")
    cols = [si.PARAM_NAMES[s] for s in wl.sampled()]
    with open(out, "w") as f:
        f.write(f"# oracle NS, config 1 (H1, 4 s), nlive={NLIVE} nrep={NREP} seed={SEED}\n")
        f.write(f"# logz={res['logz']:.6f} logz_err={res['logz_err']:.6f} ess={res['ess']:.1f} "
                f"n_evals={res['n_evals']}\n")
        f.write(",".join(cols + ["logl", "logw"]) + "\n")
        for row, ll, lw in zip(theta[:, wl.sampled()], res["logl"], res["logw"]):
            f.write(",".join(f"{v:.12g}" for v in list(row) + [ll, lw]) + "\n")
    print(out, res["logz"], res["logz_err"], res["ess"])


if __name__ == "__main__":
    main()
