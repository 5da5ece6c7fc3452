import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    import json

    try:
        import parity
    except ImportError:
        return
    if not parity.RECORDS and not parity.NOTES:
        return
    terminalreporter.write_sep("-", "parity against the oracle (largest error per check)")
    for r in parity.RECORDS:
        terminalreporter.write_line(
            f"{r['name']:<58} n={r['n']:<6} max|err|={r['max_abs']:.3e} max rel={r['max_rel']:.3e} "
            f"err/tol={r['max_frac_of_tol']:.3f}")
    for r in parity.NOTES:
        terminalreporter.write_line(json.dumps(r))
    path = os.environ.get("SWIG_PARITY_REPORT")
    if path:
        with open(path, "w") as f:
            for r in parity.RECORDS + parity.NOTES:
                f.write(json.dumps(r) + "\n")
