"""Element-wise parity checks of GPU results against the oracle, with the
measured error of every check recorded for the session summary.

check(name, got, want, rtol, atol) asserts |got - want| <= rtol |want| + atol
element by element and records the largest absolute error, the largest error
relative to |want| and the largest ratio of error to tolerance.  The summary
is printed at the end of the pytest session and, when the environment
variable SWIG_PARITY_REPORT names a file, written there as JSON lines;
note(name, **values) records other measured values the same way.
"""
import numpy as np

RECORDS = []
NOTES = []


def note(name, **values):
    """Record measured values of a check that is not element-wise (p-values,
    evidence differences) for the session summary."""
    NOTES.append(dict(name=name, **values))


def check(name, got, want, rtol, atol):
    got = np.atleast_1d(np.asarray(got, dtype=np.float64))
    want = np.atleast_1d(np.asarray(want, dtype=np.float64))
    assert got.shape == want.shape, (name, got.shape, want.shape)
    err = np.abs(got - want)
    tol = rtol * np.abs(want) + atol
    both_inf = np.isneginf(got) & np.isneginf(want)
    err = np.where(both_inf, 0.0, err)
    rec = dict(name=name, n=int(err.size), max_abs=float(np.max(err)) if err.size else 0.0,
               max_rel=float(np.max(err / np.maximum(np.abs(want), 1e-300))) if err.size else 0.0,
               max_frac_of_tol=float(np.max(err / tol)) if err.size else 0.0, rtol=rtol, atol=atol)
    RECORDS.append(rec)
    bad = ~(err <= tol)
    assert not np.any(bad), (name, rec, np.flatnonzero(bad)[:8])
    return err
