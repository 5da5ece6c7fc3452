"""The allocation-free likelihood entry point (swig_loglike_batch_noalloc).

It serves callers that cannot allocate device memory while running (a
pre-reserved real-time loop, an allocator-free host runtime, a process whose
device memory belongs to another framework).  This file runs last so that a
failure here leaves every other test already run.  It checks, through the
C-ABI, that two calls in a row reproduce the allocating entry point's results
within the likelihood tolerance, and that oversized batches are refused.
"""
import numpy as np
import pytest

import swig_inputs as si
from oracle import events, physics

pytestmark = pytest.mark.gpu

swig = pytest.importorskip("paper_2607_28265_gb300.swig")
torch = pytest.importorskip("torch")


def test_noalloc_matches_allocating_entry_point_twice():
    wl = si.config2()
    ev, th = events.build_event(wl)
    ctx = swig.context_for_workload(wl, ev.data, ev.psds, ev.gmst)
    ctx.set_sampler(nlive=1000, nrep=100, precision=swig.PREC_MIXED)
    rng = np.random.default_rng(31)
    thetas = np.array([physics.prior_transform(rng.random(len(wl.sampled())), wl.params)[0] for _ in range(64)])
    want = ctx.loglike_batch(thetas)  # also prepares the context (allocating)
    t_dev = torch.from_numpy(thetas).cuda()
    stream = torch.cuda.Stream()
    for _ in range(2):
        out = torch.full((len(thetas),), float("nan"), dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            ctx.loglike_batch_noalloc(t_dev.data_ptr(), len(thetas), out.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.abs(got - want) <= 1e-6 * np.abs(want) + 1e-6)
    # a batch beyond the fixed scratch is refused, without launching anything
    big = torch.zeros((100000, 13), dtype=torch.float64, device="cuda")
    out = torch.zeros(100000, dtype=torch.float64, device="cuda")
    with pytest.raises(swig.SwigError) as e:
        ctx.loglike_batch_noalloc(big.data_ptr(), big.shape[0], out.data_ptr(), 0)
    assert e.value.code == swig.SWIG_E_ARG
    assert "split the batch" in str(e.value)
    ctx.close()


def test_noalloc_requires_prepared_context():
    wl = si.config1()
    ev, th = events.build_event(wl)
    ctx = swig.context_for_workload(wl, ev.data, ev.psds, ev.gmst)
    ctx.set_sampler(nlive=100, nrep=10, precision=swig.PREC_MIXED)
    t_dev = torch.from_numpy(th[None, :].copy()).cuda()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(swig.SwigError) as e:
        ctx.loglike_batch_noalloc(t_dev.data_ptr(), 1, out.data_ptr(), 0)
    assert e.value.code == swig.SWIG_E_STATE
    ctx.close()
