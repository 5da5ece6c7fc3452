"""The allocation-free likelihood entry point (swig_loglike_batch_noalloc).

It serves callers that cannot allocate device memory while running (a
pre-reserved real-time loop, an allocator-free host runtime, a process whose
device memory belongs to another framework).  This file runs last so that a
failure here leaves every other test already run.  It checks, through the
C-ABI, that two calls in a row reproduce the allocating entry point's results
bit for bit (both launch the same kernels with the same work split), that the
second call takes no device memory, and that oversized batches are refused.
"""
import numpy as np
import pytest

import swig_inputs as si
from oracle import events, physics
from oracle import likelihood as L

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
    # a few values straight from the FP64 oracle, within the parity bound
    ref = np.array([L.loglike(ev, t) for t in thetas[:3]])
    assert np.all(np.abs(want[:3] - ref) <= 1e-6 * np.abs(ref) + 1e-6)
    t_dev = torch.from_numpy(thetas).cuda()
    stream = torch.cuda.Stream()
    outs = [torch.full((len(thetas),), float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    for call, out in enumerate(outs):
        free0 = torch.cuda.mem_get_info()[0]
        with torch.cuda.stream(stream):
            ctx.loglike_batch_noalloc(t_dev.data_ptr(), len(thetas), out.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        got = out.cpu().numpy()
        # same launches, same work split, same data: bit for bit the allocating path
        assert np.array_equal(got, want), np.max(np.abs(got - want))
        if call == 1:  # the first call looked up the scratch address; the second takes no device memory
            assert free1 == free0
    # a batch beyond the fixed scratch is refused, without launching anything
    big = torch.zeros((100000, 13), dtype=torch.float64, device="cuda")
    out = torch.zeros(100000, dtype=torch.float64, device="cuda")
    with pytest.raises(swig.SwigError) as e:
        ctx.loglike_batch_noalloc(big.data_ptr(), big.shape[0], out.data_ptr(), 0)
    assert e.value.code == swig.SWIG_E_ARG
    assert "split the batch" in str(e.value)
    # a size whose byte counts would wrap around 2^64 is refused the same way
    with pytest.raises(swig.SwigError) as e:
        ctx.loglike_batch_noalloc(big.data_ptr(), (1 << 62) + 1, out.data_ptr(), 0)
    assert e.value.code == swig.SWIG_E_ARG
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
