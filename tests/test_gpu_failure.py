"""Failure detection without a GPU fault.

The tensor-core stages wait for their MMAs with a wait bounded by the GPU's
global timer; when it expires the CTA skips further MMAs and the plan reports
POND_E_TIMEOUT.  Here a kernel waits on a barrier that nothing ever arrives on
(a flag nothing sets) with a short limit: the wait must give up by itself, the
status must reach the host, and the context must stay usable.
"""
import numpy as np
import pytest

from oracle import pcd
from paper_1503_01405_gb300 import pond, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1503_01405_gb300 import build as pbuild
    pbuild.build()


def test_bounded_wait_gives_up_and_context_survives():
    rc, waited = pond.check_bounded_wait(0.05)
    assert rc == pond.POND_E_TIMEOUT
    assert 0.05 <= waited < 1.0
    # the device still runs the engine, tensor-core stages included
    p = pcd.make_plan(326.5, 16.0, 32e6, 0.05, 1 << 14, 4, 64, 0.0123)
    x = synth.make_stream(synth.StreamSpec(n=4 * p.S + 999, seed=3, dm=p.dm, period=p.period, snr=60.0))
    r = pcd.run(p, x)
    with pond.Engine(p.f0, p.bw, p.fs, p.dm, p.nfft, p.nchan, p.nbins, p.period,
                     precision=pond.POND_SPLIT_BF16) as e:
        e.push(x)
        e.flush()
        s, h, _ = e.profile()
    assert np.array_equal(h, r.prof_hits)


def test_bounded_wait_argument_errors():
    rc, _ = pond.check_bounded_wait(0.0)
    assert rc == pond.POND_E_ARG
    rc, _ = pond.check_bounded_wait(11.0)
    assert rc == pond.POND_E_ARG
