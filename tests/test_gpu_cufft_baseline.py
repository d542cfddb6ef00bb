"""The cuFFT comparison path computes the same outputs as the oracle and the engine.

The comparison path (baseline/cufft_path.py: cuFFT R2C, inverse filter, batched
C2C inverse, detection, torch scatter-add fold and decimation) is timed beside
the engine in bench.py; this checks it is a like-for-like baseline.  Tolerance
as for the engine: relative L2 <= 1e-4 on profile and series, hits and counts
exact.
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


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


@pytest.mark.parametrize("cfg", [(1 << 16, 16, 0.3, 16.0, 128, 0.033), (1 << 18, 1, 0.5, -16.0, 256, 0.0317)])
def test_cufft_path_matches_oracle_and_engine(cfg):
    import torch
    from baseline.cufft_path import CufftPath
    nfft, nchan, dm, bw, nbins, period = cfg
    p = pcd.make_plan(326.5, bw, 32e6, dm, nfft, nchan, nbins, period)
    x = synth.make_stream(synth.StreamSpec(n=4 * p.S + p.nfft // 3 + 5, seed=nfft + 7, dm=dm, period=period,
                                           snr=60.0, duty=0.05, bw=bw))
    r = pcd.run(p, x)
    dev = torch.device("cuda", 0)
    cp = CufftPath(326.5, bw, 32e6, dm, nfft, nchan, nbins, period, 61.44e-6, dev)
    assert (cp.g.n_past, cp.g.n_fut, cp.g.S_c) == (p.n_past, p.n_fut, p.S_c)
    s, h, T, C, j0 = cp.run(torch.from_numpy(x).to(dev))
    assert np.array_equal(h.cpu().numpy(), r.prof_hits)
    assert np.array_equal(C.cpu().numpy(), r.ts_counts) and j0 == r.ts_first
    assert rel(s.cpu().numpy(), r.prof_sum) <= 1e-4
    assert rel(T.cpu().numpy(), r.ts) <= 1e-4
    with pond.Engine(326.5, bw, 32e6, dm, nfft, nchan, nbins, period) as e:
        e.push(x)
        e.flush()
        es, eh, _ = e.profile()
    assert np.array_equal(eh, h.cpu().numpy())
    assert rel(es, s.cpu().numpy()) <= 1e-4
