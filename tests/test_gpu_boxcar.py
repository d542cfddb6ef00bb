"""Boxcar detector on the GPU vs the FP64 oracle: identical candidate lists.

Every S/N value is a chain of correctly rounded FP64 operations in the same
order on both sides, so trials, indices, widths and S/N values agree exactly.
"""
import numpy as np
import pytest

from oracle import boxcar as ob
from paper_1503_01405_gb300 import pond, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1503_01405_gb300 import build as pbuild
    pbuild.build()


def gpu_detect(block, thr=6.0):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(block, dtype=np.float32)).cuda()
    c = pond.boxcar(t.data_ptr(), block.shape[0], block.shape[1], block.shape[1], thr,
                    stream=torch.cuda.current_stream().cuda_stream)
    return [(x["trial"], x["index"], x["width"], x["snr"]) for x in c]


@pytest.mark.parametrize("ndm,n", [(1, 1), (3, 7), (8, 4096), (5, 10001), (20, 65536)])
def test_boxcar_matches_oracle(ndm, n):
    rng = np.random.default_rng(ndm * 1000 + n)
    block = (1000 + 30 * rng.standard_normal((ndm, n))).astype(np.float32)
    for k in range(min(6, n // 100)):           # boxes of several widths and heights
        d = int(rng.integers(ndm))
        w = int(2 ** rng.integers(0, 7))
        t = int(rng.integers(0, max(1, n - w)))
        block[d, t:t + w] += float(rng.uniform(20, 200))
    assert gpu_detect(block) == ob.detect(block)


def test_constant_and_even_odd_rows():
    block = np.stack([np.full(1000, 5.0), np.arange(1000, dtype=np.float64) % 7, np.r_[np.zeros(999), 100.0]])
    block = block.astype(np.float32)
    assert gpu_detect(block, thr=3.0) == ob.detect(block, threshold=3.0)


def test_candidates_from_a_batched_plan():
    dms = [0.0, 0.1, 0.2, 0.3, 0.4]
    spec = synth.StreamSpec(n=3_000_000, seed=41, dm=0.0, period=0.0, snr=0.0)
    pulses = [synth.Pulse(0.03, 0.2, 2e-4, 40.0), synth.Pulse(0.06, 0.35, 1e-4, 25.0)]
    x = synth.make_chunk(spec, pulses)
    with pond.Engine(326.5, 16.0, 32e6, 0.0, 1 << 16, 16, 1, 1.0, t_dec=8e-6, dms=dms) as e:
        e.push(x)
        e.flush()
        cands = e.candidates(6.0)
        T, C, j0 = e.timeseries()
    want = ob.detect(T)
    got = [(c["trial"], c["index"] - j0, c["width"], c["snr"]) for c in cands]
    assert got == want
    assert all(c["dm"] == dms[c["trial"]] for c in cands)
    # the brightest candidate sits at the pulse's DM and time
    best = max(cands, key=lambda c: c["snr"])
    assert best["trial"] == 2
    assert abs((best["index"] + best["width"] / 2) * 8e-6 - 0.03) < 1e-3
