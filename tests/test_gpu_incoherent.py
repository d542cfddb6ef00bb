"""GPU parity of the incoherent modes (PONDER Sec. 3.4: AID and CID) against the
FP64 oracle, through the C ABI: filterbank, channel delays, dedispersed series
and folded profile, on seeded streams with a dispersed pulsar and ragged tails.
Tolerance: relative L2 1e-5 for the FP32 arrays (single-precision FFTs of up to
4096 points and sums of up to 2048 channels), exact for delays, ranges and hits."""
import numpy as np
import pytest

from oracle import incoherent as inc
from paper_1503_01405_gb300 import pond, synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _stream(n, seed, dm, bw):
    spec = synth.StreamSpec(n=n, seed=seed, dm=dm, period=0.02, duty=0.05, snr=200.0, bw=bw)
    return synth.make_stream(spec)


def _input(p, n, seed):
    if p.channels == 1:
        return _stream(n, seed, p.dm, p.bw)
    a, b = _stream(n, seed, p.dm, p.bw), _stream(n, seed + 100, p.dm, p.bw)
    inter = np.empty(2 * n, np.int8)
    inter[0::2], inter[1::2] = a, b
    return inter


def _engine(p):
    return pond.Incoherent(p.f0, p.bw, p.fs, p.dm, p.nchan, p.nint, p.nbins, p.period, mode=p.mode,
                           input_channels=p.channels)


def _compare(e, p, raw):
    import torch
    r = inc.run(p, raw)
    e.run_tensor(torch.from_numpy(raw).cuda())
    F = e.filterbank()
    D, t_first = e.series()
    s, h = e.profile()
    assert F.shape == r.F.T.shape
    if F.size:
        assert rel(F, r.F.T) <= TOL
    assert t_first == r.t_first and len(D) == len(r.D)
    if len(D):
        assert rel(D, r.D) <= TOL
        assert rel(s, r.prof_sum) <= TOL
    assert np.array_equal(h, r.prof_hits)
    return F, D, s, h


CASES = [  # nchan, nint, mode, channels, bw, dm, input samples
    (1024, 1, inc.AID, 1, 16.0, 10.0, (1 << 21) + 333),
    (256, 4, inc.AID, 2, 16.0, 5.0, (1 << 21) + 7),
    (64, 16, inc.CID, 2, -16.0, 3.0, 1 << 21),
    (2048, 2, inc.AID, 1, 16.0, 2.0, (1 << 22) + 1),
    (512, 1, inc.CID, 2, 16.0, 1.0, (1 << 20) + 4096 + 10),
    (128, 256, inc.AID, 1, -16.0, 20.0, 1 << 22),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"nch{c[0]}_nint{c[1]}_{'CID' if c[2] else 'AID'}{c[3]}_bw{c[4]:+.0f}")
def test_incoherent_matches_oracle(case):
    nchan, nint, mode, ch, bw, dm, n = case
    p = inc.make_plan(326.5, bw, 32e6, dm, nchan, nint, mode, ch, 64, 0.02)
    raw = _input(p, n, seed=11)
    with _engine(p) as e:
        assert np.array_equal(e.delays(), inc.channel_delays(p))
        F, D, s, h = _compare(e, p, raw)
        info = e.info()
        assert info["T"] == F.shape[0] and info["n_out"] == len(D)
        assert info["launches"] == (4 if len(D) else 1)
        # a second run of the same input gives the same bits
        import torch
        e.run_tensor(torch.from_numpy(raw).cuda())
        assert np.array_equal(e.filterbank(), F)
        D2, _ = e.series()
        assert np.array_equal(D2, D)
        assert np.array_equal(e.profile()[0], s)


def test_incoherent_buffers_grow_and_shrink():
    """Short, long, short inputs on one handle: each run matches the oracle."""
    p = inc.make_plan(326.5, 16.0, 32e6, 4.0, 256, 2, inc.AID, 1, 32, 0.02)
    with _engine(p) as e:
        for n in ((1 << 19) + 99, (1 << 21) + 5, 1 << 19):
            _compare(e, p, _stream(n, 5, p.dm, p.bw))


def test_incoherent_empty_and_short_inputs():
    """Less than one spectrum: nothing at all; fewer samples than the delay span:
    a filterbank but no series, and an empty profile."""
    import torch
    p = inc.make_plan(326.5, 16.0, 32e6, 30.0, 1024, 1, inc.AID, 1, 16, 0.02)
    with _engine(p) as e:
        e.run_tensor(torch.zeros(1000, dtype=torch.int8, device="cuda"))
        assert e.filterbank().shape == (0, 1024)
        assert len(e.series()[0]) == 0
        assert e.info()["launches"] == 0 and e.profile()[1].sum() == 0
        e.run_device(0, 0)
        assert e.info()["T"] == 0
        F, D, _, h = _compare(e, p, _stream(2048 * 300, 3, p.dm, p.bw))
        assert F.shape == (300, 1024) and len(D) == 0 and h.sum() == 0


def test_incoherent_argument_errors():
    import torch
    p = inc.make_plan(326.5, 16.0, 32e6, 1.0, 64, 1, inc.AID, 2, 16, 0.02)
    with _engine(p) as e:
        t = torch.zeros(4096 + 16, dtype=torch.int8, device="cuda")
        with pytest.raises(pond.PondError) as ei:
            e.run_device(t.data_ptr() + 1, 4096)          # not 16-byte aligned
        assert ei.value.name == "ARG"
        with pytest.raises(pond.PondError) as ei:
            e.run_device(t.data_ptr(), 4095)              # splits an N / S pair
        assert ei.value.name == "ARG"
    for kw, name in ((dict(mode=pond.POND_INCOH_CID, input_channels=1), "ARG"), (dict(nchan=32), "NCHAN"),
                     (dict(nchan=4096), "NCHAN"), (dict(nint=3), "ARG"), (dict(nbins=0), "ARG"),
                     (dict(fs=31e6), "ARG")):
        a = dict(f0=326.5, bw=16.0, fs=32e6, dm=1.0, nchan=64, nint=1, nbins=16, period=0.02)
        a.update(kw)
        with pytest.raises(pond.PondError) as ei:
            pond.Incoherent(**a)
        assert ei.value.name == name
