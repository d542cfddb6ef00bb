"""Pins of the incoherent-mode oracle (PONDER Sec. 3.4: FFT filterbank, AID / CID
detection, integration, Eq. 3 channel delays, fold) against what the paper and
the mathematics fix: brute-force DFT sums, a tone's closed form, the linearity
that ties AID to CID, the Eq. 3 delays with the paper's printed constant, a
hand-built dispersed impulse, and the generator's dispersed pulsar."""
import numpy as np
import pytest

from oracle import incoherent as inc
from oracle import pcd
from paper_1503_01405_gb300 import synth

ORT = dict(f0=326.5, bw=16.0, fs=32e6)


def _plan(**kw):
    a = dict(ORT, dm=0.0, nchan=8, nint=1, mode=inc.AID, channels=1, nbins=16, period=0.01)
    a.update(kw)
    return inc.make_plan(**a)


def _brute_spectrum(block):
    """X[k] = sum_n x[n] exp(-2 pi i k n / R) by direct summation, k < R / 2."""
    R = len(block)
    n = np.arange(R)
    return np.array([np.sum(block * (np.cos(2 * np.pi * k * n / R) - 1j * np.sin(2 * np.pi * k * n / R)))
                     for k in range(R // 2)])


def test_filterbank_matches_direct_sums():
    """AID (one stream, two halves added) and CID against direct DFT sums,
    integrated by hand; the ragged tail that fills no output sample is unused."""
    rng = np.random.default_rng(3)
    nchan, nint, T = 8, 2, 3
    R = 2 * nchan
    n = rng.integers(-128, 128, R * nint * T + 5).astype(np.int8)
    s = rng.integers(-128, 128, R * nint * T + 5).astype(np.int8)
    inter = np.empty(2 * n.size, np.int8)
    inter[0::2], inter[1::2] = n, s
    want_one = np.zeros((nchan, T))
    want_two = np.zeros((nchan, T))
    want_cid = np.zeros((nchan, T))
    for t in range(T):
        for i in range(nint):
            b = slice((t * nint + i) * R, (t * nint + i + 1) * R)
            xn, xs = _brute_spectrum(n[b].astype(float)), _brute_spectrum(s[b].astype(float))
            xa = _brute_spectrum(n[b].astype(float) + s[b].astype(float))
            want_one[:, t] += np.abs(xn) ** 2
            want_two[:, t] += np.abs(xa) ** 2
            want_cid[:, t] += (xn * np.conj(xs)).real
    got_one = inc.filterbank(_plan(nint=nint), n)
    got_two = inc.filterbank(_plan(nint=nint, channels=2), inter)
    got_cid = inc.filterbank(_plan(nint=nint, channels=2, mode=inc.CID), inter)
    for got, want in ((got_one, want_one), (got_two, want_two), (got_cid, want_cid)):
        assert got.shape == (nchan, T)
        assert np.allclose(got, want, rtol=0, atol=1e-9 * np.abs(want).max())


@pytest.mark.parametrize("k0", [1, 5, 31])
def test_tone_lands_in_its_channel(k0):
    """x[n] = A cos(2 pi k0 n / R + theta): |X[k0]|^2 = (A R / 2)^2 per spectrum,
    nothing in any other channel."""
    nchan, nint, T = 32, 4, 3
    R = 2 * nchan
    A, theta = 7.0, 0.4
    x = A * np.cos(2 * np.pi * k0 * np.arange(R * nint * T) / R + theta)
    F = inc.filterbank(_plan(nchan=nchan, nint=nint), x)
    want = nint * (A * R / 2) ** 2
    assert np.allclose(F[k0], want, rtol=1e-12)
    others = np.delete(F, k0, axis=0)
    assert np.abs(others).max() < 1e-18 * want


def test_aid_equals_halves_plus_twice_cid():
    """Linearity of the DFT: |X_N + X_S|^2 = |X_N|^2 + |X_S|^2 + 2 Re(X_N conj X_S),
    so AID of the added halves is the halves' own AID plus twice their CID."""
    rng = np.random.default_rng(4)
    n = rng.integers(-128, 128, 64 * 40).astype(np.int8)
    s = rng.integers(-128, 128, 64 * 40).astype(np.int8)
    inter = np.empty(2 * n.size, np.int8)
    inter[0::2], inter[1::2] = n, s
    kw = dict(nchan=32, nint=2)
    aid = inc.filterbank(_plan(channels=2, **kw), inter)
    cid = inc.filterbank(_plan(channels=2, mode=inc.CID, **kw), inter)
    fn = inc.filterbank(_plan(**kw), n)
    fs_ = inc.filterbank(_plan(**kw), s)
    assert np.allclose(aid, fn + fs_ + 2 * cid, rtol=0, atol=1e-9 * aid.max())


def test_cid_of_equal_and_opposite_halves():
    """Correlated halves: CID(N, N) is N's power, CID(N, -N) its negative; AID of
    opposite halves is zero (they cancel when added in phase)."""
    rng = np.random.default_rng(5)
    n = rng.integers(-127, 128, 64 * 10).astype(np.int8)
    same = np.repeat(n, 2)
    opp = np.empty(2 * n.size, np.int8)
    opp[0::2], opp[1::2] = n, -n
    kw = dict(nchan=32, nint=1)
    pn = inc.filterbank(_plan(**kw), n)
    assert np.allclose(inc.filterbank(_plan(channels=2, mode=inc.CID, **kw), same), pn, rtol=1e-12)
    assert np.allclose(inc.filterbank(_plan(channels=2, mode=inc.CID, **kw), opp), -pn, rtol=1e-12)
    assert np.all(inc.filterbank(_plan(channels=2, **kw), opp) == 0)


@pytest.mark.parametrize("bw", [16.0, -16.0])
def test_delays_follow_eq3(bw):
    """d_k t_s against Eq. 3 with the paper's printed 4.15e6 ms constant, rescaled to
    the oracle's K (the two agree to 0.01 %): within half a sample plus that
    difference.  Channels below f0 are read later, channels above earlier; the
    channel at f0 itself has no delay."""
    p = _plan(bw=bw, dm=26.8, nchan=1024, nint=1)
    d = inc.channel_delays(p)
    f = inc.channel_freqs(p)
    eq3_s = np.array([pcd.channel_delay_ms(p.f0, fk, p.dm) for fk in f]) * 1e-3
    assert np.all(np.abs(d * p.ts - (-eq3_s)) <= p.ts / 2 + 3e-4 * np.abs(eq3_s) + 1e-12)
    assert d[512] == 0 and f[512] == p.f0
    lower = f < p.f0
    assert np.all(d[lower] > 0) and np.all(d[~lower] <= 0)
    assert np.all(np.diff(d) <= 0) if bw > 0 else np.all(np.diff(d) >= 0)
    # the delay span is the dispersion sweep between the lowest and highest
    # channel frequencies (the coherent pins' closed form), to a sample
    fmin, fmax = f.min(), f.max()
    sweep_s = pcd.band_smear_s((fmin + fmax) / 2, fmax - fmin, p.dm)
    assert abs((d.max() - d.min()) * p.ts - sweep_s) <= p.ts


def test_dedisperse_aligns_a_dispersed_impulse():
    """A filterbank holding one impulse per channel at t0 + (its delay) dedisperses
    to a single sample of height nchan at t0."""
    p = _plan(dm=40.0, nchan=64, nint=8)
    T, t0 = 8000, 4000            # delays span about -2240 .. 2475 samples of 32 us
    f = p.f0 - 8.0 + np.arange(64) * (16.0 / 64)
    arrive_s = pcd.K_DM * p.dm * (f ** -2.0 - p.f0 ** -2.0)
    dk = np.floor(arrive_s / p.ts + 0.5).astype(int)
    F = np.zeros((64, T))
    F[np.arange(64), t0 + dk] = 1.0
    D, t_first = inc.dedisperse(p, F)
    assert t_first == -dk.min()
    assert len(D) == T - dk.max() - t_first
    assert D[t0 - t_first] == 64
    assert np.count_nonzero(D) == 1


def test_output_range_edges():
    """No output when the stream is no longer than the delay span; exactly one
    when it is one sample longer; less than one spectrum gives nothing at all."""
    p = _plan(dm=20.0, nchan=64, nint=4)
    span = inc.delay_span_samples(p)
    F = np.ones((64, span))
    assert len(inc.dedisperse(p, F)[0]) == 0
    D, _ = inc.dedisperse(p, np.ones((64, span + 1)))
    assert len(D) == 1 and D[0] == 64
    r = inc.run(p, np.zeros(127, np.int8))
    assert r.F.shape == (64, 0) and len(r.D) == 0 and r.prof_hits.sum() == 0


def test_plan_rejects_invalid_forms():
    with pytest.raises(inc.IncoPlanError):
        _plan(mode=inc.CID, channels=1)
    with pytest.raises(inc.IncoPlanError):
        _plan(nchan=48)
    with pytest.raises(inc.IncoPlanError):
        _plan(nint=3)
    with pytest.raises(ValueError):
        inc.filterbank(_plan(channels=2), np.zeros(7, np.int8))


def test_generator_pulsar_recovered_at_its_phase():
    """The generator's pulsar (dispersed by the exact ISM response, pinned to the
    closed-form delay elsewhere), dedispersed incoherently at its DM, folds to a
    peak at its phase; left dispersed (DM 0) the sweep over the band (19 ms of a
    50 ms period) flattens the peak several-fold."""
    spec = synth.StreamSpec(n=1 << 23, seed=9, dm=5.0, period=0.05, duty=0.04, snr=80.0)
    x = synth.make_stream(spec)
    kw = dict(nchan=256, nint=4, nbins=64, period=0.05)
    r = inc.run(_plan(dm=5.0, **kw), x)
    r0 = inc.run(_plan(dm=0.0, **kw), x)

    def excess(res):
        prof = res.prof_sum / np.maximum(res.prof_hits, 1)
        return prof - np.median(prof), int(np.argmax(prof))

    e, peak = excess(r)
    e0, _ = excess(r0)
    assert peak in range(30, 34)                # phase 0.5 of 64 bins
    assert e.max() > 4 * e0.max()


def test_eq2_smear_of_the_1024_channel_filterbank():
    """Eq. 2 for the filterbank's own channels (1024 over 16 MHz, per unit DM):
    the channel at the band centre and the lowest channel bracket the 3.8 us the
    paper quotes, and the smear falls with frequency across the band."""
    import os
    golden = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_numbers.txt")
    quoted = None
    for line in open(golden):
        if line.startswith("eq2_smear_1024ch_per_dm"):
            quoted = float(line.split()[1])
    p = _plan(dm=1.0, nchan=1024)
    smear_us = np.array([inc.residual_smear_ms(p, k) for k in range(1024)]) * 1e3
    assert smear_us[512] < quoted < smear_us[0]
    assert np.all(np.diff(smear_us) < 0)
