"""The seeded generator: Philox known answers, deviates, and the ISM sky model."""
import math
import os

import numpy as np
import pytest

from paper_1503_01405_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(t, 16) for t in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,want", _kat_rows())
def test_philox_known_answers(ctr, key, want):
    out = synth.philox4x32_10([np.array([c], dtype=np.uint64) for c in ctr], key)
    assert [int(o[0]) for o in out] == want


def test_words_chunk_independent():
    a = synth.random_words(7, 3, 0, 1001)
    b = synth.random_words(7, 3, 333, 100)
    assert np.array_equal(a[333:433], b)


def test_gaussian_moments_and_chunks():
    z = synth.gaussian(11, 0, 0, 400_000)
    assert abs(z.mean()) < 5 * 1 / math.sqrt(len(z))
    assert abs(z.var() - 1) < 0.01
    # fourth moment of a standard normal is 3
    assert abs(np.mean(z ** 4) - 3) < 0.06
    assert np.allclose(synth.gaussian(11, 0, 12345, 77), z[12345:12345 + 77])
    assert np.allclose(synth.gaussian(11, 0, 12346, 77), z[12346:12346 + 77])


def test_quantise_rounds_half_even_and_clips():
    q = synth.quantise(np.array([0.5, 1.5, -0.5, -2.5, 300.0, -300.0, 126.6]))
    assert q.tolist() == [0, 2, 0, -2, 127, -127, 127]
    assert q.dtype == np.int8


def _envelope_peak(x, fs, f_lo_bb, f_hi_bb):
    """Time (samples) of the power peak of x band-limited to [f_lo_bb, f_hi_bb) MHz baseband."""
    X = np.fft.rfft(x)
    f = np.fft.rfftfreq(len(x), 1 / fs) * 1e-6
    X[(f < f_lo_bb) | (f >= f_hi_bb)] = 0
    env = np.abs(np.fft.ifft(np.concatenate([X, np.zeros(len(x) - len(X))]))) ** 2
    return float(np.sum(np.arange(len(x)) * env) / np.sum(env))


@pytest.mark.parametrize("bw", [16.0, -16.0])
def test_ism_delay_matches_closed_form(bw):
    """An impulse through the sky model arrives at f at t0 + K DM (f^-2 - f0^-2).

    This is the cold-plasma delay of Eq. 3 with K = 1/2.41e-4 s MHz^2; it pins
    the sign, the constant and the sideband mapping of the generator's H.
    """
    spec = synth.StreamSpec(n=1 << 17, dm=0.2, bw=bw)
    n = 1 << 18
    x = np.zeros(n)
    n0 = n // 2
    x[n0] = 1.0
    xd = synth.ism_disperse(x, spec)
    for b_lo in (1.0, 7.5, 14.0):
        b_hi = b_lo + 0.25
        t = _envelope_peak(xd, spec.fs, b_lo, b_hi)
        b_mid = 0.5 * (b_lo + b_hi)
        sky = spec.f0 - 8.0 + b_mid if bw > 0 else spec.f0 + 8.0 - b_mid
        want = n0 + synth.dispersion_delay(sky, spec.f0, spec.dm) * spec.fs
        assert abs(t - want) < 3.0, (b_lo, t, want)


def test_ism_is_all_pass():
    spec = synth.StreamSpec(n=4096, dm=1.0)
    x = synth.gaussian(3, 0, 0, 1 << 14)
    xd = synth.ism_disperse(x, spec)
    X, Xd = np.fft.rfft(x), np.fft.rfft(xd)
    inner = slice(1, len(X) - 1)
    assert np.allclose(np.abs(X[inner]), np.abs(Xd[inner]), rtol=1e-9, atol=1e-9)


def test_pulsar_amplitude_small_config():
    # A = S/N sqrt(2 / sum g^2); the small workload gives A of about 0.16
    a = synth.pulsar_amplitude(synth.SMALL)
    assert 0.15 < a < 0.17
    g = synth.pulse_shape(np.arange(synth.SMALL.n) / (synth.SMALL.fs * synth.SMALL.period) % 1.0,
                          synth.SMALL.duty, synth.SMALL.phase_c)
    direct = synth.SMALL.snr * math.sqrt(2.0 / np.sum(g * g))
    assert abs(direct / a - 1) < 0.05


def test_stream_is_int8_and_seeded():
    spec = synth.StreamSpec(n=1 << 16, dm=0.5, rfi_duty=0.01)
    a = synth.make_stream(spec)
    b = synth.make_stream(spec)
    assert a.dtype == np.int8 and np.array_equal(a, b)
    assert 18 < a.astype(np.float64).std() < 40
    assert a.min() >= -127 and a.max() <= 127
