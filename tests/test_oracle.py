"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: a brute-force sum on a tiny
input, a closed form of the mathematics, an identity, or a number the paper
prints.  A dropped term, a wrong sign or index, a transposed operand or a
wrong constant in ``oracle.pcd`` fails at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import pcd
from paper_1503_01405_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ORT = dict(f0=326.5, bw=16.0, fs=32e6)


def _paper_numbers():
    out = {}
    with open(os.path.join(GOLDEN, "paper_numbers.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, value = line.split()[:2]
            out[name] = float(value)
    return out


PAPER = _paper_numbers()


# --- the DFT steps, by brute force on tiny inputs ----------------------------------

def _brute_segment(p, x):
    """v_c[m] from explicit double sums (the definitions, no FFT)."""
    N, L, M = p.nfft, p.L, p.M
    n = np.arange(N)
    X = np.array([np.sum(x * np.exp(-2j * np.pi * k * n / N)) for k in range(L)])
    step = p.fs / N * 1e-6
    half = abs(p.bw) / 2
    out = np.zeros((p.nchan, M), dtype=complex)
    sgn = 1.0 if p.bw > 0 else -1.0
    for k in range(L):
        f = k * step - half if p.bw > 0 else half - k * step
        phase = pcd.K_DM * 1e6 * p.dm * f * f / (p.f0 ** 2 * (p.f0 + f))
        Y = X[k] * complex(math.cos(2 * math.pi * phase), -sgn * math.sin(2 * math.pi * phase))
        c, j = divmod(k, M)
        for m in range(M):
            out[c, m] += Y * np.exp(2j * np.pi * j * m / M) / M
    return out


@pytest.mark.parametrize("nchan", [1, 2, 4])
@pytest.mark.parametrize("bw", [0.5, -0.5])
def test_segment_matches_brute_force(nchan, bw):
    p = pcd.make_plan(f0=1.0, bw=bw, fs=1e6, dm=2e-9, nfft=32, nchan=nchan, nbins=8,
                      period=1e-3)
    x = synth.gaussian(5, 0, 0, 32) * 20
    got = pcd.dedisperse_segment(p, x)
    want = _brute_segment(p, x)
    assert np.max(np.abs(got - want)) < 1e-10 * np.max(np.abs(want))
    # the chirp is not trivial at this DM: it moves the result
    q = pcd.make_plan(f0=1.0, bw=bw, fs=1e6, dm=0.0, nfft=32, nchan=nchan, nbins=8,
                      period=1e-3)
    assert np.max(np.abs(pcd.dedisperse_segment(q, x) - want)) > 1e-2 * np.max(np.abs(want))


# --- closed forms -------------------------------------------------------------------

def test_dm0_single_channel_identity():
    """DM = 0, nchan = 1: Re v[m] = x[2m] + (X[0] - X[N/2]) / N.

    Derived from the inverse real DFT: keeping bins 0..N/2-1 and inverting at
    half rate leaves the even samples except for half the DC and Nyquist terms.
    """
    p = pcd.make_plan(**ORT, dm=0.0, nfft=4096, nchan=1, nbins=16, period=1e-3)
    x = synth.gaussian(9, 0, 0, 4096) * 20
    v = pcd.dedisperse_segment(p, x)[0]
    X0 = np.sum(x)
    XN = np.sum(x * (-1.0) ** np.arange(4096))
    assert np.max(np.abs(v.real - (x[0::2] + (X0 - XN) / 4096))) < 1e-12 * 4096


@pytest.mark.parametrize("nchan,bw", [(1, 16.0), (4, 16.0), (8, -16.0)])
def test_tone_closed_form_across_segments(nchan, bw):
    """A tone cos(2 pi k0 n / N + theta) dedisperses to a closed form at every g.

    X has one line (A N/2) e^{i theta} at k0 < N/2, so sub-channel c0 = k0 // M
    carries v[g] = A nchan e^{i theta} e^{-i sgn 2 pi c(f_k0)} e^{2 pi i j0 g / M}
    (j0 = k0 % M, g global) and every other sub-channel is zero.  This fixes the
    chirp phase and sign, the channel mapping, the normalisation and the
    overlap-save bookkeeping of the global index g.
    """
    p = pcd.make_plan(f0=326.5, bw=bw, fs=32e6, dm=0.01, nfft=4096, nchan=nchan,
                      nbins=16, period=1e-3)
    k0 = (3 * p.L) // 7 + 5
    A, theta = 7.5, 0.3
    n_seg = 6
    n = n_seg * p.S + p.nfft
    x = synth.tone(n, k0, p.nfft, A, theta)
    r = pcd.run(p, x, want_voltages=True)
    f = (k0 * p.fs / p.nfft * 1e-6 - 8.0) if bw > 0 else (8.0 - k0 * p.fs / p.nfft * 1e-6)
    c = pcd.K_DM * 1e6 * p.dm * f * f / (p.f0 ** 2 * (p.f0 + f))
    sgn = 1.0 if bw > 0 else -1.0
    c0, j0 = divmod(k0, p.M)
    g = r.first_g + np.arange(r.voltages.shape[1])
    complete = g < n_seg * p.S_c + p.n_past          # outputs of whole segments
    want = A * nchan * np.exp(1j * theta) * np.exp(-1j * sgn * 2 * np.pi * (c - round(c))) \
        * np.exp(2j * np.pi * ((j0 * g) % p.M) / p.M)
    got = r.voltages[:, complete]
    assert np.max(np.abs(got[c0] - want[complete])) < 1e-9 * A * nchan
    others = np.delete(got, c0, axis=0)
    assert others.size == 0 or np.max(np.abs(others)) < 1e-9 * A * nchan
    assert r.first_g == p.n_past


def test_parseval_per_segment():
    """sum_c sum_m |v_c[m]|^2 = (1/M) sum_{k<N/2} |X_k|^2, with the right side from
    Parseval of the real DFT: sum_{k<N/2} |X_k|^2 = (N sum x^2 + X_0^2 - X_{N/2}^2) / 2.
    Holds because |H| = 1 (Sec. 3.7: a unity-gain phase filter).
    """
    for nchan in (1, 16):
        p = pcd.make_plan(**ORT, dm=0.1, nfft=1 << 15, nchan=nchan, nbins=16, period=1e-3)
        x = synth.gaussian(4, 0, 0, p.nfft) * 20
        v = pcd.dedisperse_segment(p, x)
        lhs = np.sum(np.abs(v) ** 2)
        X0 = np.sum(x)
        XN = np.sum(x * (-1.0) ** np.arange(p.nfft))
        rhs = (p.nfft * np.sum(x * x) + X0 ** 2 - XN ** 2) / 2 / p.M
        assert abs(lhs / rhs - 1) < 1e-12


@pytest.mark.parametrize("bw", [16.0, -16.0])
def test_dispersed_impulse_compresses_to_delta(bw):
    """An impulse dispersed by the sky model compresses back to one sample.

    The sky model is pinned to the closed-form delay in test_synth; here the
    oracle's inverse filter must undo it: the dedispersed power peaks at the
    impulse's own channel sample and holds most of the energy there.
    """
    dm = 0.05
    spec = synth.StreamSpec(n=1, dm=dm, bw=bw)
    n = 1 << 16
    x = np.zeros(n)
    n0 = 30000
    x[n0] = 1000.0
    xd = synth.ism_disperse(x, spec)
    # the sweep spans K DM (f_lo^-2 - f_hi^-2): energy of the dispersed stream is spread
    sweep = pcd.band_smear_s(326.5, 16.0, dm) * 32e6
    assert np.max(np.abs(xd)) < 0.05 * 1000.0
    p = pcd.make_plan(326.5, bw, 32e6, dm, 1 << 14, 1, 16, 1e-3)
    r = pcd.run(p, xd)
    g_peak = r.first_g + int(np.argmax(r.power))
    assert g_peak == n0 // 2
    # near-delta: the peak and its neighbours carry almost all of the power
    i = g_peak - r.first_g
    assert np.sum(r.power[i - 2:i + 3]) > 0.9 * np.sum(r.power)
    assert sweep > 2 * p.nfft / 2 / 8        # the sweep is many samples long


def test_overlap_geometry_matches_band_sweep():
    p = pcd.make_plan(**ORT, dm=26.8, nfft=1 << 24, nchan=64, nbins=1024, period=0.7145)
    sweep_ch = pcd.band_smear_s(326.5, 16.0, 26.8) / p.dtc
    assert p.n_past + p.n_fut - 2 < sweep_ch <= p.n_past + p.n_fut
    assert p.S == 2 * p.nchan * p.S_c
    assert p.dtc == 4e-6


# --- fold and decimation -----------------------------------------------------------

def _plan_fold(nbins, period, nchan=1):
    return pcd.make_plan(**ORT, dm=0.0, nfft=1 << 12, nchan=nchan, nbins=nbins,
                         period=period)


def test_fold_period_equal_nbins_samples():
    """P = nbins * dtc exactly: bin(g) = g mod nbins, so every bin is exact."""
    nbins = 64
    p = _plan_fold(nbins, 64 * (2.0 / 32e6))
    assert p.inc == 1.0 / 64
    P = synth.uniform(2, 0, 0, 10_000) * 5
    g0 = 37
    s, h = pcd.fold(p, P, g0)
    g = np.arange(g0, g0 + len(P))
    for b in range(nbins):
        sel = (g % nbins) == b
        assert h[b] == np.count_nonzero(sel)
        assert abs(s[b] - np.sum(P[sel])) < 1e-9


def test_fold_cosine_profile_closed_form():
    """P[g] = 1 + a cos(2 pi g / (q nbins)) with period q nbins samples.

    Bin b averages q consecutive samples: mean = 1 + a / q * sum_i cos(2 pi (bq+i)/(q nbins))
    = 1 + a / q * Re[e^{i w bq} (1 - e^{i w q}) / (1 - e^{i w})], w = 2 pi / (q nbins).
    """
    nbins, q, a = 32, 8, 0.4
    p = _plan_fold(nbins, q * nbins * (2.0 / 32e6))
    P = 1 + a * np.cos(2 * np.pi * np.arange(q * nbins * 10) / (q * nbins))
    s, h = pcd.fold(p, P, 0)
    w = 2 * np.pi / (q * nbins)
    b = np.arange(nbins)
    want = 1 + a / q * np.real(np.exp(1j * w * b * q) * (1 - np.exp(1j * w * q)) / (1 - np.exp(1j * w)))
    assert np.all(h == 10 * q)
    assert np.max(np.abs(s / h - want)) < 1e-12


def test_fold_constant_power_and_conservation():
    p = _plan_fold(1024, 0.7145, nchan=64)
    P = np.full(500_000, 3.25)
    s, h = pcd.fold(p, P, 12_326)
    assert h.sum() == len(P)
    assert np.allclose(s[h > 0] / h[h > 0], 3.25, rtol=0, atol=1e-12)
    # bins cover 0.7145 / 1024 / 4e-6 = 174.4 samples: all hits within one of that
    assert h.min() >= 174 * 2 and h.max() <= 175 * 3


def test_decimation_rational_bins():
    """t_dec = 61.44 us at 4 us channel samples: D = 15.36 = 384/25.

    In each run of 384 samples there are 25 output samples, 9 of 16 and 16 of 15.
    """
    p = pcd.make_plan(**ORT, dm=0.0, nfft=1 << 12, nchan=64, nbins=16, period=1.0,
                      t_dec_s=61.44e-6)
    assert p.dec == Fraction(384, 25)
    P = synth.uniform(3, 0, 0, 384 * 4) + 1
    T, C, j0 = pcd.decimate(p, P, 0)
    assert j0 == 0 and len(T) == 100
    assert np.all(C.reshape(4, 25).sum(axis=1) == 384)
    assert np.count_nonzero(C == 16) == 36 and np.count_nonzero(C == 15) == 64
    assert abs(T.sum() - P.sum()) < 1e-9
    first = [math.ceil(j * Fraction(384, 25)) for j in range(100)]
    assert np.allclose(T, [P[first[j]:first[j] + C[j]].sum() for j in range(100)])


def test_decimation_offset_start():
    p = pcd.make_plan(**ORT, dm=0.0, nfft=1 << 12, nchan=1, nbins=16, period=1.0,
                      t_dec_s=1e-6)
    assert p.dec == 16
    P = np.ones(100)
    T, C, j0 = pcd.decimate(p, P, 37)
    assert j0 == 2 and C[0] == 11 and C[1] == 16 and C.sum() == 100


# --- the numbers the paper prints --------------------------------------------------

def test_constants_match_paper():
    assert abs(pcd.K_DM * 1e3 / PAPER["eq3_constant"] - 1) < 2e-3
    assert abs(1 / pcd.K_DM / PAPER["eq1_constant"] - 1) < 1e-12
    assert abs(2 * pcd.K_DM / PAPER["eq4_prefactor_over_pi"] - 1) < 1e-3


def test_eq2_residual_smear_per_dm():
    """Eq. 2 for 1024 channels over 16 MHz, per unit DM: 3.73 us at 326.5 MHz and
    4.01 us at the band's low edge; the paper quotes 3.8 us."""
    v_mid = pcd.residual_smear_ms(16.0 / 1024, 1.0, 326.5) * 1e3
    v_lo = pcd.residual_smear_ms(16.0 / 1024, 1.0, 318.5) * 1e3
    assert abs(v_mid - 3.73) < 0.01 and abs(v_lo - 4.01) < 0.01
    assert v_mid < PAPER["eq2_smear_1024ch_per_dm"] < v_lo


def test_max_dm_with_paper_fft_length():
    """N = 2^27 carries DM 130 at 326.5 MHz / 16 MHz (Sec. 3.7); 2^23 does not."""
    nmax = int(PAPER["pcd_max_nfft"])
    p = pcd.make_plan(**ORT, dm=PAPER["pcd_max_dm"], nfft=nmax, nchan=1, nbins=256, period=1.0)
    assert p.S_c > 0
    with pytest.raises(pcd.PlanError) as e:
        pcd.make_plan(**ORT, dm=130.0, nfft=1 << 23, nchan=1, nbins=256, period=1.0)
    assert e.value.code == "NFFT"
    assert abs(pcd.band_smear_s(326.5, 16.0, 130.0) - 0.4965) < 1e-3


def test_base_resolution():
    p = pcd.make_plan(**ORT, dm=3.0, nfft=1 << 21, nchan=1, nbins=256, period=0.253)
    assert p.dtc * 1e9 == PAPER["base_resolution"]


@pytest.mark.parametrize("kw,code", [
    (dict(nfft=3000), "NFFT"),
    (dict(nfft=1 << 10, dm=3.0), "NFFT"),
    (dict(nchan=3), "NCHAN"),
    (dict(nchan=1 << 12, nfft=1 << 12), "NCHAN"),
    (dict(dm=-1.0), "ARG"),
    (dict(period=0.0), "ARG"),
    (dict(fs=31e6), "ARG"),
    (dict(nbins=0), "ARG"),
])
def test_plan_errors(kw, code):
    args = dict(**ORT, dm=0.5, nfft=1 << 16, nchan=4, nbins=64, period=0.1)
    args.update(kw)
    with pytest.raises(pcd.PlanError) as e:
        pcd.make_plan(**args)
    assert e.value.code == code


# --- the streaming rules -----------------------------------------------------------

def test_stream_edges_and_segment_count():
    p = pcd.make_plan(**ORT, dm=0.01, nfft=4096, nchan=4, nbins=16, period=1e-3)
    n = 5 * p.S + 1234
    x = synth.make_stream(synth.StreamSpec(n=n, dm=0.0, period=0.0))
    r = pcd.run(p, x)
    g_end = n // (2 * p.nchan) - p.n_fut
    assert r.first_g == p.n_past
    assert len(r.power) == g_end - p.n_past
    assert r.prof_hits.sum() == len(r.power) and r.ts_counts.sum() == len(r.power)


def test_selected_outputs_match_full_run():
    p = pcd.make_plan(**ORT, dm=0.05, nfft=1 << 14, nchan=2, nbins=16, period=1e-3)
    x = synth.make_stream(synth.StreamSpec(n=6 * p.S, dm=0.05, period=1e-3, snr=30))
    r = pcd.run(p, x, want_voltages=True)
    g = np.array([r.first_g, r.first_g + 1, r.first_g + p.S_c - 1, r.first_g + p.S_c,
                  r.first_g + 3 * p.S_c + 17])
    V, P = pcd.dedisperse_at(p, x, g)
    assert np.allclose(V, r.voltages[:, g - r.first_g], rtol=0, atol=1e-9)
    assert np.allclose(P, r.power[g - r.first_g], rtol=1e-12)


@pytest.mark.slow
def test_pulsar_recovered_small_workload():
    """The small workload (2^23 samples, DM 3, P 0.253 s, S/N 50 over the fold):
    the dedispersed, folded profile shows the pulse at its phase with a
    matched-filter S/N near 50 (statistical, fixed seed)."""
    x = synth.make_stream(synth.SMALL)
    p = pcd.make_plan(**ORT, dm=3.0, nfft=1 << 21, nchan=1, nbins=256, period=0.253)
    r = pcd.run(p, x)
    prof = r.prof_sum / np.maximum(r.prof_hits, 1)
    phase = (np.arange(256) + 0.5) / 256
    tmpl = synth.pulse_shape(phase, 0.03, 0.5)
    hit = r.prof_hits > 0      # 2^23 samples cover slightly less than one period
    off = (tmpl < 1e-3) & hit
    mu = np.mean(prof[off])
    # per-bin noise of a mean of |v|^2 (complex Gaussian: std = mean / sqrt(hits))
    sig = mu / np.sqrt(r.prof_hits[hit])
    t, d = tmpl[hit], (prof - mu)[hit]
    snr = np.sum(t * d / sig ** 2) / np.sqrt(np.sum(t ** 2 / sig ** 2))
    assert int(np.argmax(prof)) in range(124, 132)
    assert 40 < snr < 60, snr


# --- the fold with a polynomial phase model (replacing the constant period) -------

def test_phase_model_fold_is_the_constant_period_off_bin_edges():
    """A model phi = tau / P (t_ref 0) bins every sample as the constant-period
    rule does, except samples within 1e-9 of a bin edge (the two phases round
    differently: (g dtc)(1/P) against g (dtc/P)), which move by one bin; the
    fold's histogram is that of the model's bins."""
    from oracle import stack
    P = 0.0123457
    p0 = pcd.make_plan(**ORT, dm=0.0, nfft=1 << 12, nchan=4, nbins=64, period=P)
    p1 = pcd.make_plan(**ORT, dm=0.0, nfft=1 << 12, nchan=4, nbins=64, period=P, phase=(0.0, [0.0, 1.0 / P]))
    g0 = 12345
    g = np.arange(g0, g0 + 400_000, dtype=np.int64)
    x = g.astype(np.float64) * p0.inc
    fr = (x - np.floor(x)) * 64
    b0 = np.minimum(fr.astype(np.int64), 63)
    b1 = stack.rotation_and_bin(p1.phase_coef, 0.0, g, p1.dtc, 64)[1]
    edge = np.abs(fr - np.round(fr)) < 1e-6
    assert np.array_equal(b0[~edge], b1[~edge])
    assert np.all(np.abs((b0 - b1 + 32) % 64 - 32)[edge] <= 1)
    w = np.random.default_rng(4).random(len(g))
    s, h = pcd.fold(p1, w, g0)
    assert np.array_equal(h, np.bincount(b1, minlength=64))
    assert np.allclose(s, np.bincount(b1, weights=w, minlength=64), rtol=1e-12)


def test_phase_model_fold_aligns_a_spinning_down_train():
    """Unit pulses at the closed-form times where a spinning-down pulsar's phase
    t / P - Pdot t^2 / (2 P^2) reaches n + 17/32 (the middle of bin 8 of 16,
    rounded to the nearest 62.5 ns sample: within 3e-5 cycles) fold into that
    bin with the model, and smear over many bins at the constant period."""
    from oracle import stack
    P, Pdot, nb = 1e-3, 1e-4, 16
    t_ref, c = stack.spin_model(P, Pdot)
    p_model = pcd.make_plan(**ORT, dm=0.0, nfft=1 << 10, nchan=1, nbins=nb, period=P, phase=(t_ref, c))
    p_const = pcd.make_plan(**ORT, dm=0.0, nfft=1 << 10, nchan=1, nbins=nb, period=P)
    dtc = p_model.dtc
    n = np.arange(200)
    t = P * (1.0 - np.sqrt(1.0 - 2.0 * Pdot * (n + 17 / 32))) / Pdot
    gi = np.rint(t / dtc).astype(np.int64)
    power = np.zeros(int(gi[-1]) + 10)
    power[gi] = 1.0
    s, h = pcd.fold(p_model, power, 0)
    assert s[nb // 2] == len(n) and s.sum() == len(n)
    s2, _ = pcd.fold(p_const, power, 0)
    assert np.count_nonzero(s2) >= nb // 2


def test_phase_model_plan_errors():
    for bad in ((0.0, []), (0.0, [0.0] * 9), (float("nan"), [0.0, 1.0]), (0.0, [0.0, float("inf")])):
        with pytest.raises(pcd.PlanError):
            pcd.make_plan(**ORT, dm=0.0, nfft=1 << 10, nchan=1, nbins=16, period=1e-3, phase=bad)


# --- the batched form (many DM trials on shared segments) ---------------------------

def test_batched_trial_with_own_geometry_is_single_dm_run():
    p = pcd.make_plan(**ORT, dm=0.05, nfft=1 << 14, nchan=4, nbins=16, period=1e-3)
    x = synth.make_stream(synth.StreamSpec(n=5 * p.S + 777, seed=13, dm=0.05, period=1e-3, snr=40))
    q = pcd.trial_plan(p, 0.05, 0.05)
    assert (q.n_past, q.n_fut, q.S_c, q.S) == (p.n_past, p.n_fut, p.S_c, p.S)
    a = pcd.run(p, x)
    b = pcd.run_batched(p, [(0.05, p.nfft, 0.05)], x)[0]
    assert np.array_equal(a.power, b.power) and np.array_equal(a.ts, b.ts)
    c = pcd.run(p, x, g_range=pcd.emitted_range(p, len(x)))
    assert np.array_equal(a.power, c.power)


@pytest.mark.parametrize("dms", [(0.0, 0.004, 0.01), (0.01, 0.002)])
def test_batched_trials_tone_closed_form(dms):
    """Each trial of a batch obeys the tone closed form at its own DM, on the
    group's (larger-overlap) segments and the batch's common output range."""
    base = pcd.make_plan(326.5, 16.0, 32e6, 0.0, 4096, 4, 16, 1e-3)
    gmax = max(dms)
    k0 = (3 * base.L) // 7 + 5
    A, theta = 7.5, 0.3
    g_geo = pcd.make_plan(326.5, 16.0, 32e6, gmax, 4096, 4, 16, 1e-3)
    n_seg = 6
    n = n_seg * g_geo.S + 4096
    x = synth.tone(n, k0, 4096, A, theta)
    res = pcd.run_batched(base, [(dm, 4096, gmax) for dm in dms], x, want_voltages=True)
    g_first, g_end = pcd.batched_range(base, gmax, n)
    c0, j0 = divmod(k0, base.M)
    f = k0 * base.fs / base.nfft * 1e-6 - 8.0
    for dm, r in zip(dms, res):
        assert r.first_g == g_first
        g = r.first_g + np.arange(r.voltages.shape[1])
        complete = g < n_seg * g_geo.S_c + g_geo.n_past
        c = pcd.K_DM * 1e6 * dm * f * f / (326.5 ** 2 * (326.5 + f))
        want = A * 4 * np.exp(1j * theta) * np.exp(-2j * np.pi * (c - round(c))) \
            * np.exp(2j * np.pi * ((j0 * g) % base.M) / base.M)
        assert np.max(np.abs(r.voltages[c0, complete] - want[complete])) < 1e-9 * A * 4


def test_adding_in_phase_special_cases():
    """AIP (Sec. 3.4.1, Sec. 3.7): a silent second half leaves the first, equal
    halves double it, opposite halves cancel, and the int8 extremes add without
    wrapping (-256 .. 254)."""
    rng = np.random.default_rng(7)
    n = rng.integers(-128, 128, 1000).astype(np.int8)
    inter = np.empty(2 * n.size, np.int8)
    inter[0::2], inter[1::2] = n, 0
    assert np.array_equal(pcd.adding_in_phase(inter), n.astype(np.float64))
    inter[1::2] = n
    assert np.array_equal(pcd.adding_in_phase(inter), 2.0 * n)
    inter[1::2] = -np.maximum(n, -127)
    assert np.array_equal(pcd.adding_in_phase(inter), n.astype(np.float64) - np.maximum(n, -127))
    ext = np.array([127, 127, -128, -128, 127, -128], np.int8)
    assert np.array_equal(pcd.adding_in_phase(ext), [254.0, -256.0, -1.0])
    with pytest.raises(ValueError):
        pcd.adding_in_phase(ext[:5])


def test_adding_in_phase_dedisperses_linearly():
    """Up to detection the path is linear, so the voltages of the added stream are
    the sum of each half's voltages (brute force over one segment)."""
    p = pcd.make_plan(**ORT, dm=0.05, nfft=1 << 14, nchan=4, nbins=16, period=0.01)
    rng = np.random.default_rng(8)
    n = rng.integers(-128, 128, p.nfft).astype(np.int8)
    s_ = rng.integers(-128, 128, p.nfft).astype(np.int8)
    inter = np.empty(2 * p.nfft, np.int8)
    inter[0::2], inter[1::2] = n, s_
    v = pcd.dedisperse_segment(p, pcd.adding_in_phase(inter))
    vn, vs = pcd.dedisperse_segment(p, n), pcd.dedisperse_segment(p, s_)
    assert np.allclose(v, vn + vs, rtol=0, atol=1e-9 * np.abs(v).max())