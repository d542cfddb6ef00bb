"""FP64 CPU oracle for phase-coherent dedispersion (PCD) -- TEST INFRASTRUCTURE.

This module is the plain, slow definition that the CUDA engine is checked
against.  Only the test suite, the smoke check and the benchmark's CPU
baseline may import it; the engine never does, and it shares no code with
the engine (the one thing both see is the seeded input generator).

What it computes, step by step (PONDER, Naidu et al., Sec. 3.7 "Phase-coherent
dedispersion mode", Fig. "gpuflow", with the fold of Sec. 3.4):

1. overlap-save segmentation of the real 8-bit stream into ``nfft``-sample
   segments (Sec. 3.7: the filter length must exceed the dispersion smear and
   cover the cyclic-convolution edges);
2. forward DFT of each segment, X[k] = sum_n x[n] exp(-2 pi i k n / N),
   k = 0 .. N/2-1 (DC kept, Nyquist bin dropped);
3. multiplication by the inverse ISM response conj(H) of Eq. 4,
   H(f0+f) = exp(+2 pi i K 1e6 DM f^2 / (f0^2 (f0+f))), f in MHz,
   K = 1/2.41e-4 s MHz^2 (taper = 1);
4. per-sub-channel inverse DFT, v_c[m] = (1/M) sum_j Y[cM+j] exp(+2 pi i j m/M);
5. discard of the n_past / n_fut channel samples that the cyclic wrap
   corrupts at each segment edge;
6. square-law detection |v|^2 summed over sub-channels (Sec. 3.4: "squared to
   get power");
7. fold at the pulsar period into nbins (Sec. 3.4 fold thread, Sec. 3.7 last
   thread), phase in FP64;
8. decimation ("added to achieve the desired temporal resolution", Sec. 3.4)
   to a dedispersed time series.

Readings of points the paper leaves open (constant, sign, sideband, Nyquist
bin, rounding of the overlap, stream edges, fold epoch, decimation binning)
are the ones listed with the design notes of this repository; each function
states the one it uses.  FFTs are numpy's (pocketfft) in complex128: a library
primitive used as the DFT step, pinned against brute-force sums in the tests.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace
from fractions import Fraction

import numpy as np

# Dispersion constant, s MHz^2: 1/2.41e-4 (the constant of Eq. 1, and Eq. 3's
# 4.15e6 ms with f in MHz).  The phase of Eq. 4 in cycles is K*1e6*DM*f^2/(f0^2(f0+f)).
K_DM = 1.0 / 2.41e-4


class PlanError(ValueError):
    """Invalid plan; ``code`` names the error class (ARG / NFFT / NCHAN)."""

    def __init__(self, code: str, msg: str):
        super().__init__(f"{code}: {msg}")
        self.code = code


@dataclass(frozen=True)
class Plan:
    f0: float          # band centre, MHz
    bw: float          # bandwidth, MHz (negative: inverted sideband)
    fs: float          # real samples per second
    dm: float          # pc cm^-3
    nfft: int          # real samples per segment, N
    nchan: int         # detected sub-channels
    nbins: int         # fold bins
    period: float      # s
    t_dec_ns: int      # decimated time-series resolution, ns
    # derived
    L: int = 0         # N/2 spectrum bins kept
    M: int = 0         # complex samples per sub-channel per segment
    dtc: float = 0.0   # channel sample time, s
    n_past: int = 0
    n_fut: int = 0
    S_c: int = 0       # segment step in channel samples
    S: int = 0         # segment step in real samples
    inc: float = 0.0   # fold phase increment per channel sample
    dec: Fraction = Fraction(1)   # channel samples per time-series sample
    # optional polynomial phase model of the fold (replaces the constant period):
    # phi(g) = sum_i phase_coef[i] tau^i, tau = g dtc - phase_tref (seconds from the first sample)
    phase_coef: tuple = ()
    phase_tref: float = 0.0


def adding_in_phase(raw: np.ndarray) -> np.ndarray:
    """Adding in phase (Sec. 3.4.1; the first kernel of the GPU flow in Sec. 3.7):
    the two halves' int8 samples arrive interleaved, N0 S0 N1 S1 ..., and the
    real sample the path transforms is their sum, x[m] = N[m] + S[m]."""
    raw = np.asarray(raw, dtype=np.int8)
    if raw.size % 2:
        raise ValueError("interleaved N / S stream of odd length")
    return raw[0::2].astype(np.float64) + raw[1::2].astype(np.float64)


def overlap(f0: float, bw: float, dm: float, dtc: float) -> tuple[int, int]:
    """(n_past, n_fut) in channel samples, rounded up per side.

    A dedispersed sample at time t (arrival time at f0) draws on input from
    t - K DM (f0^-2 - f_hi^-2) to t + K DM (f_lo^-2 - f0^-2) (Sec. 3.7: the
    impulse response must span the dispersion smear).
    """
    half = abs(bw) / 2.0
    f_lo, f_hi = f0 - half, f0 + half
    past = K_DM * dm * (f0 ** -2 - f_hi ** -2)
    fut = K_DM * dm * (f_lo ** -2 - f0 ** -2)
    return int(math.ceil(past / dtc)), int(math.ceil(fut / dtc))


def make_plan(f0: float, bw: float, fs: float, dm: float, nfft: int, nchan: int,
              nbins: int, period: float, t_dec_s: float = 61.44e-6, phase=None) -> Plan:
    """Validate a plan and derive the overlap-save geometry.  ``phase`` =
    (t_ref, coefficients) folds with that polynomial phase model instead of the
    constant period (1 .. 8 coefficients, cycles per second^i)."""
    if not (f0 > 0 and bw != 0 and abs(bw) < 2 * f0 and fs > 0):
        raise PlanError("ARG", "bad band")
    if abs(fs - 2.0 * abs(bw) * 1e6) > 1e-6 * fs:
        raise PlanError("ARG", "fs must be 2|bw| (real Nyquist sampling)")
    if fs != math.floor(fs):
        raise PlanError("ARG", "fs must be a whole number of Hz")
    if not (dm >= 0 and math.isfinite(dm)):
        raise PlanError("ARG", "DM must be >= 0")
    if not (period > 0 and math.isfinite(period)):
        raise PlanError("ARG", "period must be > 0")
    if nbins < 1:
        raise PlanError("ARG", "nbins must be >= 1")
    if nfft < 4 or nfft & (nfft - 1):
        raise PlanError("NFFT", "nfft must be a power of two >= 4")
    if nchan < 1 or nchan & (nchan - 1) or (nfft // 2) % nchan:
        raise PlanError("NCHAN", "nchan must be a power of two dividing nfft/2")
    L = nfft // 2
    M = L // nchan
    dtc = 2.0 * nchan / fs
    n_past, n_fut = overlap(f0, bw, dm, dtc)
    S_c = M - n_past - n_fut
    if S_c <= 0:
        raise PlanError("NFFT", "nfft does not exceed the overlap: no valid output")
    t_dec_ns = int(round(t_dec_s * 1e9))
    if t_dec_ns <= 0:
        raise PlanError("ARG", "t_dec must be >= 1 ns")
    dec = Fraction(t_dec_ns) * Fraction(int(fs)) / (Fraction(10 ** 9) * 2 * nchan)
    inc = dtc / period
    pc, pt = (), 0.0
    if phase is not None:
        pt, pc = float(phase[0]), tuple(float(c) for c in phase[1])
        if not 1 <= len(pc) <= 8 or not all(math.isfinite(c) for c in pc + (pt,)):
            raise PlanError("ARG", "phase model: 1 .. 8 finite coefficients and a finite t_ref")
    return Plan(f0, bw, fs, dm, nfft, nchan, nbins, period, t_dec_ns, phase_coef=pc, phase_tref=pt,
                L=L, M=M, dtc=dtc, n_past=n_past, n_fut=n_fut, S_c=S_c,
                S=2 * nchan * S_c, inc=inc, dec=dec)


def freq_offsets(p: Plan) -> np.ndarray:
    """Offset f_k (MHz) from f0 of spectrum bin k = 0..L-1.

    Upper sideband (bw > 0): baseband b maps to sky f_lo + b.  Inverted
    (bw < 0): sky f_hi - b.
    """
    k = np.arange(p.L, dtype=np.float64)
    step = p.fs / p.nfft * 1e-6
    half = abs(p.bw) / 2.0
    return k * step - half if p.bw > 0 else half - k * step


def chirp_sign(p: Plan) -> float:
    """+1 for an upper sideband, -1 for an inverted one.

    Mixing with a local oscillator above the band maps sky f to baseband
    f_hi - f and conjugates the spectrum, so the baseband image of H is
    conj(H) there and the inverse filter is H itself.
    """
    return 1.0 if p.bw > 0 else -1.0


def chirp_cycles(p: Plan, f: np.ndarray) -> np.ndarray:
    """Phase of H (Eq. 4) in cycles: K 1e6 DM f^2 / (f0^2 (f0 + f))."""
    return K_DM * 1e6 * p.dm * f * f / (p.f0 * p.f0 * (p.f0 + f))


def dedisperse_segment(p: Plan, seg: np.ndarray) -> np.ndarray:
    """Steps 2-4 on one segment of N real samples -> v[nchan, M] (complex128)."""
    x = np.asarray(seg, dtype=np.float64)
    assert x.shape == (p.nfft,)
    X = np.fft.rfft(x)[:p.L]                      # DFT bins 0..N/2-1
    c = chirp_cycles(p, freq_offsets(p))
    r = c - np.rint(c)                            # exact reduction mod 1 (FP64)
    Y = X * np.exp(-chirp_sign(p) * 2j * np.pi * r)   # x H^-1: dedisperse
    return np.fft.ifft(Y.reshape(p.nchan, p.M), axis=1)   # includes 1/M


@dataclass
class Result:
    first_g: int                 # global channel-sample index of the first output
    power: np.ndarray            # P[g], summed over sub-channels (float64)
    voltages: np.ndarray | None  # v[c, g] (complex128) when requested
    prof_sum: np.ndarray         # float64[nbins]
    prof_hits: np.ndarray        # int64[nbins]
    ts: np.ndarray               # float64 decimated series
    ts_counts: np.ndarray        # int64 channel samples per series sample
    ts_first: int                # series index of ts[0]


def emitted_range(p: Plan, n_total: int) -> tuple[int, int]:
    """[g_first, g_end): the channel samples a stream of n_total real samples yields.

    The first n_past and the last n_fut channel samples lack full support and
    are not emitted; the stream is not zero-extended at either end.
    """
    g_end = n_total // (2 * p.nchan) - p.n_fut
    return p.n_past, max(p.n_past, g_end)


def fold(p: Plan, power: np.ndarray, g0: int) -> tuple[np.ndarray, np.ndarray]:
    """Fold P[g], g = g0.., at the period (FP64 phase, epoch at g = 0).

    bin(g) = min(floor(frac(g * inc) * nbins), nbins - 1), inc = (2 nchan / fs) / P.
    With a phase model the phase is phi(g) of that polynomial at t = g dtc
    (Horner's rule, each FP64 operation rounded on its own; the reading of the
    TEMPO2 predictors of Sec. 3.4 used by the pulse stacks), and
    bin(g) = min(floor((phi - floor(phi)) nbins), nbins - 1).
    """
    if p.phase_coef:
        from oracle import stack
        b = stack.rotation_and_bin(p.phase_coef, p.phase_tref,
                                   np.arange(g0, g0 + len(power), dtype=np.int64), p.dtc, p.nbins)[1]
    else:
        g = np.arange(g0, g0 + len(power), dtype=np.float64)
        x = g * p.inc
        phi = x - np.floor(x)
        b = np.minimum((phi * p.nbins).astype(np.int64), p.nbins - 1)
    s = np.bincount(b, weights=power, minlength=p.nbins).astype(np.float64)
    h = np.bincount(b, minlength=p.nbins).astype(np.int64)
    return s, h


def decimate(p: Plan, power: np.ndarray, g0: int) -> tuple[np.ndarray, np.ndarray, int]:
    """T[j] = sum of P[g] with floor(g / D) = j, D = t_dec fs / (2 nchan) (exact rational)."""
    if len(power) == 0:
        return np.zeros(0), np.zeros(0, dtype=np.int64), 0
    num, den = p.dec.numerator, p.dec.denominator
    g = np.arange(g0, g0 + len(power), dtype=np.int64)
    j = (g * den) // num
    j0 = int(j[0])
    T = np.bincount(j - j0, weights=power).astype(np.float64)
    C = np.bincount(j - j0).astype(np.int64)
    return T, C, j0


def run(p: Plan, x: np.ndarray, want_voltages: bool = False, g_range=None) -> Result:
    """The whole path on a finite stream x (int8 or float), FP64.

    ``g_range`` = (g_first, g_end) narrows the emitted channel samples (the
    batched form emits one common range for all DM trials).
    """
    x = np.asarray(x)
    n_total = len(x)
    g_first, g_end = emitted_range(p, n_total)
    if g_range is not None:
        g_first, g_end = max(g_first, g_range[0]), min(g_end, g_range[1])
        g_end = max(g_end, g_first)
    P_parts, V_parts = [], []
    s = 0
    while s * p.S_c + p.n_past < g_end:
        m_lo = max(p.n_past, g_first - s * p.S_c)
        m_hi = min(p.M - p.n_fut, g_end - s * p.S_c)
        if m_hi <= m_lo:
            s += 1
            continue
        a = s * p.S
        seg = np.zeros(p.nfft, dtype=np.float64)
        take = x[a:a + p.nfft].astype(np.float64)
        seg[:len(take)] = take                    # zeros past the end of the stream
        v = dedisperse_segment(p, seg)
        vv = v[:, m_lo:m_hi]
        P_parts.append(np.sum(vv.real ** 2 + vv.imag ** 2, axis=0))
        if want_voltages:
            V_parts.append(vv)
        s += 1
    power = np.concatenate(P_parts) if P_parts else np.zeros(0)
    volt = None
    if want_voltages:
        volt = np.concatenate(V_parts, axis=1) if V_parts else np.zeros((p.nchan, 0), complex)
    ps, ph = fold(p, power, g_first)
    T, C, j0 = decimate(p, power, g_first)
    return Result(g_first, power, volt, ps, ph, T, C, j0)


def dedisperse_at(p: Plan, x: np.ndarray, g_list) -> tuple[np.ndarray, np.ndarray]:
    """v[c, g] and P[g] for selected global channel samples g only.

    Each g is produced by the one segment whose valid span holds it; this
    runs that segment alone, so single outputs of a long stream can be checked.
    """
    g_list = np.asarray(g_list, dtype=np.int64)
    V = np.zeros((p.nchan, len(g_list)), dtype=np.complex128)
    segs = (g_list - p.n_past) // p.S_c
    for s in np.unique(segs):
        a = int(s) * p.S
        seg = np.zeros(p.nfft)
        take = np.asarray(x[a:a + p.nfft], dtype=np.float64)
        seg[:len(take)] = take
        v = dedisperse_segment(p, seg)
        sel = segs == s
        V[:, sel] = v[:, g_list[sel] - int(s) * p.S_c]
    return V, np.sum(V.real ** 2 + V.imag ** 2, axis=0)


def trial_plan(p: Plan, dm: float, dm_group_max: float) -> Plan:
    """One DM trial of the batched form: the chirp at ``dm`` on the segmentation
    (n_past, n_fut, segment step) that the trial's group takes from its largest
    DM ``dm_group_max``; all trials of a group share the group's segments."""
    q = make_plan(p.f0, p.bw, p.fs, float(dm_group_max), p.nfft, p.nchan, p.nbins, p.period,
                  p.t_dec_ns * 1e-9)
    return replace(q, dm=float(dm))


def batched_range(p: Plan, dm_max: float, n_total: int) -> tuple[int, int]:
    """[g_first, g_end): the channel samples every trial of a batch up to dm_max emits."""
    n_past, n_fut = overlap(p.f0, p.bw, dm_max, p.dtc)
    return n_past, max(n_past, n_total // (2 * p.nchan) - n_fut)


def run_batched(p: Plan, trials, x: np.ndarray, want_voltages: bool = False) -> list[Result]:
    """The batched form: ``trials`` is a list of (dm, nfft, dm_group_max); each
    trial runs the single-DM path at its DM on its group's segmentation, over
    the common emitted range of the largest DM of the batch."""
    dm_max = max(t[0] for t in trials)
    rng = batched_range(p, dm_max, len(x))
    out = []
    for dm, nfft, gmax in trials:
        q = trial_plan(make_plan(p.f0, p.bw, p.fs, 0.0, int(nfft), p.nchan, p.nbins, p.period,
                                 p.t_dec_ns * 1e-9), dm, gmax)
        out.append(run(q, x, want_voltages=want_voltages, g_range=rng))
    return out


# --- closed forms the paper prints (Sec. 3.2 Eq. 1, Sec. 3.4 Eqs. 2 and 3) ---------

def residual_smear_ms(df_ch_mhz: float, dm: float, f_ch_mhz: float) -> float:
    """Eq. 2: residual intra-channel dispersion smear, ms."""
    return 8.3e6 * df_ch_mhz * dm / f_ch_mhz ** 3


def channel_delay_ms(f_ref_mhz: float, f_chan_mhz: float, dm: float) -> float:
    """Eq. 3: dispersive delay of a channel relative to the reference, ms."""
    return 4.15e6 * (f_ref_mhz ** -2 - f_chan_mhz ** -2) * dm


def band_smear_s(f0: float, bw: float, dm: float) -> float:
    """Dispersion sweep across the band, K DM (f_lo^-2 - f_hi^-2), s."""
    half = abs(bw) / 2.0
    return K_DM * dm * ((f0 - half) ** -2 - (f0 + half) ** -2)
