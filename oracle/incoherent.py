"""FP64 CPU oracle for the incoherent dedispersion modes -- TEST INFRASTRUCTURE.

Only the test suite, the smoke check and the benchmark's CPU legs may import
this module; the engine never does and shares no code with it.

What it computes (PONDER, Naidu et al., Sec. 3.4 "Real-time pulsar mode with
incoherent dedispersion", with its sub-modes AID of Sec. 3.4.1 and CID of
Sec. 3.4.2):

1. an FFT filterbank: the real stream is cut into consecutive, non-overlapping
   blocks of 2 nchan samples and each block transformed,
   X[k] = sum_n x[n] exp(-2 pi i k n / (2 nchan)), k = 0 .. nchan-1 (DC kept,
   Nyquist dropped, no window);
2. detection: AID (adding in phase) squares the spectrum of the added stream,
   x = N + S (or the single stream), |X[k]|^2; CID (correlation) multiplies the
   two halves' spectra, Re(X_N[k] conj(X_S[k]));
3. integration of nint consecutive spectra into one output sample of
   t_s = nint * 2 nchan / fs seconds (the integration thread);
4. incoherent dedispersion by per-channel delays (Eq. 3): channel k at sky
   frequency f_k is read d_k samples later, d_k = floor(K DM (f_k^-2 - f0^-2)
   / t_s + 1/2), and the channels are summed, D[t] = sum_k F[k][t + d_k];
5. the fold of D at the period (FP64 phase, epoch at t = 0), the same rule as
   the coherent mode's fold.

Readings (the paper leaves them open): channel k of the FFT filterbank sits at
the sky frequency of its bin, f_lo + k df (upper sideband; f_hi - k df when the
band is inverted), df = |bw| / nchan; delays refer to the band centre f0, the
reference of the coherent mode's output times, with the constant K of the
coherent oracle; trailing samples that do not fill an output sample are not
used; D is emitted only where every channel's shifted sample exists.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from oracle.pcd import K_DM, adding_in_phase

AID = 0
CID = 1


class IncoPlanError(ValueError):
    pass


@dataclass(frozen=True)
class IncoPlan:
    f0: float          # band centre, MHz
    bw: float          # MHz (negative: inverted sideband)
    fs: float          # real samples per second
    dm: float
    nchan: int         # filterbank channels
    nint: int          # spectra per output sample
    mode: int          # AID or CID
    channels: int      # input channels: 1 (one stream) or 2 (N / S interleaved)
    nbins: int
    period: float      # s
    ts: float = 0.0    # output sample time, s
    inc: float = 0.0   # fold phase per output sample


def make_plan(f0: float, bw: float, fs: float, dm: float, nchan: int, nint: int, mode: int,
              channels: int, nbins: int, period: float) -> IncoPlan:
    if nchan < 1 or nchan & (nchan - 1) or nint < 1 or nint & (nint - 1):
        raise IncoPlanError("nchan and nint must be powers of two")
    if mode not in (AID, CID) or channels not in (1, 2) or (mode == CID and channels != 2):
        raise IncoPlanError("AID takes 1 or 2 input channels, CID takes 2")
    if nbins < 1 or not period > 0 or not fs > 0 or bw == 0 or dm < 0:
        raise IncoPlanError("bad band, fold or DM")
    ts = 2.0 * nchan * nint / fs
    return IncoPlan(f0, bw, fs, dm, nchan, nint, mode, channels, nbins, period, ts, ts / period)


def channel_freqs(p: IncoPlan) -> np.ndarray:
    """Sky frequency (MHz) of filterbank channel k: the frequency of its bin."""
    k = np.arange(p.nchan, dtype=np.float64)
    df = abs(p.bw) / p.nchan
    if p.bw > 0:
        return (p.f0 - abs(p.bw) / 2.0) + k * df
    return (p.f0 + abs(p.bw) / 2.0) - k * df


def channel_delays(p: IncoPlan) -> np.ndarray:
    """d_k in output samples (Eq. 3 referred to f0, rounded to the nearest sample)."""
    f = channel_freqs(p)
    delay_s = K_DM * p.dm * (f ** -2.0 - p.f0 ** -2.0)
    return np.floor(delay_s / p.ts + 0.5).astype(np.int64)


def spectra(p: IncoPlan, x: np.ndarray, n_spec: int) -> np.ndarray:
    """The first n_spec spectra of the real series x (blocks of 2 nchan), bins 0 .. nchan-1."""
    R = 2 * p.nchan
    blocks = np.asarray(x[:n_spec * R], dtype=np.float64).reshape(n_spec, R)
    return np.fft.fft(blocks, axis=1)[:, :p.nchan]


def n_samples(p: IncoPlan, raw: np.ndarray) -> int:
    """Time samples in the raw int8 input (pairs when it holds two channels)."""
    if len(raw) % p.channels:
        raise ValueError("input splits an N / S pair")
    return len(raw) // p.channels


def filterbank(p: IncoPlan, raw: np.ndarray) -> np.ndarray:
    """Integrated detected filterbank F[k][t], k < nchan, t < T (channel-major, FP64)."""
    n = n_samples(p, raw)
    T = n // (2 * p.nchan) // p.nint
    n_spec = T * p.nint
    if p.mode == AID:
        x = adding_in_phase(raw) if p.channels == 2 else np.asarray(raw, dtype=np.float64)
        X = spectra(p, x, n_spec)
        pw = X.real ** 2 + X.imag ** 2
    else:
        r = np.asarray(raw)
        XN = spectra(p, r[0::2].astype(np.float64), n_spec)
        XS = spectra(p, r[1::2].astype(np.float64), n_spec)
        pw = (XN * np.conj(XS)).real
    F = pw.reshape(T, p.nint, p.nchan).sum(axis=1)
    return np.ascontiguousarray(F.T)


def dedisperse(p: IncoPlan, F: np.ndarray) -> tuple[np.ndarray, int]:
    """D[t] = sum_k F[k][t + d_k] for every t whose shifted samples all exist; (D, t_first)."""
    d = channel_delays(p)
    T = F.shape[1]
    t_first = max(0, -int(d.min()))
    t_end = T - max(0, int(d.max()))
    if t_end <= t_first:
        return np.zeros(0), t_first
    D = np.zeros(t_end - t_first)
    for k in range(p.nchan):
        D += F[k, t_first + d[k]:t_end + d[k]]
    return D, t_first


def fold(p: IncoPlan, D: np.ndarray, t_first: int) -> tuple[np.ndarray, np.ndarray]:
    """bin(t) = min(floor(frac(t * inc) * nbins), nbins - 1), inc = t_s / P, FP64."""
    t = np.arange(t_first, t_first + len(D), dtype=np.float64)
    x = t * p.inc
    phi = x - np.floor(x)
    b = np.minimum((phi * p.nbins).astype(np.int64), p.nbins - 1)
    s = np.bincount(b, weights=D, minlength=p.nbins).astype(np.float64)
    h = np.bincount(b, minlength=p.nbins).astype(np.int64)
    return s, h


@dataclass
class IncoResult:
    F: np.ndarray          # [nchan][T] integrated filterbank
    D: np.ndarray          # dedispersed series, samples t_first ..
    t_first: int
    prof_sum: np.ndarray
    prof_hits: np.ndarray


def run(p: IncoPlan, raw: np.ndarray) -> IncoResult:
    F = filterbank(p, raw)
    D, t_first = dedisperse(p, F)
    s, h = fold(p, D, t_first)
    return IncoResult(F, D, t_first, s, h)


def residual_smear_ms(p: IncoPlan, k: int) -> float:
    """Eq. 2 for channel k of the plan: the smear left inside one channel, ms."""
    f = float(channel_freqs(p)[k])
    return 8.3e6 * (abs(p.bw) / p.nchan) * p.dm / f ** 3


def delay_span_samples(p: IncoPlan) -> int:
    d = channel_delays(p)
    return int(d.max() - d.min())
