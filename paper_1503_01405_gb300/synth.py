"""Seeded synthetic voltage streams shaped like the ORT 16 MHz band.

This module is the one place that both the FP64 oracle tests and the CUDA
engine draw their inputs from.  It holds a counter-based random number
generator, the pulse/RFI sky model and the 8-bit quantiser; it does not
dedisperse, detect, fold or decimate anything.

Stream model (all quantities per real sample at ``fs`` samples/s):

* receiver noise: Gaussian, standard deviation ``sigma`` ADC counts;
* pulsar: extra Gaussian noise of variance ``A * g(phase) * sigma**2``
  (amplitude-modulated noise, the emission a pulsar makes), where ``g`` is a
  Gaussian pulse of peak 1 and full width at half maximum ``duty`` (in
  rotational phase), and ``A`` is set from the requested matched-filter S/N
  (``A = snr * sqrt(2 / sum_i g_i**2)``, the sum over the fold or over one
  period);
* the pulsar voltage is passed through the cold-plasma transfer function of
  the interstellar medium, H(f0+f) = exp(+2 pi i K DM f^2 / (f0^2 (f0+f))),
  f in MHz with K = 1/2.41e-4 s MHz^2 scaled by 1e6 to cycles (the paper's
  Sec. 3.7, Eq. 4, and the constant of Eq. 1).  This is the sky, not the
  method: an impulse emitted at t arrives at frequency f0+f at
  t + K DM ((f0+f)^-2 - f0^-2) seconds.  With an inverted sideband (bw < 0)
  baseband bin b holds the conjugate of the sky spectrum at f_hi - b, so the
  phase of H enters with the opposite sign;
* impulsive broadband RFI (undispersed), and optionally narrowband
  sinusoidal RFI;
* quantisation to int8: round half to even, then clip to [-clip, clip]
  (the ADC of Sec. 3.1 gives -128..127).

Random numbers come from Philox4x32-10 (Salmon, Moraes, Dror & Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11) with a Box-Muller
transform, so any sample range can be generated independently.  The large
stream used for throughput measurement is generated on the GPU with torch's
own seeded generator instead (``make_stream_torch``); it follows the same
recipe with different random draws.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import numpy as np

# Dispersion constant K = 1/2.41e-4 s MHz^2 (Eq. 1's constant; Eq. 3's 4.15e6 ms).
K_DM = 1.0 / 2.41e-4

# Philox4x32-10 constants (Salmon et al. 2011, Sec. 5).
_PHILOX_M0 = 0xD2511F53
_PHILOX_M1 = 0xCD9E8D57
_PHILOX_W0 = 0x9E3779B9
_PHILOX_W1 = 0xBB67AE85
_M32 = np.uint64(0xFFFFFFFF)

# Sub-stream identifiers (third counter word).
STREAM_NOISE = 0
STREAM_PULSAR = 1
STREAM_RFI_NOISE = 2
STREAM_RFI_EVENTS = 3
STREAM_EVENTS = 4


def philox4x32_10(ctr, key):
    """Philox4x32-10 block function.

    ``ctr`` is a sequence of four uint64 arrays holding 32-bit words, ``key``
    a pair of 32-bit integers.  Returns four uint64 arrays of 32-bit words.
    """
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _M32 for c in ctr)
    k0 = np.uint64(int(key[0]) & 0xFFFFFFFF)
    k1 = np.uint64(int(key[1]) & 0xFFFFFFFF)
    m0 = np.uint64(_PHILOX_M0)
    m1 = np.uint64(_PHILOX_M1)
    sh = np.uint64(32)
    for r in range(10):
        if r:
            k0 = np.uint64((int(k0) + _PHILOX_W0) & 0xFFFFFFFF)
            k1 = np.uint64((int(k1) + _PHILOX_W1) & 0xFFFFFFFF)
        p0 = m0 * c0  # exact: both factors < 2**32
        p1 = m1 * c2
        hi0, lo0 = p0 >> sh, p0 & _M32
        hi1, lo1 = p1 >> sh, p1 & _M32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def random_words(seed: int, stream: int, start: int, n: int) -> np.ndarray:
    """32-bit random words ``start .. start+n-1`` of sub-stream ``stream``.

    Word i comes from counter (i // 4 low, i // 4 high, stream, 0), lane i % 4,
    key (seed low, seed high).
    """
    if n <= 0:
        return np.zeros(0, dtype=np.uint64)
    b0 = start // 4
    b1 = (start + n - 1) // 4 + 1
    blk = np.arange(b0, b1, dtype=np.uint64)
    out = philox4x32_10(
        (blk & _M32, blk >> np.uint64(32), np.full_like(blk, stream), np.zeros_like(blk)),
        (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF),
    )
    words = np.stack(out, axis=1).reshape(-1)
    off = start - 4 * b0
    return words[off:off + n]


def uniform(seed: int, stream: int, start: int, n: int) -> np.ndarray:
    """Uniform deviates in (0, 1): (word + 0.5) / 2**32."""
    return (random_words(seed, stream, start, n).astype(np.float64) + 0.5) * 2.0**-32


def gaussian(seed: int, stream: int, start: int, n: int) -> np.ndarray:
    """Standard normal deviates by Box-Muller on word pairs (0,1) and (2,3).

    Deviate i uses the pair that holds word i: even i takes r cos(theta), odd
    i takes r sin(theta), with r = sqrt(-2 ln u_even), theta = 2 pi u_odd.
    """
    if n <= 0:
        return np.zeros(0)
    a = start - (start % 2)
    b = start + n + ((start + n) % 2)
    u = uniform(seed, stream, a, b - a).reshape(-1, 2)
    r = np.sqrt(-2.0 * np.log(u[:, 0]))
    th = 2.0 * np.pi * u[:, 1]
    z = np.stack([r * np.cos(th), r * np.sin(th)], axis=1).reshape(-1)
    return z[start - a:start - a + n]


@dataclass(frozen=True)
class StreamSpec:
    """Recipe for one synthetic stream (see the module docstring)."""

    n: int                       # real samples
    seed: int = 1
    fs: float = 32e6             # real samples per second (Nyquist for |bw| = 16 MHz)
    f0: float = 326.5            # band centre, MHz
    bw: float = 16.0             # MHz; negative = inverted sideband
    sigma: float = 20.0          # receiver noise, ADC counts
    dm: float = 3.0              # pc cm^-3 (0 = no pulsar dispersion)
    period: float = 0.253        # s (0 = no pulsar)
    duty: float = 0.03           # FWHM of the pulse in rotational phase
    snr: float = 50.0            # matched-filter S/N of the pulsar
    snr_per: str = "fold"        # "fold": over the whole stream; "period": per rotation
    phase_c: float = 0.5         # pulse centre in rotational phase
    rfi_duty: float = 0.0        # fraction of time covered by impulsive RFI bursts
    rfi_sigma: float = 5.0       # burst noise standard deviation / sigma
    clip: int = 127


# The workloads the engine is measured and checked on.
SMALL = StreamSpec(n=2**23, seed=1, dm=3.0, period=0.253, duty=0.03, snr=50.0,
                   snr_per="fold")
FULL_RATE = StreamSpec(n=1_920_000_000, seed=2, dm=26.8, period=0.7145, duty=0.05,
                       snr=20.0, snr_per="period", rfi_duty=0.01)


def pulse_shape(phase: np.ndarray, duty: float, phase_c: float) -> np.ndarray:
    """Gaussian pulse of peak 1 and FWHM ``duty`` centred at ``phase_c``."""
    d = phase - phase_c
    d = d - np.floor(d + 0.5)
    return np.exp(-4.0 * math.log(2.0) * (d / duty) ** 2)


def sum_g2(spec: StreamSpec) -> float:
    """Sum of g(phase_i)^2 over the samples the S/N refers to."""
    if spec.snr_per == "period":
        count = spec.fs * spec.period
    else:
        count = float(spec.n)
    # integral of g^2 over one rotation, g Gaussian of FWHM duty
    w = spec.duty
    integral = w * math.sqrt(math.pi / (8.0 * math.log(2.0)))
    return count * integral


def pulsar_amplitude(spec: StreamSpec) -> float:
    """Variance scale A so that the pulsar has matched-filter S/N ``spec.snr``."""
    if spec.period <= 0 or spec.snr <= 0:
        return 0.0
    return spec.snr * math.sqrt(2.0 / sum_g2(spec))


def dispersion_delay(f_mhz, f0: float, dm: float):
    """Arrival delay (s) at sky frequency ``f_mhz`` relative to ``f0`` (Eq. 3 form)."""
    return K_DM * dm * (np.asarray(f_mhz, dtype=np.float64) ** -2 - f0 ** -2)


def ism_cycles(f_off, f0: float, dm: float):
    """Phase (cycles) of the ISM transfer function at offset ``f_off`` MHz from f0."""
    f = np.asarray(f_off, dtype=np.float64)
    return K_DM * 1e6 * dm * f * f / (f0 * f0 * (f0 + f))


def margins(spec: StreamSpec) -> tuple[int, int]:
    """Real samples of emission needed before / after an observed span."""
    if spec.dm == 0:
        return 0, 0
    bw = abs(spec.bw)
    lo, hi = spec.f0 - bw / 2, spec.f0 + bw / 2
    late = K_DM * spec.dm * (lo ** -2 - spec.f0 ** -2)    # low edge arrives late
    early = K_DM * spec.dm * (spec.f0 ** -2 - hi ** -2)   # high edge arrives early
    return int(math.ceil(late * spec.fs)) + 64, int(math.ceil(early * spec.fs)) + 64


def _next_fast(n: int) -> int:
    m = 1
    while m < n:
        m *= 2
    for cand in (m, 3 * m // 4, 5 * m // 8):
        if cand >= n:
            m = min(m, cand)
    return m


def ism_disperse(emitted: np.ndarray, spec: StreamSpec) -> np.ndarray:
    """Apply the ISM transfer function to a real voltage (circular, FP64).

    The caller pads the emission so that the span it keeps is free of wrap.
    """
    L = len(emitted)
    spec_v = np.fft.rfft(emitted)
    k = np.arange(len(spec_v), dtype=np.float64)
    step = spec.fs / L * 1e-6
    half = abs(spec.bw) / 2
    f_off = k * step - half if spec.bw > 0 else half - k * step
    c = ism_cycles(f_off, spec.f0, spec.dm)
    c = c - np.rint(c)
    # an inverted sideband conjugates the baseband spectrum, so H's phase flips sign
    sign = 1.0 if spec.bw > 0 else -1.0
    return np.fft.irfft(spec_v * np.exp(sign * 2j * np.pi * c), n=L)


def pulsar_voltage(spec: StreamSpec, start: int, n: int) -> np.ndarray:
    """Observed (dispersed) pulsar voltage for real samples [start, start+n)."""
    amp = pulsar_amplitude(spec)
    if amp == 0.0 or n == 0:
        return np.zeros(n)
    late, early = margins(spec)
    e0 = start - late
    ne = n + late + early
    L = _next_fast(ne)
    idx = np.arange(e0, e0 + ne, dtype=np.float64)
    phase = idx / (spec.fs * spec.period)
    phase -= np.floor(phase)
    env = spec.sigma * np.sqrt(amp * pulse_shape(phase, spec.duty, spec.phase_c))
    w = gaussian(spec.seed, STREAM_PULSAR, e0 + (1 << 40), ne)
    emitted = np.zeros(L)
    emitted[:ne] = env * w
    if spec.dm == 0:
        return emitted[late:late + n]
    return ism_disperse(emitted, spec)[late:late + n]


def rfi_bursts(spec: StreamSpec, n: int) -> list[tuple[int, int]]:
    """Impulsive RFI bursts as (start, length) in real samples.

    Starts form a Poisson process (exponential gaps), lengths are log-uniform
    on [1 us, 100 us]; the rate is set so that the bursts cover ``rfi_duty``
    of the time.
    """
    if spec.rfi_duty <= 0:
        return []
    lo, hi = 1e-6, 100e-6
    mean_len = (hi - lo) / math.log(hi / lo)
    rate = spec.rfi_duty / mean_len
    expect = int(rate * n / spec.fs * 1.2) + 64
    u = uniform(spec.seed, STREAM_RFI_EVENTS, 0, 2 * expect)
    gaps = -np.log(u[0::2]) / rate * spec.fs
    lens = np.exp(math.log(lo) + u[1::2] * math.log(hi / lo)) * spec.fs
    starts = np.cumsum(gaps)
    out = []
    for s, ln in zip(starts, lens):
        if s >= n:
            break
        out.append((int(s), max(1, int(round(ln)))))
    return out


def quantise(v: np.ndarray, clip: int = 127) -> np.ndarray:
    """Round half to even, clip to [-clip, clip], store as int8."""
    return np.clip(np.rint(v), -clip, clip).astype(np.int8)


def make_stream(spec: StreamSpec) -> np.ndarray:
    """The whole stream of ``spec`` as int8 (CPU, FP64 model)."""
    n = spec.n
    v = spec.sigma * gaussian(spec.seed, STREAM_NOISE, 0, n)
    v += pulsar_voltage(spec, 0, n)
    for s, ln in rfi_bursts(spec, n):
        e = min(n, s + ln)
        v[s:e] += spec.rfi_sigma * spec.sigma * gaussian(spec.seed, STREAM_RFI_NOISE, s, e - s)
    return quantise(v, spec.clip)


def tone(n: int, k0: int, nfft: int, amp: float, theta: float) -> np.ndarray:
    """A real tone amp*cos(2 pi k0 n / nfft + theta) (FP64, unquantised)."""
    t = np.arange(n, dtype=np.float64)
    return amp * np.cos(2.0 * np.pi * ((k0 * (t % nfft)) % nfft) / nfft + theta)


def make_stream_torch(spec: StreamSpec, device, block: int = 1 << 26):
    """The stream of ``spec`` generated on a CUDA device with torch (int8 tensor).

    Same recipe as ``make_stream`` with torch's seeded generator in place of
    Philox, for streams too long to generate on the host.  Used only to make
    inputs; it is not part of the engine.
    """
    import torch

    n = spec.n
    out = torch.empty(n, dtype=torch.int8, device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(spec.seed)
    amp = pulsar_amplitude(spec)
    late, early = margins(spec)
    # dispersion by overlap-save blocks: FFT length Lb, output span B per block
    Lb = 1 << 27
    while Lb < 4 * (late + early + 1):
        Lb *= 2
    B = Lb - late - early
    H = None
    if amp > 0 and spec.dm != 0:
        k = torch.arange(Lb // 2 + 1, dtype=torch.float64, device=device)
        step = spec.fs / Lb * 1e-6
        half = abs(spec.bw) / 2
        f_off = k * step - half if spec.bw > 0 else half - k * step
        c = K_DM * 1e6 * spec.dm * f_off * f_off / (spec.f0 * spec.f0 * (spec.f0 + f_off))
        c = c - torch.round(c)
        sign = 1.0 if spec.bw > 0 else -1.0
        H = torch.polar(torch.ones_like(c), sign * 2 * math.pi * c).to(torch.complex64)
        del k, f_off, c
    bursts = rfi_bursts(spec, n)
    mask = None
    if bursts:
        delta = torch.zeros(n + 1, dtype=torch.int8, device=device)
        st = torch.tensor([b[0] for b in bursts], dtype=torch.int64, device=device)
        en = torch.clamp(st + torch.tensor([b[1] for b in bursts], dtype=torch.int64,
                                           device=device), max=n)
        ones = torch.ones_like(st, dtype=torch.int8)
        delta.index_put_((st,), ones, accumulate=True)
        delta.index_put_((en,), -ones, accumulate=True)
        mask = delta
    run = torch.zeros((), dtype=torch.int32, device=device)
    for b0 in range(0, n, B):
        nb = min(B, n - b0)
        v = torch.randn(nb, generator=gen, device=device, dtype=torch.float32) * spec.sigma
        if amp > 0:
            e0 = b0 - late
            ne = nb + late + early
            idx = torch.arange(e0, e0 + ne, dtype=torch.float64, device=device)
            ph = idx / (spec.fs * spec.period)
            ph = ph - torch.floor(ph)
            d = ph - spec.phase_c
            d = d - torch.floor(d + 0.5)
            g = torch.exp(-4.0 * math.log(2.0) * (d / spec.duty) ** 2).to(torch.float32)
            del idx, ph, d
            w = torch.randn(ne, generator=gen, device=device, dtype=torch.float32)
            em = torch.zeros(Lb, dtype=torch.float32, device=device)
            em[:ne] = spec.sigma * torch.sqrt(amp * g) * w
            del g, w
            if H is not None:
                em = torch.fft.irfft(torch.fft.rfft(em) * H, n=Lb)
            v += em[late:late + nb]
            del em
        if mask is not None:
            seg = torch.cumsum(mask[b0:b0 + nb].to(torch.int32), 0) + run
            run = seg[-1].clone()
            on = seg > 0
            v += on.to(torch.float32) * (spec.rfi_sigma * spec.sigma) * torch.randn(
                nb, generator=gen, device=device, dtype=torch.float32)
            del seg, on
        out[b0:b0 + nb] = torch.clamp(torch.round(v), -spec.clip, spec.clip).to(torch.int8)
        del v
    return out


def with_n(spec: StreamSpec, n: int) -> StreamSpec:
    return replace(spec, n=n)


# --- single dispersed pulses (transient search workloads) ----------------------------

@dataclass(frozen=True)
class Pulse:
    t0: float        # emission time referenced to arrival at f0, s from the chunk start
    dm: float        # pc cm^-3
    width: float     # FWHM, s
    snr: float       # matched-filter S/N over the pulse (same definition as the pulsar)


def draw_pulses(seed: int, n_pulses: int, duration: float, dm_range=(2.0, 58.0), edge=0.25,
                width_range=(1e-4, 2e-3), snr_range=(6.0, 30.0)) -> list[Pulse]:
    """Pulses at uniform times (``edge`` s away from the chunk ends), uniform DM,
    log-uniform width and uniform S/N, drawn from Philox sub-stream STREAM_EVENTS."""
    u = uniform(seed, STREAM_EVENTS, 0, 4 * n_pulses).reshape(n_pulses, 4)
    out = []
    for a, b, c, d in u:
        t0 = edge + a * (duration - 2 * edge)
        dm = dm_range[0] + b * (dm_range[1] - dm_range[0])
        w = math.exp(math.log(width_range[0]) + c * math.log(width_range[1] / width_range[0]))
        snr = snr_range[0] + d * (snr_range[1] - snr_range[0])
        out.append(Pulse(float(t0), float(dm), float(w), float(snr)))
    return sorted(out, key=lambda p: p.t0)


def pulse_window(spec: StreamSpec, p: Pulse, index: int) -> tuple[int, np.ndarray]:
    """(first sample, dispersed voltage) of one pulse: extra Gaussian noise of
    variance A g(t) sigma^2 with g a Gaussian of peak 1 and FWHM p.width,
    A = snr sqrt(2 / sum g^2), passed through the ISM response at p.dm."""
    fs = spec.fs
    half_w = int(math.ceil(3 * p.width * fs))
    sp = replace(spec, dm=p.dm)
    late, early = margins(sp)
    c = int(round(p.t0 * fs))
    e0 = c - half_w - late
    ne = 2 * half_w + late + early
    t = (np.arange(e0, e0 + ne) - p.t0 * fs) / fs
    g = np.exp(-4.0 * math.log(2.0) * (t / p.width) ** 2)
    amp = p.snr * math.sqrt(2.0 / np.sum(g * g))
    w = gaussian(spec.seed, STREAM_PULSAR, (1 << 44) + index * (1 << 36), ne)
    L = _next_fast(ne)
    em = np.zeros(L)
    em[:ne] = spec.sigma * np.sqrt(amp * g) * w
    v = ism_disperse(em, sp) if p.dm > 0 else em
    return e0, v[:ne]


def make_chunk(spec: StreamSpec, pulses: list[Pulse]) -> np.ndarray:
    """Noise (plus RFI per spec) with the given dispersed pulses, as int8 (CPU)."""
    n = spec.n
    v = spec.sigma * gaussian(spec.seed, STREAM_NOISE, 0, n)
    for i, p in enumerate(pulses):
        e0, pv = pulse_window(spec, p, i)
        a, b = max(0, e0), min(n, e0 + len(pv))
        if b > a:
            v[a:b] += pv[a - e0:b - e0]
    for s0, ln in rfi_bursts(spec, n):
        e = min(n, s0 + ln)
        v[s0:e] += spec.rfi_sigma * spec.sigma * gaussian(spec.seed, STREAM_RFI_NOISE, s0, e - s0)
    return quantise(v, spec.clip)


def make_chunk_torch(spec: StreamSpec, pulses: list[Pulse], device):
    """``make_chunk`` on a CUDA device (torch RNG for the noise; pulses from the
    CPU model, each generated over its own dispersed window)."""
    import torch
    n = spec.n
    gen = torch.Generator(device=device)
    gen.manual_seed(spec.seed)
    v = torch.randn(n, generator=gen, device=device, dtype=torch.float32) * spec.sigma
    for i, p in enumerate(pulses):
        e0, pv = pulse_window(spec, p, i)
        a, b = max(0, e0), min(n, e0 + len(pv))
        if b > a:
            v[a:b] += torch.from_numpy(pv[a - e0:b - e0].astype(np.float32)).to(device)
    return torch.clamp(torch.round(v), -spec.clip, spec.clip).to(torch.int8)


# The batched workload: 8 s chunks, 10 single pulses, 128 DM trials 0..60.
BATCH_CHUNK = StreamSpec(n=256_000_000, seed=4, dm=0.0, period=0.0, snr=0.0)
BATCH_DMS = [60.0 * d / 127.0 for d in range(128)]


# --- labelled events for the candidate classifier ------------------------------------

EV_PULSE, EV_BURST, EV_NARROW, EV_NOISE = 0, 1, 2, 3


@dataclass(frozen=True)
class Event:
    kind: int        # EV_PULSE, EV_BURST (undispersed broadband), EV_NARROW (sinusoid), EV_NOISE
    t0: float        # s from the chunk start (arrival at f0 for pulses)
    dm: float        # pulse DM; 0 for a burst; the DM row a patch is centred on otherwise
    width: float     # FWHM (pulse, burst) or duration (sinusoid), s
    snr: float       # matched-filter S/N (pulse, burst)
    freq: float      # baseband frequency of a sinusoid, MHz


def draw_events(seed: int, n: int, duration: float, dm_max: float = 60.0, spacing: float = 0.3,
                first: float = 0.3) -> list[Event]:
    """n events of uniformly drawn kind at t = first + i spacing (the DM-60 sweep
    is 0.23 s, so events do not overlap).  Pulses: DM U(2, dm_max - 2), width
    log-U(0.1, 2) ms, S/N U(6, 30); bursts: DM 0, width log-U(0.05, 2) ms,
    S/N U(6, 30); sinusoids: amplitude 2 sigma, 1-20 ms, uniform frequency;
    noise: nothing (centre DM drawn uniformly)."""
    u = uniform(seed, STREAM_EVENTS, 1 << 20, 6 * n).reshape(n, 6)
    out = []
    for i in range(n):
        k = int(u[i, 0] * 4) % 4
        t0 = first + i * spacing
        if t0 > duration - 0.25:
            break
        if k == EV_PULSE:
            dm = 2.0 + u[i, 1] * (dm_max - 4.0)
            w = math.exp(math.log(1e-4) + u[i, 2] * math.log(20.0))
        elif k == EV_BURST:
            dm = 0.0
            w = math.exp(math.log(5e-5) + u[i, 2] * math.log(40.0))
        elif k == EV_NARROW:
            dm = u[i, 1] * dm_max
            w = 1e-3 + u[i, 2] * 19e-3
        else:
            dm = u[i, 1] * dm_max
            w = 0.0
        out.append(Event(k, float(t0), float(dm), float(w), float(6.0 + u[i, 3] * 24.0), float(u[i, 4] * 16.0)))
    return out


def _ism_phase_torch(Lb: int, spec: StreamSpec, dm: float, device):
    import torch
    k = torch.arange(Lb // 2 + 1, dtype=torch.float64, device=device)
    step = spec.fs / Lb * 1e-6
    half = abs(spec.bw) / 2
    f = k * step - half if spec.bw > 0 else half - k * step
    c = K_DM * 1e6 * dm * f * f / (spec.f0 * spec.f0 * (spec.f0 + f))
    c = c - torch.round(c)
    sign = 1.0 if spec.bw > 0 else -1.0
    return torch.polar(torch.ones_like(c), sign * 2 * math.pi * c).to(torch.complex64)


def make_labelled_chunk_torch(spec: StreamSpec, events: list[Event], device, seed_offset: int = 0):
    """Noise plus the events of ``events`` on a CUDA device, as int8.  Pulses and
    bursts follow the pulse model of ``pulse_window`` (dispersed by the ISM
    response with torch.fft); sinusoids are 2 sigma tones with a Hann envelope."""
    import torch
    n = spec.n
    gen = torch.Generator(device=device)
    gen.manual_seed(spec.seed + seed_offset)
    v = torch.randn(n, generator=gen, device=device, dtype=torch.float32) * spec.sigma
    fs = spec.fs
    for ev in events:
        if ev.kind in (EV_PULSE, EV_BURST):
            sp = replace(spec, dm=ev.dm)
            late, early = margins(sp)
            half_w = int(math.ceil(3 * ev.width * fs))
            c = int(round(ev.t0 * fs))
            e0 = c - half_w - late
            ne = 2 * half_w + late + early
            t = (torch.arange(e0, e0 + ne, device=device, dtype=torch.float64) - ev.t0 * fs) / fs
            g = torch.exp(-4.0 * math.log(2.0) * (t / ev.width) ** 2)
            amp = ev.snr * math.sqrt(2.0 / float(torch.sum(g * g)))
            w = torch.randn(ne, generator=gen, device=device, dtype=torch.float64)
            em = spec.sigma * torch.sqrt(amp * g) * w
            if ev.dm > 0:
                L = 1 << int(math.ceil(math.log2(ne)))
                buf = torch.zeros(L, dtype=torch.float32, device=device)
                buf[:ne] = em.to(torch.float32)
                em = torch.fft.irfft(torch.fft.rfft(buf) * _ism_phase_torch(L, spec, ev.dm, device), n=L)[:ne]
            a, b = max(0, e0), min(n, e0 + ne)
            if b > a:
                v[a:b] += em[a - e0:b - e0].to(torch.float32)
        elif ev.kind == EV_NARROW:
            ln = int(ev.width * fs)
            a = int(round(ev.t0 * fs)) - ln // 2
            t = torch.arange(ln, device=device, dtype=torch.float64)
            env = 0.5 - 0.5 * torch.cos(2 * math.pi * t / max(ln - 1, 1))
            tone = 2.0 * spec.sigma * env * torch.cos(2 * math.pi * ev.freq * 1e6 * t / fs)
            a0, b0 = max(0, a), min(n, a + ln)
            if b0 > a0:
                v[a0:b0] += tone[a0 - a:b0 - a].to(torch.float32)
    return torch.clamp(torch.round(v), -spec.clip, spec.clip).to(torch.int8)
