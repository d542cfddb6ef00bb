"""cuFFT comparison path for coherent dedispersion (timed beside the engine).

This is the library-FFT way to compute what the engine computes (PONDER
Sec. 3.7), written with torch on the GPU: per overlap-save segment of N real
samples

  X = cuFFT R2C of the float32 segment, Nyquist bin dropped (k < N/2);
  Y[k] = X[k] exp(-2 pi i sgn c(f_k)), c(f) = K 1e6 DM f^2 / (f0^2 (f0 + f))
         (Eq. 4; the response is one complex64 table built once in FP64);
  v_c = cuFFT batched C2C inverse of each sub-channel's M bins (1/M included);
  keep n_past <= m < M - n_fut, P = sum_c |v_c|^2;

then the fold (FP64 phase, FP64 sums) and the decimation (exact integer
binning) with torch scatter-adds.  It is a baseline, not the product: it runs
several library and elementwise kernels per segment where the engine runs
four fused passes.  It shares no code with the engine or the oracle.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

K_DM = 1.0 / 2.41e-4    # s MHz^2 (Eq. 1 constant)


@dataclass
class Geometry:
    nfft: int
    nchan: int
    L: int
    M: int
    n_past: int
    n_fut: int
    S_c: int
    S: int


def geometry(f0: float, bw: float, fs: float, dm: float, nfft: int, nchan: int) -> Geometry:
    """Overlap-save geometry: the filter spans the smear above and below f0."""
    L = nfft // 2
    M = L // nchan
    dtc = 2.0 * nchan / fs
    half = abs(bw) / 2.0
    n_past = math.ceil(K_DM * dm * (f0 ** -2 - (f0 + half) ** -2) / dtc)
    n_fut = math.ceil(K_DM * dm * ((f0 - half) ** -2 - f0 ** -2) / dtc)
    S_c = M - n_past - n_fut
    if S_c <= 0:
        raise ValueError("nfft too short for this DM")
    return Geometry(nfft, nchan, L, M, n_past, n_fut, S_c, 2 * nchan * S_c)


class CufftPath:
    def __init__(self, f0, bw, fs, dm, nfft, nchan, nbins, period, t_dec, device):
        import torch
        self.torch = torch
        self.g = geometry(f0, bw, fs, dm, nfft, nchan)
        self.dev = device
        self.nbins = nbins
        self.inc = (2.0 * nchan / fs) / period
        # decimation: j = floor(g den / num) with D = t_dec fs / (2 nchan) = num / den
        t_ns = int(round(t_dec * 1e9))
        num, den = t_ns * int(fs), 1_000_000_000 * 2 * nchan
        q = math.gcd(num, den)
        self.num, self.den = num // q, den // q
        # inverse ISM response, FP64 phase reduced mod 1 before the complex64 cast
        k = torch.arange(self.g.L, dtype=torch.float64, device=device)
        du = fs / nfft * 1e-6
        half = abs(bw) / 2.0
        f = k * du - half if bw > 0 else half - k * du
        c = K_DM * 1e6 * dm * f * f / (f0 * f0 * (f0 + f))
        c = c - torch.round(c)
        sgn = 1.0 if bw > 0 else -1.0
        self.H = torch.polar(torch.ones_like(c), -2.0 * math.pi * sgn * c).to(torch.complex64)

    def run(self, x):
        """Whole int8 stream (device tensor) -> (profile sums FP64, hits int64,
        series FP64 sums, series counts int64, first series index)."""
        torch = self.torch
        g = self.g
        n_total = x.numel()
        g_end = n_total // (2 * g.nchan) - g.n_fut
        prof = torch.zeros(self.nbins, dtype=torch.float64, device=self.dev)
        hits = torch.zeros(self.nbins, dtype=torch.int64, device=self.dev)
        j_first = (g.n_past * self.den) // self.num
        j_last = (max(g_end - 1, g.n_past) * self.den) // self.num
        nj = max(0, j_last - j_first + 1)
        T = torch.zeros(nj, dtype=torch.float64, device=self.dev)
        C = torch.zeros(nj, dtype=torch.int64, device=self.dev)
        s = 0
        while True:
            g0 = s * g.S_c + g.n_past
            if g0 >= g_end:
                break
            a = s * g.S
            seg = x[a:a + g.nfft].to(torch.float32)
            if seg.numel() < g.nfft:
                seg = torch.nn.functional.pad(seg, (0, g.nfft - seg.numel()))
            X = torch.fft.rfft(seg)[:g.L]
            v = torch.fft.ifft((X * self.H).reshape(g.nchan, g.M), dim=1)
            v = v[:, g.n_past:g.M - g.n_fut]
            P = (v.real * v.real + v.imag * v.imag).sum(dim=0)
            nv = min(g.S_c, g_end - g0)
            P = P[:nv].to(torch.float64)
            gi = torch.arange(g0, g0 + nv, dtype=torch.int64, device=self.dev)
            ph = gi.to(torch.float64) * self.inc
            b = torch.clamp(((ph - torch.floor(ph)) * self.nbins).to(torch.int64), max=self.nbins - 1)
            prof.index_add_(0, b, P)
            hits.index_add_(0, b, torch.ones_like(b))
            j = (gi * self.den) // self.num - j_first
            T.index_add_(0, j, P)
            C.index_add_(0, j, torch.ones_like(j))
            s += 1
        return prof, hits, T, C, j_first
