"""FP64 CPU oracle for the interplanetary scintillation mode -- TEST INFRASTRUCTURE.

Only the test suite, the smoke check and the benchmark's CPU legs may import
this module; the engine never does and shares no code with it.

What it computes (PONDER, Naidu et al., Sec. 3.5 "Inter planetary scintillation
mode"): the two halves are correlated as in the CID mode (FFT filterbank,
cross-spectra Re(X_N conj X_S)), the cross-spectra are integrated and collapsed
over the band into an intensity scintillation series, the series is integrated
further, and the temporal power spectrum of consecutive stretches of it (the
fluctuation spectrum) is accumulated:

1. c[u] = sum_k F_CID[u][k], F_CID the CID filterbank integrated over nint
   spectra (the incoherent oracle at DM 0, where every channel delay is zero);
2. the further integration to the spectra's time resolution is linear, so it is
   the same as integrating nint * m spectra in step 1;
3. chunk j of L samples, S_j[f] = |sum_u c[j L + u] exp(-2 pi i f u / L)|^2,
   f = 0 .. L/2 (DC and Nyquist included; no window, no mean removed);
4. A[f] = sum_j S_j[f] over the complete chunks; a trailing partial chunk is
   not used.
"""
from __future__ import annotations

import numpy as np

from oracle import incoherent as inc


def collapsed_series(p: inc.IncoPlan, raw: np.ndarray) -> np.ndarray:
    """Step 1: the band-collapsed cross-power series (the CID series at DM 0)."""
    if p.mode != inc.CID or p.dm != 0:
        raise inc.IncoPlanError("the scintillation series is the CID series at DM 0")
    r = inc.run(p, raw)
    assert r.t_first == 0
    return r.D


def fluctuation_spectra(c: np.ndarray, L: int) -> np.ndarray:
    """Step 3: S_j[f] for every complete chunk j, shape (J, L/2 + 1)."""
    if L < 2 or L & (L - 1):
        raise ValueError("L must be a power of two")
    J = len(c) // L
    X = np.fft.fft(np.asarray(c[:J * L], dtype=np.float64).reshape(J, L), axis=1)[:, :L // 2 + 1]
    return X.real ** 2 + X.imag ** 2


def accumulated_spectrum(c: np.ndarray, L: int) -> tuple[np.ndarray, int]:
    """Step 4: (A, J), A[f] summed over the J complete chunks."""
    S = fluctuation_spectra(c, L)
    return S.sum(axis=0), S.shape[0]


def run(p: inc.IncoPlan, raw: np.ndarray, L: int):
    """(collapsed series, accumulated fluctuation spectrum, chunks)."""
    c = collapsed_series(p, raw)
    A, J = accumulated_spectrum(c, L)
    return c, A, J
