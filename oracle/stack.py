"""FP64 CPU oracle for folding with a phase model and for pulse stacks -- TEST
INFRASTRUCTURE.

Only the test suite, the smoke check and the benchmark's CPU legs may import
this module; the engine never does and shares no code with it.

What it computes (PONDER, Naidu et al.: the fold thread folds "with appropriate
period, obtained from the TEMPO2 predictors", Sec. 3.4; Sec. 4 shows a stack of
the single pulses of J1709-1640, one row per rotation):

1. the pulsar's rotational phase at series sample g (sample time t = g dt from
   the first stream sample) from a polynomial phase model about a reference
   time t_ref:  phi(g) = sum_i c_i tau^i,  tau = g dt - t_ref  (cycles; c_1 is
   the spin frequency 1/P, c_2 = -Pdot / (2 P^2), ...), evaluated by Horner's
   rule, each multiply and add rounded on its own in FP64;
2. rotation q = floor(phi), bin b = min(floor((phi - q) nbins), nbins - 1) (the
   constant-period fold's rule with phi in place of g inc);
3. a stack S[row][b] of the series and its hit counts H[row][b], where the row
   is the rotation counted from the first sample's (single-pulse stack), or
   (g - g0) // n_sub (sub-integrations of n_sub samples); summing the rows gives
   the folded profile.

Reading (the predictors themselves come from TEMPO2, an external program): the
phase model is a plain polynomial in seconds of up to eight coefficients; a
spin-down model (P, Pdot, epoch) is one such polynomial.
"""
from __future__ import annotations

import numpy as np

ROTATION = 0
SUBINT = 1
MAX_COEFFS = 8


def spin_model(period: float, pdot: float = 0.0, epoch_s: float = 0.0, phase0: float = 0.0):
    """(t_ref, coefficients) of phi = phase0 + tau / P - Pdot tau^2 / (2 P^2)."""
    c = [phase0, 1.0 / period]
    if pdot:
        c.append(-pdot / (2.0 * period * period))
    return epoch_s, np.array(c, dtype=np.float64)


def phase(coeffs, t_ref: float, g, dt: float) -> np.ndarray:
    """phi(g) by Horner's rule, every operation rounded separately in FP64."""
    c = np.asarray(coeffs, dtype=np.float64)
    if not 1 <= len(c) <= MAX_COEFFS:
        raise ValueError("1 .. 8 phase coefficients")
    tau = np.asarray(g, dtype=np.float64) * dt - t_ref
    x = np.full_like(tau, c[-1])
    for ci in c[-2::-1]:
        x = x * tau
        x = x + ci
    return x


def rotation_and_bin(coeffs, t_ref: float, g, dt: float, nbins: int):
    x = phase(coeffs, t_ref, g, dt)
    q = np.floor(x)
    b = np.minimum(((x - q) * nbins).astype(np.int64), nbins - 1)
    return q.astype(np.int64), b


def stack(series, g0: int, dt: float, coeffs, t_ref: float, nbins: int, mode: int = ROTATION, n_sub: int = 0):
    """(S, H, first_rotation): the stack of series[i] (sample g0 + i) and its hits."""
    y = np.asarray(series, dtype=np.float64)
    g = np.arange(g0, g0 + len(y), dtype=np.int64)
    if len(y) == 0:
        return np.zeros((0, nbins)), np.zeros((0, nbins), np.int64), 0
    q, b = rotation_and_bin(coeffs, t_ref, g, dt, nbins)
    if np.any(np.diff(q * nbins + b) < 0):
        raise ValueError("the phase model must not run backwards over the series")
    if mode == ROTATION:
        row = q - q[0]
    elif mode == SUBINT:
        if n_sub < 1:
            raise ValueError("n_sub >= 1")
        row = (g - g0) // n_sub
    else:
        raise ValueError("mode")
    nrows = int(row.max()) + 1
    S = np.zeros((nrows, nbins))
    H = np.zeros((nrows, nbins), np.int64)
    np.add.at(S, (row, b), y)
    np.add.at(H, (row, b), 1)
    return S, H, int(q[0])


def fold(series, g0: int, dt: float, coeffs, t_ref: float, nbins: int):
    """The folded profile: the stack summed over its rows."""
    S, H, _ = stack(series, g0, dt, coeffs, t_ref, nbins)
    return S.sum(axis=0), H.sum(axis=0)
