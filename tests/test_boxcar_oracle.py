"""Pins of the boxcar detector oracle: order statistics from the standard
library, closed-form S/N of a box pulse, and the suppression rule."""
import math
import statistics

import numpy as np
import pytest

from oracle import boxcar


@pytest.mark.parametrize("n", [1, 2, 7, 10, 101, 1000])
def test_median_and_mad_match_stdlib(n):
    x = np.random.default_rng(n).standard_normal(n).astype(np.float32) * 5 + 100
    assert boxcar.median_fp64(x) == statistics.median([float(v) for v in x])
    mu, sig = boxcar.robust_stats(x)
    mad = statistics.median([abs(float(v) - mu) for v in x])
    assert sig == 1.4826 * mad


def test_robust_stats_closed_form():
    mu, sig = boxcar.robust_stats(np.arange(1, 102, dtype=np.float32))
    assert mu == 51.0 and sig == 1.4826 * 25.0


def test_box_pulse_snr_closed_form_and_single_candidate():
    """Alternating background c +- 1 with a box of height h on w0 samples.
    Counting order statistics: 8 of the c-1 samples move above c+1, so the
    median is c+1 and the MAD is 2 (sigma = 2 x 1.4826); the box of width w0
    starting at t0 gives S = (sum of its samples - w0 (c+1)) / (sigma sqrt(w0))
    and is the one candidate."""
    n, c, h, w0, t0 = 4096, 50.0, 9.0, 16, 2000
    T = c + np.where(np.arange(n) % 2 == 0, -1.0, 1.0)
    T[t0:t0 + w0] += h
    T = T.astype(np.float32)
    flat = (np.full(n, c) + np.where(np.arange(n) % 2, 1.0, -1.0)).astype(np.float32)
    mu, sig = boxcar.robust_stats(T)
    assert mu == c + 1 and sig == 1.4826 * 2
    want = (float(np.sum(T[t0:t0 + w0].astype(np.float64))) - w0 * (c + 1)) / (1.4826 * 2 * math.sqrt(w0))
    assert boxcar.detect(np.stack([T, flat])) == [(0, t0, w0, want)]


def test_suppression_across_trials_and_ties():
    n = 2048
    rng = np.random.default_rng(5)
    base = (100 + rng.standard_normal((5, n))).astype(np.float32)
    amp = [2.0, 5.0, 9.0, 5.0, 2.0]              # one event peaking in trial 2
    for d in range(5):
        base[d, 1000:1008] += amp[d]
    c = boxcar.detect(base)
    assert [(d, t) for d, t, w, s in c if 990 <= t <= 1010] == [(2, 1000)]
    # identical copies: the earlier trial wins the tie
    twin = np.stack([base[2], base[2]])
    c2 = boxcar.detect(twin)
    assert [(d, t) for d, t, w, s in c2 if 990 <= t <= 1010] == [(0, 1000)]


def test_constant_series_has_no_candidates():
    assert boxcar.detect(np.full((3, 100), 7.0, np.float32)) == []
