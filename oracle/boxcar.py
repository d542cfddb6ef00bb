"""FP64 CPU oracle of the boxcar S/N single-pulse detector -- TEST INFRASTRUCTURE.

The paper only names automatic transient detection as a plan (Sec. 5); the
detector here is the plain matched-filter search the batched DM trials feed:

* per trial series T_d (n samples): mu = median(T_d), sigma = 1.4826 MAD, with
  MAD = median(|T_d - mu|); the median of an even count is the mean of the two
  middle values, taken in FP64;
* for widths w in {1, 2, 4, ..., 64} and starts t with t + w <= n:
  S_w(d, t) = (sum_{i<w} T_d[t+i] - w mu) / (sigma sqrt(w)); the boxcar sum is
  accumulated in FP64 in index order (i = 0, 1, ..., w-1);
* s(d, t) = max over w of S_w(d, t), w*(d, t) its smallest maximising width;
* (d, t) is a candidate when s(d, t) >= threshold and no point (d', t') with
  |d' - d| <= 2 and |t' - t| <= w*(d, t) beats it: s(d', t') > s(d, t), or an
  equal s at an earlier (d', t') in (trial, sample) order.

Every floating-point step is a single correctly rounded IEEE operation, so
the CUDA kernels reproduce these values bit for bit.
"""
from __future__ import annotations

import numpy as np

WIDTHS = (1, 2, 4, 8, 16, 32, 64)
MAD_SCALE = 1.4826


def median_fp64(x: np.ndarray) -> float:
    """Median; for an even count the FP64 mean of the two middle values."""
    x = np.asarray(x)
    n = len(x)
    s = np.sort(x)
    if n % 2:
        return float(s[n // 2])
    return (float(s[n // 2 - 1]) + float(s[n // 2])) / 2.0


def robust_stats(T: np.ndarray) -> tuple[float, float]:
    """(mu, sigma) of one series: median and 1.4826 x median absolute deviation."""
    mu = median_fp64(T)
    dev = np.abs(np.asarray(T, dtype=np.float64) - mu)
    return mu, MAD_SCALE * median_fp64(dev)


def snr_planes(T: np.ndarray, mu: float, sigma: float) -> tuple[np.ndarray, np.ndarray]:
    """s(t) and w*(t) of one series (s = -inf where no width fits)."""
    T = np.asarray(T, dtype=np.float64)
    n = len(T)
    best = np.full(n, -np.inf)
    bw = np.zeros(n, dtype=np.int32)
    acc = np.zeros(n)
    done = 0
    for w in WIDTHS:
        # extend the running sums from `done` terms to `w` terms, in index order
        for i in range(done, w):
            acc[:max(0, n - i)] += T[i:]
        done = w
        valid = n - w + 1
        if valid <= 0:
            break
        s = (acc[:valid] - w * mu) / (sigma * np.sqrt(float(w)))
        better = s > best[:valid]
        best[:valid][better] = s[better]
        bw[:valid][better] = w
    return best, bw


def detect(series: np.ndarray, threshold: float = 6.0, trial_radius: int = 2):
    """Candidates of a [ndm, n] series block: list of (trial, t, width, snr), sorted."""
    series = np.asarray(series)
    ndm, n = series.shape
    S = np.full((ndm, n), -np.inf)
    W = np.zeros((ndm, n), dtype=np.int32)
    for d in range(ndm):
        mu, sigma = robust_stats(series[d])
        if sigma > 0:               # a constant series has no scale: no candidates
            S[d], W[d] = snr_planes(series[d], mu, sigma)
    out = []
    for d, t in zip(*np.nonzero(S >= threshold)):
        s, w = S[d, t], int(W[d, t])
        d0, d1 = max(0, d - trial_radius), min(ndm, d + trial_radius + 1)
        t0, t1 = max(0, t - w), min(n, t + w + 1)
        keep = True
        for dd in range(d0, d1):
            for tt in range(t0, t1):
                if (dd, tt) == (d, t):
                    continue
                o = S[dd, tt]
                if o > s or (o == s and (dd, tt) < (d, t)):
                    keep = False
                    break
            if not keep:
                break
        if keep:
            out.append((int(d), int(t), w, float(s)))
    return out
