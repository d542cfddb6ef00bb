"""Pins of the scintillation-mode oracle (PONDER Sec. 3.5): the band-collapsed
cross-power series and the accumulated fluctuation spectrum, against Parseval's
theorem, a sinusoid's closed form and hand-made chunking."""
import numpy as np
import pytest

from oracle import incoherent as inc
from oracle import ips


def _cid_plan(nchan=64, nint=4, dm=0.0):
    return inc.make_plan(326.5, 16.0, 32e6, dm, nchan, nint, inc.CID, 2, 16, 0.5)


def test_collapse_of_identical_halves_is_the_block_energy():
    """With S = N the cross-power is N's power; summed over bins 0 .. R/2-1 it is,
    by Parseval for a real block of R samples, (R sum x^2 + X_0^2 - X_{R/2}^2) / 2
    with X_0 = sum x and X_{R/2} = sum (-1)^n x, added over the nint blocks."""
    rng = np.random.default_rng(2)
    nchan, nint, U = 64, 4, 5
    R = 2 * nchan
    n = rng.integers(-127, 128, R * nint * U + 17).astype(np.int8)
    c = ips.collapsed_series(_cid_plan(nchan, nint), np.repeat(n, 2))
    want = np.zeros(U)
    alt = (-1.0) ** np.arange(R)
    for u in range(U):
        for i in range(nint):
            x = n[(u * nint + i) * R:(u * nint + i + 1) * R].astype(np.float64)
            want[u] += (R * np.sum(x * x) + np.sum(x) ** 2 - np.sum(alt * x) ** 2) / 2
    assert np.allclose(c, want, rtol=1e-12)


def test_collapse_needs_cid_at_dm_zero():
    with pytest.raises(inc.IncoPlanError):
        ips.collapsed_series(_cid_plan(dm=1.0), np.zeros(4096, np.int8))
    with pytest.raises(inc.IncoPlanError):
        ips.collapsed_series(inc.make_plan(326.5, 16.0, 32e6, 0.0, 64, 1, inc.AID, 2, 16, 0.5),
                             np.zeros(4096, np.int8))


@pytest.mark.parametrize("f0", [1, 37, 127])
def test_sinusoid_fluctuation_spectrum(f0):
    """c[u] = B + A cos(2 pi f0 u / L + theta): S[0] = (B L)^2, S[f0] = (A L / 2)^2,
    every other bin zero; J chunks add J times that."""
    L, J = 256, 3
    u = np.arange(L * J + 100)                  # a ragged tail of 100 samples
    A, B, theta = 3.0, 10.0, 0.7
    c = B + A * np.cos(2 * np.pi * f0 * u / L + theta)
    S, nj = ips.accumulated_spectrum(c, L)
    assert nj == J and S.shape == (L // 2 + 1,)
    assert S[0] == pytest.approx(J * (B * L) ** 2, rel=1e-12)
    assert S[f0] == pytest.approx(J * (A * L / 2) ** 2, rel=1e-12)
    rest = np.delete(S, [0, f0])
    assert np.abs(rest).max() < 1e-18 * S[0]


def test_fluctuation_parseval_and_nyquist():
    """sum_f w_f S_j[f] = L sum_u c^2 per chunk (w = 1 at DC and Nyquist, 2 elsewhere);
    an alternating series puts everything into the Nyquist bin."""
    rng = np.random.default_rng(6)
    L = 64
    c = rng.normal(size=5 * L)
    S = ips.fluctuation_spectra(c, L)
    w = np.full(L // 2 + 1, 2.0)
    w[0] = w[-1] = 1.0
    for j in range(5):
        assert np.sum(w * S[j]) == pytest.approx(L * np.sum(c[j * L:(j + 1) * L] ** 2), rel=1e-12)
    alt = (-1.0) ** np.arange(L)
    Sa = ips.fluctuation_spectra(alt, L)[0]
    assert Sa[-1] == pytest.approx(L ** 2) and np.abs(Sa[:-1]).max() < 1e-20 * L ** 2


def test_chunks_are_consecutive_and_complete():
    """Accumulation adds the chunks' own spectra; a tail shorter than L is dropped."""
    L = 32
    u = np.arange(L)
    c = np.concatenate([np.cos(2 * np.pi * 3 * u / L), np.cos(2 * np.pi * 5 * u / L), np.ones(L - 1)])
    S, J = ips.accumulated_spectrum(c, L)
    assert J == 2
    assert S[3] == pytest.approx((L / 2) ** 2) and S[5] == pytest.approx((L / 2) ** 2)
    assert S[0] < 1e-20
    with pytest.raises(ValueError):
        ips.fluctuation_spectra(c, 48)
