"""Pins of the phase-model fold and pulse stacks (PONDER Sec. 3.4 fold with a
predicted period; Sec. 4 single-pulse stack): the constant-period fold as a
special case, a spin-down pulse train's closed-form arrival times, row counts
at phase wraps and sub-integration boundaries, and a phase offset's rotation."""
import numpy as np
import pytest

from oracle import pcd
from oracle import stack as st


def test_constant_period_is_the_plain_fold():
    """phi = g dt / P with exactly representable dt, 1/P and dt/P: bin for bin the
    constant-period rule floor(frac(g inc) nbins), inc = dt / P."""
    dt, P, nbins = 2.0 ** -16, 0.25, 64
    y = np.random.default_rng(1).normal(size=50_000)
    g0 = 1234
    t_ref, c = st.spin_model(P)
    s, h = st.fold(y, g0, dt, c, t_ref, nbins)
    g = np.arange(g0, g0 + len(y), dtype=np.float64)
    x = g * (dt / P)
    b = np.minimum(((x - np.floor(x)) * nbins).astype(np.int64), nbins - 1)
    assert np.array_equal(h, np.bincount(b, minlength=nbins))
    assert np.allclose(s, np.bincount(b, weights=y, minlength=nbins), rtol=0, atol=1e-9)


def test_spin_down_pulses_line_up_in_the_stack():
    """A train with one unit sample per rotation at the closed-form arrival of phase
    k + 25.5/50 (the middle of bin 25) under phi = tau/P - Pdot tau^2 / (2 P^2):
    every row of the single-pulse stack holds its pulse in bin 25 (rounding the
    arrival to the sample grid moves it by 0.001 of a turn, a twentieth of a bin);
    with Pdot dropped from the model the pulses drift out of it."""
    P, pdot, dt, nbins = 0.05, 4e-5, 1e-4, 50
    epoch = 0.0123
    n = int(2.0 / dt)
    y = np.zeros(n)
    a = -pdot / (2 * P * P)
    k = np.arange(0, 60)
    # tau with a tau^2 + tau / P = k + 25.5 / 50 (the root near k P)
    tau = (-1 / P + np.sqrt(1 / P ** 2 + 4 * a * (k + 25.5 / nbins))) / (2 * a)
    gk = np.rint((tau + epoch) / dt).astype(np.int64)
    gk = gk[(gk >= 0) & (gk < n)]
    y[gk] = 1.0
    t_ref, c = st.spin_model(P, pdot, epoch)
    S, H, q0 = st.stack(y, 0, dt, c, t_ref, nbins)
    rows = np.nonzero(S.sum(axis=1))[0]
    assert len(rows) == len(gk)
    assert np.all(np.argmax(S[rows], axis=1) == nbins // 2)
    t_ref2, c2 = st.spin_model(P, 0.0, epoch)
    S2, _, _ = st.stack(y, 0, dt, c2, t_ref2, nbins)
    assert np.any(np.argmax(S2[np.nonzero(S2.sum(axis=1))[0]], axis=1) != nbins // 2)


def test_rows_change_at_phase_wraps_and_subint_boundaries():
    """Single-pulse rows: floor(phi_last) - floor(phi_first) + 1 of them, each full
    rotation holding P / dt samples; sub-integration rows: ceil(n / n_sub), each
    full one holding n_sub samples; both sum to the plain fold."""
    dt, P, nbins = 2.0 ** -12, 0.125, 32           # 512 samples per rotation, exactly
    y = np.random.default_rng(2).normal(size=10_000)
    g0 = 300
    t_ref, c = st.spin_model(P, 0.0, 0.0, 0.1)
    S, H, q0 = st.stack(y, g0, dt, c, t_ref, nbins)
    x0 = g0 * dt / P + 0.1
    x1 = (g0 + len(y) - 1) * dt / P + 0.1
    assert S.shape[0] == int(np.floor(x1)) - int(np.floor(x0)) + 1 and q0 == int(np.floor(x0))
    assert np.all(H[1:-1].sum(axis=1) == 512)
    Ss, Hs, _ = st.stack(y, g0, dt, c, t_ref, nbins, mode=st.SUBINT, n_sub=3000)
    assert Ss.shape[0] == 4 and np.all(Hs[:3].sum(axis=1) == 3000) and Hs[3].sum() == 1000
    f, fh = st.fold(y, g0, dt, c, t_ref, nbins)
    assert np.array_equal(H.sum(axis=0), fh) and np.array_equal(Hs.sum(axis=0), fh)
    assert np.allclose(S.sum(axis=0), f) and np.allclose(Ss.sum(axis=0), f)


def test_phase_offset_rotates_the_profile():
    """A quarter-turn phase offset moves every sample nbins / 4 bins on (exact
    arithmetic: dt, 1/P and the offset are binary fractions)."""
    dt, P, nbins = 2.0 ** -14, 0.5, 64
    y = np.random.default_rng(3).normal(size=40_000)
    t_ref, c = st.spin_model(P)
    _, c4 = st.spin_model(P, 0.0, 0.0, 0.25)
    s, h = st.fold(y, 0, dt, c, t_ref, nbins)
    s4, h4 = st.fold(y, 0, dt, c4, t_ref, nbins)
    assert np.array_equal(np.roll(h, nbins // 4), h4)
    assert np.allclose(np.roll(s, nbins // 4), s4, rtol=0, atol=1e-9)


def test_cubic_phase_matches_direct_polynomial():
    """Horner's rule gives the polynomial's value (to rounding) for four
    coefficients, and the model is checked for running backwards."""
    c = np.array([0.3, 7.0, -0.02, 1e-4])
    g = np.arange(0, 100_000, 37)
    dt, t_ref = 1e-4, 2.5
    tau = g * dt - t_ref
    want = c[0] + c[1] * tau + c[2] * tau ** 2 + c[3] * tau ** 3
    assert np.allclose(st.phase(c, t_ref, g, dt), want, rtol=0, atol=1e-10)
    with pytest.raises(ValueError):
        st.stack(np.ones(10), 0, 1.0, [0.0, -1.0], 0.0, 8)
    with pytest.raises(ValueError):
        st.phase(np.ones(9), 0.0, g, dt)


def test_the_coherent_fold_rule_is_the_same_rule():
    """The coherent oracle's fold and this one's ROTATION stack, summed over rows,
    agree bin for bin when inc is exactly representable."""
    p = pcd.make_plan(326.5, 16.0, 32e6, 0.0, 1 << 12, 1, 16, 2.0 ** -6)
    y = np.random.default_rng(4).normal(size=8192)
    s_ref, h_ref = pcd.fold(p, y, 100)
    t_ref, c = st.spin_model(2.0 ** -6)
    s, h = st.fold(y, 100, p.dtc, c, t_ref, 16)
    assert p.inc == p.dtc * 2.0 ** 6
    assert np.array_equal(h, h_ref) and np.allclose(s, s_ref)
