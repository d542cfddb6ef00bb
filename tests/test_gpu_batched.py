"""Batched DM trials on the GPU vs the oracle's batched form, through the C ABI.

Trial d of a batched plan is the single-DM path at DM_d on its group's
segmentation (the group's FFT length, with the overlap of the group's largest
DM) over the common output range of the plan's largest DM; the oracle computes
exactly that (oracle.pcd.run_batched).  Tolerance as for single-DM series:
relative L2 <= 1e-4 per trial, counts and indices exact.
"""
import numpy as np
import pytest

from oracle import pcd
from paper_1503_01405_gb300 import pond, synth

pytestmark = pytest.mark.gpu
TOL = 1e-4
F0, BW, FS = 326.5, 16.0, 32e6


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1503_01405_gb300 import build as pbuild
    pbuild.build()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def run_engine(x, dms, nfft, nchan, t_dec, chunks=None, **kw):
    with pond.Engine(F0, BW, FS, 0.0, nfft, nchan, 1, 1.0, t_dec=t_dec, dms=dms, **kw) as e:
        pos = 0
        for c in (chunks or [len(x)]):
            e.push(x[pos:pos + c])
            pos += c
        e.flush()
        T, C, j0 = e.timeseries()
        dm_out, nf = e.trials()
    return T, C, j0, nf


def oracle_batched(x, dms, nfft_of, nchan, t_dec):
    base = pcd.make_plan(F0, BW, FS, 0.0, int(min(nfft_of)), nchan, 1, 1.0, t_dec)
    gmax = {}
    for dm, nf in zip(dms, nfft_of):
        gmax[nf] = max(gmax.get(nf, 0.0), dm)
    return pcd.run_batched(base, [(dm, nf, gmax[nf]) for dm, nf in zip(dms, nfft_of)], x)


def stream(n, seed, dm=0.2):
    return synth.make_stream(synth.StreamSpec(n=n, seed=seed, dm=dm, period=0.011, snr=80.0, duty=0.05))


def test_batched_fixed_nfft_matches_oracle():
    dms = [0.0, 0.05, 0.3, 0.15, 0.25]
    nfft, nchan, t_dec = 1 << 16, 16, 8e-6
    x = stream(7 * (1 << 16) + 12345, seed=31)
    T, C, j0, nf = run_engine(x, dms, nfft, nchan, t_dec)
    assert np.all(nf == nfft)
    res = oracle_batched(x, dms, nf, nchan, t_dec)
    assert T.shape[0] == len(dms)
    for d, r in enumerate(res):
        assert j0 == r.ts_first
        assert np.array_equal(C, r.ts_counts)
        assert rel(T[d], r.ts) <= TOL, (d, rel(T[d], r.ts))


def test_batched_autotune_groups_match_oracle():
    dms = list(np.linspace(0.0, 0.6, 9))
    nchan, t_dec = 16, 8e-6
    x = stream(6 * (1 << 17) + 999, seed=32, dm=0.4)
    T, C, j0, nf = run_engine(x, dms, 1 << 17, nchan, t_dec,
                              nfft_choices=(1 << 15, 1 << 16, 1 << 17), autotune=True)
    # every group's FFT length carries its largest DM; lengths grow with DM
    for nfft in set(nf.tolist()):
        gm = max(dm for dm, n in zip(dms, nf) if n == nfft)
        pcd.make_plan(F0, BW, FS, gm, int(nfft), nchan, 1, 1.0, t_dec)
    assert all(np.diff(nf[np.argsort(dms)]) >= 0)
    res = oracle_batched(x, dms, nf, nchan, t_dec)
    for d, r in enumerate(res):
        assert j0 == r.ts_first and np.array_equal(C, r.ts_counts)
        assert rel(T[d], r.ts) <= TOL, (d, nf[d], rel(T[d], r.ts))


def test_batched_streaming_invariance_bit_exact():
    dms = [0.1, 0.0, 0.2]
    x = stream(5 * (1 << 15) + 4321, seed=33)
    a = run_engine(x, dms, 1 << 15, 8, 8e-6)
    rng = np.random.default_rng(3)
    cuts, left = [], len(x)
    while left > 0:
        c = int(min(left, rng.integers(1, 70_000)))
        cuts.append(c)
        left -= c
    b = run_engine(x, dms, 1 << 15, 8, 8e-6, chunks=cuts)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]


def test_single_trial_batch_equals_single_dm_plan():
    dm, nfft, nchan, t_dec = 0.2, 1 << 15, 8, 8e-6
    x = stream(6 * nfft, seed=34)
    T, C, j0, _ = run_engine(x, [dm], nfft, nchan, t_dec)
    with pond.Engine(F0, BW, FS, dm, nfft, nchan, 16, 0.011, t_dec=t_dec) as e:
        e.push(x)
        e.flush()
        Ts, Cs, js = e.timeseries()
    assert js == j0 and np.array_equal(Cs, C)
    assert rel(T[0], Ts) <= 1e-5


def test_batched_three_pass_matches_oracle():
    """Trials of a plan with M = 64 R2 (nfft 2^21, 16 sub-channels: two sub-channel
    groups per column) run F1 and F2 once, then per trial the row pass with the
    trial's chirp and the column pass; both schedules against the oracle."""
    dms = [0.0, 1.5, 3.0, 0.5, 2.2]
    nfft, nchan, t_dec = 1 << 21, 16, 16e-6
    p = pcd.make_plan(F0, BW, FS, max(dms), nfft, nchan, 1, 1.0, t_dec)
    x = stream(3 * p.S + nfft + 777, seed=35, dm=1.5)
    res = oracle_batched(x, dms, [nfft] * len(dms), nchan, t_dec)
    for sched in (pond.POND_SCHEDULE_AUTO, pond.POND_SCHEDULE_FOUR_PASS):
        T, C, j0, nf = run_engine(x, dms, nfft, nchan, t_dec, schedule=sched)
        assert np.all(nf == nfft) and T.shape[0] == len(dms)
        for d, r in enumerate(res):
            assert j0 == r.ts_first and np.array_equal(C, r.ts_counts)
            assert rel(T[d], r.ts) <= TOL, (sched, d, rel(T[d], r.ts))


def test_single_trial_batch_equals_single_dm_plan_three_pass():
    """In the three-pass geometry a one-trial batched plan (F2, then the row pass
    with the chirp from the trial's anchors) and the single-DM plan (F2 with the
    chirp from the same anchors) form the same spectrum, chirp products and
    runs: identical series, bit for bit."""
    dm, nfft, nchan, t_dec = 1.0, 1 << 18, 8, 8e-6
    x = stream(8 * nfft, seed=36, dm=dm)
    T, C, j0, _ = run_engine(x, [dm], nfft, nchan, t_dec)
    with pond.Engine(F0, BW, FS, dm, nfft, nchan, 16, 0.011, t_dec=t_dec, chirp=pond.POND_CHIRP_ANCHORS) as e:
        e.push(x)
        e.flush()
        Ts, Cs, js = e.timeseries()
    assert js == j0 and np.array_equal(Cs, C)
    assert np.array_equal(T[0], Ts)


# Uniform DM grid from 0 (whole multiples of one step), three-pass geometry
# (nfft 2^21, 16 sub-channels): the forms that run several trials per launch
# against the oracle, with a trial block that does not divide the trial count.
GRID = [0.6 * d for d in range(6)]


@pytest.fixture(scope="module")
def grid_case():
    nfft, nchan, t_dec = 1 << 21, 16, 16e-6
    p = pcd.make_plan(F0, BW, FS, max(GRID), nfft, nchan, 1, 1.0, t_dec)
    x = stream(3 * p.S + nfft + 4321, seed=37, dm=1.8)
    return x, nfft, nchan, t_dec, oracle_batched(x, GRID, [nfft] * len(GRID), nchan, t_dec)


def tuned(dms, nfft, nchan, t_dec, **kw):
    with pond.Engine(F0, BW, FS, 0.0, nfft, nchan, 1, 1.0, t_dec=t_dec, dms=dms, **kw) as e:
        return e.tuning()


@pytest.mark.parametrize("mode,kt", [(pond.POND_TRIALS_PER_TRIAL, 0), (pond.POND_TRIALS_MULTI_ANCHOR, 4),
                                     (pond.POND_TRIALS_MULTI_TABLE, 4), (pond.POND_TRIALS_MULTI_TABLE, 0),
                                     (pond.POND_TRIALS_MULTI_ANCHOR, 6)])
def test_multi_trial_forms_match_oracle(grid_case, mode, kt):
    x, nfft, nchan, t_dec, res = grid_case
    T, C, j0, nf = run_engine(x, GRID, nfft, nchan, t_dec, trial_mode=mode, trials_per_launch=kt)
    info = tuned(GRID, nfft, nchan, t_dec, trial_mode=mode, trials_per_launch=kt)
    assert len(info) == 1 and info[0]["mode"] == pond.TRIAL_MODE_NAMES[mode]
    assert info[0]["trials_per_launch"] == (1 if mode == pond.POND_TRIALS_PER_TRIAL else (kt or len(GRID)))
    assert abs(info[0]["dm_step"] - 0.6) < 1e-12 or mode == pond.POND_TRIALS_PER_TRIAL
    for d, r in enumerate(res):
        assert j0 == r.ts_first and np.array_equal(C, r.ts_counts)
        assert rel(T[d], r.ts) <= TOL, (mode, kt, d, rel(T[d], r.ts))


def test_multi_anchor_form_equals_per_trial_launches_bit_exact(grid_case):
    """The multi-trial anchor form runs the same chirp, runs and column pass per
    trial as the per-trial launches: identical series, bit for bit."""
    x, nfft, nchan, t_dec, _ = grid_case
    a = run_engine(x, GRID, nfft, nchan, t_dec, trial_mode=pond.POND_TRIALS_PER_TRIAL)
    b = run_engine(x, GRID, nfft, nchan, t_dec, trial_mode=pond.POND_TRIALS_MULTI_ANCHOR, trials_per_launch=4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]


def test_multi_table_streaming_invariance_bit_exact(grid_case):
    x, nfft, nchan, t_dec, _ = grid_case
    a = run_engine(x, GRID, nfft, nchan, t_dec, trial_mode=pond.POND_TRIALS_MULTI_TABLE, trials_per_launch=4)
    rng = np.random.default_rng(5)
    cuts, left = [], len(x)
    while left > 0:
        c = int(min(left, rng.integers(1, 3_000_000)))
        cuts.append(c)
        left -= c
    b = run_engine(x, GRID, nfft, nchan, t_dec, chunks=cuts, trial_mode=pond.POND_TRIALS_MULTI_TABLE,
                   trials_per_launch=4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]


def test_table_form_falls_back_to_anchors_off_grid():
    """DMs that are not whole multiples of one step cannot use the table: the
    lane runs the anchor form (reported by pond_tuning), still against the oracle."""
    dms = [0.0, 1.0, 2.5, 2.9]
    nfft, nchan, t_dec = 1 << 21, 16, 16e-6
    info = tuned(dms, nfft, nchan, t_dec, trial_mode=pond.POND_TRIALS_MULTI_TABLE)
    assert info[0]["mode"] == "multi-anchor" and info[0]["dm_step"] == 0.0
    p = pcd.make_plan(F0, BW, FS, max(dms), nfft, nchan, 1, 1.0, t_dec)
    x = stream(2 * p.S + nfft + 99, seed=38, dm=1.0)
    T, C, j0, _ = run_engine(x, dms, nfft, nchan, t_dec, trial_mode=pond.POND_TRIALS_MULTI_TABLE)
    res = oracle_batched(x, dms, [nfft] * len(dms), nchan, t_dec)
    for d, r in enumerate(res):
        assert j0 == r.ts_first and np.array_equal(C, r.ts_counts)
        assert rel(T[d], r.ts) <= TOL, (d, rel(T[d], r.ts))


@pytest.mark.parametrize("nfft,nchan,grid,t_dec", [(1 << 18, 8, [0.0, 0.3, 0.6, 0.9], 8e-6),
                                                   (1 << 22, 32, [0.0, 2.0, 4.0, 6.0], 16e-6)])
def test_multi_trial_forms_at_other_row_lengths(nfft, nchan, grid, t_dec):
    """The multi-trial row passes at rows of 512 bins (nfft 2^18, 8
    sub-channels: 16 rows per CTA) and 2048 bins (nfft 2^22, 32 sub-channels:
    4 rows per CTA), the table form with a trial block that does not divide the
    trial count: against the oracle, and the anchor form bit for bit against
    the per-trial launches."""
    p = pcd.make_plan(F0, BW, FS, max(grid), nfft, nchan, 1, 1.0, t_dec)
    x = stream(2 * p.S + nfft + 555, seed=43, dm=grid[2])
    res = oracle_batched(x, grid, [nfft] * len(grid), nchan, t_dec)
    T, C, j0, _ = run_engine(x, grid, nfft, nchan, t_dec, trial_mode=pond.POND_TRIALS_MULTI_TABLE,
                             trials_per_launch=3)
    info = tuned(grid, nfft, nchan, t_dec, trial_mode=pond.POND_TRIALS_MULTI_TABLE, trials_per_launch=3)
    assert info[0]["mode"] == "multi-table" and info[0]["trials_per_launch"] == 3
    for d, r in enumerate(res):
        assert j0 == r.ts_first and np.array_equal(C, r.ts_counts)
        assert rel(T[d], r.ts) <= TOL, (nfft, d, rel(T[d], r.ts))
    a = run_engine(x, grid, nfft, nchan, t_dec, trial_mode=pond.POND_TRIALS_PER_TRIAL)
    b = run_engine(x, grid, nfft, nchan, t_dec, trial_mode=pond.POND_TRIALS_MULTI_ANCHOR)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]


def test_multi_anchor_form_in_a_wide_low_band():
    """A wide low band (150 MHz, 100 MHz wide, 200 MHz sampling, nfft 2^21):
    the chirp's curvature asks for 32 to 4096 anchors per trial (2^15 down to
    2^8 bins per anchor) within one launch.  The multi-trial anchor form gives
    the per-trial launches' series bit for bit, and the oracle's."""
    f0, bw, fs = 150.0, 100.0, 200e6
    dms = [0.0, 0.004, 0.008, 0.012, 0.016]
    nfft, nchan, t_dec = 1 << 21, 16, 16e-6
    p = pcd.make_plan(f0, bw, fs, max(dms), nfft, nchan, 1, 1.0, t_dec)
    x = synth.make_stream(synth.StreamSpec(n=3 * p.S + nfft + 777, seed=41, fs=fs, f0=f0, bw=bw, dm=0.008,
                                           period=0.0041, snr=80.0, duty=0.05))

    def run(mode, kt):
        with pond.Engine(f0, bw, fs, 0.0, nfft, nchan, 1, 1.0, t_dec=t_dec, dms=dms, trial_mode=mode,
                         trials_per_launch=kt) as e:
            e.push(x)
            e.flush()
            T, C, j0 = e.timeseries()
            info = e.tuning()
        return T, C, j0, info

    a = run(pond.POND_TRIALS_PER_TRIAL, 0)
    for kt in (0, 3):
        b = run(pond.POND_TRIALS_MULTI_ANCHOR, kt)
        assert b[3][0]["mode"] == "multi-anchor"
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2], kt
    base = pcd.make_plan(f0, bw, fs, 0.0, nfft, nchan, 1, 1.0, t_dec)
    res = pcd.run_batched(base, [(dm, nfft, max(dms)) for dm in dms], x)
    for d, r in enumerate(res):
        assert a[2] == r.ts_first and np.array_equal(a[1], r.ts_counts)
        assert rel(a[0][d], r.ts) <= TOL, (d, rel(a[0][d], r.ts))


def test_trial_autotuner_times_every_form(grid_case):
    """With autotune the lane's forms (per-trial launches; anchors and table at 8
    and 32 trials per launch, clipped to the trial count; the four-pass form at
    the default inverse split 2^8 x 2^8 and its nearest admissible neighbours)
    are timed, the fastest per trial runs, and the result still matches the
    oracle."""
    x, nfft, nchan, t_dec, res = grid_case
    info = tuned(GRID, nfft, nchan, t_dec, autotune=True, nfft_choices=(nfft,))
    c = info[0]["candidates_us_per_trial"]
    assert {k["mode"] for k in c} == {"per-trial", "multi-anchor", "multi-table", "four-pass"}
    assert sorted(k["inv_split"] for k in c if k["mode"] == "four-pass") == [6, 7, 8, 9]
    assert all(k["inv_split"] == 0 for k in c if k["mode"] != "four-pass")
    assert all(k["us"] > 0 for k in c)
    best = min(c, key=lambda k: k["us"])
    assert info[0]["mode"] == best["mode"]
    if best["mode"] == "four-pass":
        assert info[0]["inv_split"] == best["inv_split"]
    T, C, j0, nf = run_engine(x, GRID, nfft, nchan, t_dec, autotune=True, nfft_choices=(nfft,))
    for d, r in enumerate(res):
        assert j0 == r.ts_first and np.array_equal(C, r.ts_counts)
        assert rel(T[d], r.ts) <= TOL, (d, rel(T[d], r.ts))


@pytest.mark.parametrize("q", [4, 6, 8, 9])
def test_four_pass_trials_at_each_split_match_oracle(grid_case, q):
    """Every trial through I1 + I2 at inverse split 2^q x 2^(16-q) (the tile
    shape of the per-sub-channel inverse) against the oracle."""
    x, nfft, nchan, t_dec, res = grid_case
    T, C, j0, nf = run_engine(x, GRID, nfft, nchan, t_dec, trial_mode=pond.POND_TRIALS_FOUR_PASS, inv_split=q)
    info = tuned(GRID, nfft, nchan, t_dec, trial_mode=pond.POND_TRIALS_FOUR_PASS, inv_split=q)
    assert info[0]["mode"] == "four-pass" and info[0]["inv_split"] == q and info[0]["trials_per_launch"] == 1
    for d, r in enumerate(res):
        assert j0 == r.ts_first and np.array_equal(C, r.ts_counts)
        assert rel(T[d], r.ts) <= TOL, (q, d, rel(T[d], r.ts))


def test_autotuned_split_outside_the_three_pass_geometry():
    """A lane without the three-pass geometry (nfft 2^16, 16 sub-channels: M 2^11,
    R2 2^7) runs the four-pass form; with autotune its inverse split is timed
    (default 2^6 and neighbours 5, 7, 4) and the chosen one matches the oracle."""
    dms = [0.0, 0.05, 0.3, 0.15, 0.25]
    nfft, nchan, t_dec = 1 << 16, 16, 8e-6
    x = stream(7 * (1 << 16) + 12345, seed=31)
    info = tuned(dms, nfft, nchan, t_dec, autotune=True, nfft_choices=(nfft,))
    c = info[0]["candidates_us_per_trial"]
    assert [k["mode"] for k in c] == ["four-pass"] * 4
    assert [k["inv_split"] for k in c] == [6, 5, 7, 4]
    best = min(c, key=lambda k: k["us"])
    assert info[0]["mode"] == "four-pass" and info[0]["inv_split"] == best["inv_split"]
    T, C, j0, nf = run_engine(x, dms, nfft, nchan, t_dec, autotune=True, nfft_choices=(nfft,))
    res = oracle_batched(x, dms, nf, nchan, t_dec)
    for d, r in enumerate(res):
        assert j0 == r.ts_first and np.array_equal(C, r.ts_counts)
        assert rel(T[d], r.ts) <= TOL, (d, rel(T[d], r.ts))


def test_batched_series_into_pinned_arrays(grid_case):
    """pond_timeseries of a batched plan into page-locked [ndm, cap] arrays (rows
    copied there directly) returns the default drain's rows bit for bit."""
    import torch
    x, nfft, nchan, t_dec, _ = grid_case
    T, C, j0, _ = run_engine(x, GRID, nfft, nchan, t_dec)
    cap = T.shape[1] + 64
    Tp = torch.zeros((len(GRID), cap), dtype=torch.float32, pin_memory=True).numpy()
    Cp = torch.zeros(cap, dtype=torch.int32, pin_memory=True).numpy()
    with pond.Engine(F0, BW, FS, 0.0, nfft, nchan, 1, 1.0, t_dec=t_dec, dms=GRID) as e:
        e.push(x)
        e.flush()
        n, j = e.timeseries_into(Tp, Cp)
    assert n == T.shape[1] and j == j0
    assert np.array_equal(Tp[:, :n], T) and np.array_equal(Cp[:n], C)
