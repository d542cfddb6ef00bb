"""CUDA path vs the FP64 oracle, through the C ABI.

Tolerances: relative L2 error <= 1e-5 on dedispersed voltages and <= 1e-4 on
folded profiles and decimated series (FP32 engine vs FP64 oracle); fold hits,
series counts and every index are exact (the fold bin is decided in FP64 on
both sides with the same correctly rounded operations).
"""
import math

import numpy as np
import pytest

from oracle import pcd
from paper_1503_01405_gb300 import pond, synth

pytestmark = pytest.mark.gpu

TOL_V = 1e-5
TOL_P = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1503_01405_gb300 import build as pbuild
    pbuild.build()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def run_engine(x, p, chunks=None, want_voltages=True, device_push=False, t_dec=61.44e-6,
               schedule=pond.POND_SCHEDULE_AUTO, input_channels=1, chirp=pond.POND_CHIRP_AUTO, pinned=False,
               inv_split=0):
    pm = (p.phase_tref, list(p.phase_coef)) if p.phase_coef else None
    with pond.Engine(p.f0, p.bw, p.fs, p.dm, p.nfft, p.nchan, p.nbins, p.period, t_dec=t_dec,
                     want_voltages=want_voltages, schedule=schedule, input_channels=input_channels,
                     chirp=chirp, inv_split=inv_split, phase_model=pm) as e:
        if pinned:
            # page-locked host memory: the pieces reach the device by the copy kernel
            import torch
            xp = torch.empty(len(x), dtype=torch.int8, pin_memory=True)
            xp.numpy()[:] = x
            xv = xp.numpy()
            pos = 0
            for c in (chunks or [len(x)]):
                e.push(xv[pos:pos + c])
                pos += c
        elif device_push:
            import torch
            t = torch.from_numpy(np.ascontiguousarray(x)).cuda()
            pos = 0
            for c in (chunks or [len(x)]):
                e.push_tensor(t[pos:pos + c])
                pos += c
            torch.cuda.synchronize()
        else:
            pos = 0
            for c in (chunks or [len(x)]):
                e.push(x[pos:pos + c])
                pos += c
        e.flush()
        s, h, meta = e.profile()
        T, C, j0 = e.timeseries()
        V, g0 = e.voltages() if want_voltages else (None, None)
        st = e.stats()
    return dict(s=s, h=h, meta=meta, T=T, C=C, j0=j0, V=V, g0=g0, stats=st)


def check(out, r, voltages=True):
    assert np.array_equal(out["h"], r.prof_hits)
    assert np.array_equal(out["C"], r.ts_counts)
    assert out["j0"] == r.ts_first
    assert rel(out["s"], r.prof_sum) <= TOL_P
    assert rel(out["T"], r.ts) <= TOL_P
    if voltages:
        assert out["g0"] == r.first_g
        assert out["V"].shape == r.voltages.shape
        ev = rel(out["V"], r.voltages)
        assert ev <= TOL_V, ev
        return ev
    return None


CONFIGS = [
    # nfft, nchan, dm, bw, nbins, period
    (1 << 10, 1, 0.002, 16.0, 16, 1.1e-3),
    (1 << 14, 4, 0.05, 16.0, 64, 0.0123),
    (1 << 14, 4, 0.05, -16.0, 64, 0.0123),
    (1 << 16, 16, 0.3, 16.0, 128, 0.033),
    (1 << 17, 64, 1.0, 16.0, 256, 0.05),
    (1 << 18, 1, 0.5, 16.0, 256, 0.0317),
    (1 << 20, 8, 2.0, -16.0, 512, 0.1),
    (1 << 12, 2, 0.0, 16.0, 1, 0.01),
    (1 << 15, 512, 0.0, 16.0, 32, 0.02),
    # fold periods shorter than a warp's 32 channel samples (64 channels: 4 us each)
    (1 << 14, 64, 0.01, 16.0, 16, 8e-5),     # 20 samples, bins of 1.25 samples
    (1 << 14, 64, 0.01, 16.0, 8, 1.6e-4),    # 40 samples
]


def _stream(p, seed, extra):
    spec = synth.StreamSpec(n=4 * p.S + p.nfft // 3 + extra, seed=seed, dm=p.dm, period=p.period,
                            snr=60.0, duty=0.05, bw=p.bw, rfi_duty=0.005)
    return synth.make_stream(spec)


@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: f"N{c[0]}_c{c[1]}_dm{c[2]}_bw{c[3]}")
def test_matches_oracle(cfg):
    nfft, nchan, dm, bw, nbins, period = cfg
    p = pcd.make_plan(326.5, bw, 32e6, dm, nfft, nchan, nbins, period)
    x = _stream(p, seed=nfft + nchan, extra=17)
    out = run_engine(x, p)
    r = pcd.run(p, x, want_voltages=True)
    check(out, r)
    assert out["stats"]["outputs"] == len(r.power)


# Plans with M / R2 = 64 (R1 = 64 nchan of 512..4096) run the three-pass
# schedule: F2 also applies Eq. 4 and a length-64 inverse factor per
# sub-channel, one column pass finishes each sub-channel's inverse and detects.
# Its column pass takes min(8192 / R2, nchan) sub-channels per CTA, so these
# cover one, two, four and sixteen sub-channel groups per output column.
THREE_PASS = [
    (1 << 18, 8, 1.0, 16.0, 128, 0.03),
    (1 << 21, 16, 3.0, -16.0, 256, 0.07),
    (1 << 22, 32, 5.0, 16.0, 512, 0.11),
    (1 << 24, 64, 26.8, 16.0, 1024, 0.7145),
]


@pytest.mark.parametrize("cfg", THREE_PASS, ids=lambda c: f"N{c[0]}_c{c[1]}_dm{c[2]}_bw{c[3]}")
def test_three_pass_schedule(cfg):
    """Both schedules of the same plan against the oracle, and the three-pass
    one runs four kernels per segment where the four-pass one runs five."""
    nfft, nchan, dm, bw, nbins, period = cfg
    p = pcd.make_plan(326.5, bw, 32e6, dm, nfft, nchan, nbins, period)
    if nfft >= 1 << 24:
        x = synth.make_stream(synth.StreamSpec(n=p.nfft + p.S // 2 + 7, seed=5, dm=dm, period=period, snr=40.0,
                                               duty=0.05, bw=bw, rfi_duty=0.005))
    else:
        x = _stream(p, seed=nfft + 3, extra=29)
    r = pcd.run(p, x, want_voltages=True)
    chunks = [len(x) // 3, len(x) - len(x) // 3]
    three = run_engine(x, p, chunks=chunks)
    four = run_engine(x, p, chunks=chunks, schedule=pond.POND_SCHEDULE_FOUR_PASS)
    check(three, r)
    check(four, r)
    # the fused row pass with its chirp read from the per-bin table instead of the anchors
    check(run_engine(x, p, chirp=pond.POND_CHIRP_TABLE), r)
    check(run_engine(x, p, chirp=pond.POND_CHIRP_ANCHORS), r)
    segs = three["stats"]["segments"]
    assert segs == four["stats"]["segments"] and segs >= 2
    # one pass fewer per segment (the pushes' carry copies are the same in both)
    assert four["stats"]["kernel_launches"] - three["stats"]["kernel_launches"] == segs


# Four-pass inverse splits M = Q1 Q2 (log2 Q1 = q) other than the default: I1's
# column tiles of Q2 and I2's rows of Q1 cover the same sub-channel inverses.
SPLITS = [((1 << 16, 16, 0.3, 16.0, 128, 0.033), (2, 3, 4, 5, 7)),       # M 2^11, R2 2^7; default 6
          ((1 << 18, 8, 1.0, -16.0, 128, 0.03), (2, 5, 8)),              # M 2^14, R2 2^8; default 7
          ((1 << 21, 16, 3.0, 16.0, 256, 0.07), (4, 9))]                  # M 2^16, R2 2^10; default 8


@pytest.mark.parametrize("cfg,splits", SPLITS, ids=[f"N{c[0]}_c{c[1]}" for c, _ in SPLITS])
def test_inverse_splits_match_oracle(cfg, splits):
    """The four-pass schedule at every listed split against the oracle (voltages,
    profile, series), with the same launches per segment as the default split."""
    nfft, nchan, dm, bw, nbins, period = cfg
    p = pcd.make_plan(326.5, bw, 32e6, dm, nfft, nchan, nbins, period)
    x = _stream(p, seed=nfft + 11, extra=5)
    r = pcd.run(p, x, want_voltages=True)
    base = run_engine(x, p, schedule=pond.POND_SCHEDULE_FOUR_PASS)
    check(base, r)
    for q in splits:
        out = run_engine(x, p, schedule=pond.POND_SCHEDULE_FOUR_PASS, inv_split=q)
        check(out, r)
        assert out["stats"]["kernel_launches"] == base["stats"]["kernel_launches"], q


@pytest.mark.parametrize("cfg", [(1 << 16, 16, 0.3, 16.0, 128, 0.033), (1 << 18, 8, 1.0, 16.0, 128, 0.03),
                                 (1 << 20, 16, 1.0, 16.0, 128, 0.03)],
                         ids=["four_pass", "three_pass", "three_pass_direct"])
def test_adding_in_phase_matches_oracle(cfg):
    """Interleaved N / S int8 input (input_channels = 2) is added in phase by the
    unpack: the engine matches the oracle on x = N + S, for host and device
    pushes cut into uneven whole pairs and for one whole device push; a push that
    splits a pair is refused."""
    nfft, nchan, dm, bw, nbins, period = cfg
    p = pcd.make_plan(326.5, bw, 32e6, dm, nfft, nchan, nbins, period)
    n, s_ = _stream(p, seed=41, extra=11), _stream(p, seed=42, extra=11)
    inter = np.empty(2 * len(n), np.int8)
    inter[0::2], inter[1::2] = n, s_
    r = pcd.run(p, pcd.adding_in_phase(inter), want_voltages=True)
    cuts = [2 * 12345, 2 * 500_001, len(inter) - 2 * (12345 + 500_001)]
    outs = []
    for chunks, dev in ((cuts, False), (cuts, True), (None, True)):
        out = run_engine(inter, p, chunks=chunks, device_push=dev, input_channels=2)
        check(out, r)
        assert out["stats"]["samples_in"] == len(n)
        outs.append(out)
    # one whole device push keeps every segment's run 4-byte aligned (4-byte loads of
    # N S N S in the first pass where its columns allow); the cuts of 2 * 12345 bytes
    # leave some segments unaligned (element-wise loads): the results agree to the bit
    for key in ("s", "T", "V"):
        assert np.array_equal(outs[2][key], outs[1][key])
    with pond.Engine(p.f0, p.bw, p.fs, p.dm, p.nfft, p.nchan, p.nbins, p.period, input_channels=2) as e:
        with pytest.raises(pond.PondError) as ei:
            e.push(inter[:3])
        assert ei.value.name == "ARG"


@pytest.mark.parametrize("plan", [(1 << 16, 16, 0.3, 128, 0.033), (1 << 21, 16, 3.0, 256, 0.07)],
                         ids=["four_pass", "three_pass"])
def test_streaming_invariance_bit_exact(plan):
    """Outputs do not depend on how the stream is cut into pushes (host or device),
    down to the bit: every reduction has a fixed order and the segment streams
    are ordered by events wherever they share a buffer."""
    nfft, nchan, dm, nbins, period = plan
    p = pcd.make_plan(326.5, 16.0, 32e6, dm, nfft, nchan, nbins, period)
    x = _stream(p, seed=5, extra=999)
    ref = run_engine(x, p)
    rng = np.random.default_rng(1)
    sizes = [0, 1, 7, 1000, 65536, 100_000, 300_001] if nfft < 1 << 20 else [0, 7, 65536, 1_000_003, 3_000_017]
    cuts = []
    left = len(x)
    while left > 0:
        c = int(min(left, rng.choice(sizes)))
        cuts.append(c)
        left -= c
    for dev, pin in ((False, False), (True, False), (False, True)):
        got = run_engine(x, p, chunks=cuts, device_push=dev, pinned=pin)
        for k in ("s", "h", "T", "C"):
            assert np.array_equal(got[k], ref[k]), (k, dev, pin)
        assert np.array_equal(got["V"], ref["V"])
        assert got["j0"] == ref["j0"] and got["g0"] == ref["g0"]


def test_pinned_host_push_matches_oracle():
    """Pushes from page-locked host memory (moved by the copy kernel in pieces of
    32 and 128 MiB, the last one ragged) give the pageable-memory outputs bit
    for bit, and the oracle's within tolerance."""
    p = pcd.make_plan(326.5, 16.0, 32e6, 3.0, 1 << 21, 16, 256, 0.07)
    x = _stream(p, seed=23, extra=12345)
    ref = run_engine(x, p)
    got = run_engine(x, p, pinned=True)
    for k in ("s", "h", "T", "C", "V"):
        assert np.array_equal(got[k], ref[k]), k
    check(got, pcd.run(p, x, want_voltages=True))


# The fold with a polynomial phase model in place of the constant period: a
# spinning-down pulsar (P, Pdot about an epoch inside the stream) and a cubic
# model with a negative reference time, on both schedules.
PHASE_CASES = [
    ((1 << 18, 8, 1.0, 16.0, 128, 0.03), "spin"),
    ((1 << 16, 16, 0.3, -16.0, 64, 0.033), "cubic"),
]


@pytest.mark.parametrize("cfg,kind", PHASE_CASES, ids=[k for _, k in PHASE_CASES])
def test_phase_model_fold_matches_oracle(cfg, kind):
    """Hits exact, sums and the series (unchanged by the model) within the FP32
    tolerance of the oracle; two push splits give the same profile bit for bit."""
    from oracle import stack
    nfft, nchan, dm, bw, nbins, period = cfg
    if kind == "spin":
        model = stack.spin_model(period, 3e-4, 0.0123, 0.25)
    else:
        model = (-0.5, [0.1, 1.0 / period, 2e-3, -7e-4])
    p = pcd.make_plan(326.5, bw, 32e6, dm, nfft, nchan, nbins, period, phase=model)
    x = _stream(p, seed=nfft + 17, extra=9)
    r = pcd.run(p, x)
    scheds = (pond.POND_SCHEDULE_AUTO, pond.POND_SCHEDULE_FOUR_PASS)
    outs = []
    for sched in scheds:
        out = run_engine(x, p, want_voltages=False, schedule=sched)
        check(out, r, voltages=False)
        outs.append(out)
    cut = run_engine(x, p, want_voltages=False, chunks=[len(x) // 3, len(x) - len(x) // 3])
    assert np.array_equal(cut["s"], outs[0]["s"]) and np.array_equal(cut["h"], outs[0]["h"])
    # the model moves samples between bins: the constant-period profile differs
    const = pcd.fold(pcd.make_plan(326.5, bw, 32e6, dm, nfft, nchan, nbins, period), r.power, r.first_g)[1]
    assert not np.array_equal(const, r.prof_hits)


def test_series_into_pinned_arrays():
    """pond_timeseries into page-locked caller arrays (copied there directly)
    returns what the default drain returns, bit for bit, and pageable arrays
    work the same way; a second drain is empty."""
    import torch
    nfft, nchan, dm, bw, nbins, period = CONFIGS[3]
    p = pcd.make_plan(326.5, bw, 32e6, dm, nfft, nchan, nbins, period)
    x = _stream(p, seed=91, extra=3)
    ref = run_engine(x, p, want_voltages=False)
    cap = len(ref["T"]) + 100
    for pinned in (True, False):
        T = torch.zeros(cap, dtype=torch.float32, pin_memory=pinned).numpy()
        C = torch.zeros(cap, dtype=torch.int32, pin_memory=pinned).numpy()
        with pond.Engine(p.f0, p.bw, p.fs, p.dm, p.nfft, p.nchan, p.nbins, p.period) as e:
            e.push(x)
            e.flush()
            n, j0 = e.timeseries_into(T, C)
            assert e.timeseries_into(T[:10].copy(), C[:10].copy())[0] == 0
        assert n == len(ref["T"]) and j0 == ref["j0"]
        assert np.array_equal(T[:n], ref["T"]) and np.array_equal(C[:n], ref["C"])


def test_repeatable_bitwise():
    p = pcd.make_plan(326.5, 16.0, 32e6, 1.0, 1 << 17, 64, 256, 0.05)
    x = _stream(p, seed=9, extra=3)
    a = run_engine(x, p)
    b = run_engine(x, p)
    for k in ("s", "h", "T", "C", "V"):
        assert np.array_equal(a[k], b[k]), k


def test_small_workload_end_to_end():
    """2^23 samples, DM 3, P 0.253 s, S/N 50; nfft 2^21, 1 channel, 256 bins."""
    x = synth.make_stream(synth.SMALL)
    p = pcd.make_plan(326.5, 16.0, 32e6, 3.0, 1 << 21, 1, 256, 0.253)
    out = run_engine(x, p)
    r = pcd.run(p, x, want_voltages=True)
    ev = check(out, r)
    assert out["stats"]["segments"] == 5
    print(f"small workload: voltages rel L2 {ev:.3e}, profile {rel(out['s'], r.prof_sum):.3e}, "
          f"series {rel(out['T'], r.ts):.3e}")


def test_largest_nfft():
    p = pcd.make_plan(326.5, 16.0, 32e6, 1.0, 1 << 25, 1, 128, 0.2)
    x = synth.make_stream(synth.StreamSpec(n=p.nfft + p.S // 2, seed=3, dm=1.0, period=0.2, snr=20.0))
    out = run_engine(x, p)
    r = pcd.run(p, x, want_voltages=True)
    check(out, r)


def test_tone_closed_form_on_gpu():
    """The closed form of a pure tone (see the oracle pins) holds for the engine too."""
    p = pcd.make_plan(326.5, 16.0, 32e6, 0.01, 4096, 4, 16, 1e-3)
    k0 = (3 * p.L) // 7 + 5
    A, theta = 7.5, 0.3
    n = 6 * p.S + p.nfft
    x = np.clip(np.rint(synth.tone(n, k0, p.nfft, A, theta)), -127, 127).astype(np.int8)
    out = run_engine(x, p)
    r = pcd.run(p, x, want_voltages=True)
    check(out, r)


def test_edge_streams():
    p = pcd.make_plan(326.5, 16.0, 32e6, 0.05, 1 << 14, 4, 64, 0.0123)
    # empty stream
    with pond.Engine(p.f0, p.bw, p.fs, p.dm, p.nfft, p.nchan, p.nbins, p.period) as e:
        e.flush()
        s, h, meta = e.profile()
        T, C, j0 = e.timeseries()
        assert h.sum() == 0 and len(T) == 0 and meta["nsamples"] == 0
    # shorter than one segment, exactly one segment, one segment plus a byte
    for n in (p.nfft // 2, p.nfft, p.nfft + 1, 2 * p.n_past * 2 * p.nchan + 3):
        x = _stream(p, seed=n, extra=0)[:n]
        out = run_engine(x, p)
        r = pcd.run(p, x, want_voltages=True)
        if len(r.power) == 0:
            assert out["h"].sum() == 0 and len(out["T"]) == 0
        else:
            check(out, r)


def test_state_errors():
    p = pcd.make_plan(326.5, 16.0, 32e6, 0.05, 1 << 14, 4, 64, 0.0123)
    with pond.Engine(p.f0, p.bw, p.fs, p.dm, p.nfft, p.nchan, p.nbins, p.period) as e:
        e.push(np.zeros(100, np.int8))
        with pytest.raises(pond.PondError) as err:
            e.voltages()
        assert err.value.name == "STATE"
        e.flush()
        with pytest.raises(pond.PondError) as err:
            e.push(np.zeros(10, np.int8))
        assert err.value.name == "STATE"


def test_decimation_options():
    p = pcd.make_plan(326.5, 16.0, 32e6, 0.3, 1 << 16, 16, 128, 0.033, t_dec_s=7.3e-6)
    x = _stream(p, seed=77, extra=5)
    out = run_engine(x, p, t_dec=7.3e-6, want_voltages=False)
    r = pcd.run(p, x)
    check(out, r, voltages=False)
