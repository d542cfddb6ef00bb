"""Split-BF16 tensor-core FFT stages vs the FP64 oracle, through the C ABI.

With precision POND_SPLIT_BF16 (three product terms) or POND_SPLIT_BF16_5T
(five) every radix-16 stage of the four FFT passes is a 16-point DFT-matrix
product on the tensor cores.  The outputs must meet the same bars as the FP32
path: relative L2 <= 1e-5 on dedispersed voltages and <= 1e-4 on folded
profiles and decimated series; fold hits, series counts and indices exact.

The error budget behind the 1e-5 bar: the data split keeps about 16
significant bits (representation error <= 2^-17 relative, about 2.3e-6 RMS
per value), W16 is held to about 24 bits, and the three-term product drops
x_lo w_lo (about 2.5e-6 RMS); with up to 8 tensor-core stages per output the
errors add in quadrature to <= 1.1e-5 (three terms) and <= 7e-6 (five terms).
"""
import numpy as np
import pytest

from oracle import pcd
from paper_1503_01405_gb300 import pond, synth

pytestmark = pytest.mark.gpu

TOL_V = 1e-5
TOL_P = 1e-4
PRECISIONS = [pond.POND_SPLIT_BF16, pond.POND_SPLIT_BF16_5T]
PNAME = {pond.POND_FP32: "fp32", pond.POND_SPLIT_BF16: "bf16x3", pond.POND_SPLIT_BF16_5T: "bf16x5"}


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1503_01405_gb300 import build as pbuild
    pbuild.build()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def run_engine(x, p, precision, want_voltages=True, chunks=None, **kw):
    with pond.Engine(p.f0, p.bw, p.fs, p.dm, p.nfft, p.nchan, p.nbins, p.period, t_dec=p.t_dec_ns * 1e-9,
                     want_voltages=want_voltages, precision=precision, **kw) as e:
        pos = 0
        for c in (chunks or [len(x)]):
            e.push(x[pos:pos + c])
            pos += c
        e.flush()
        s, h, _ = e.profile()
        T, C, j0 = e.timeseries()
        V, g0 = e.voltages() if want_voltages else (None, None)
    return dict(s=s, h=h, T=T, C=C, j0=j0, V=V, g0=g0)


def check(out, r):
    assert np.array_equal(out["h"], r.prof_hits)
    assert np.array_equal(out["C"], r.ts_counts)
    assert out["j0"] == r.ts_first
    ep, et = rel(out["s"], r.prof_sum), rel(out["T"], r.ts)
    assert ep <= TOL_P and et <= TOL_P, (ep, et)
    assert out["g0"] == r.first_g and out["V"].shape == r.voltages.shape
    ev = rel(out["V"], r.voltages)
    assert ev <= TOL_V, ev
    return ev, ep, et


CONFIGS = [
    # nfft, nchan, dm, bw, nbins, period: lines of 4..4096 in every pass, both sidebands
    (1 << 10, 1, 0.002, 16.0, 16, 1.1e-3),
    (1 << 14, 4, 0.05, 16.0, 64, 0.0123),
    (1 << 14, 4, 0.05, -16.0, 64, 0.0123),
    (1 << 16, 16, 0.3, 16.0, 128, 0.033),
    (1 << 18, 1, 0.5, 16.0, 256, 0.0317),
    (1 << 20, 8, 2.0, -16.0, 512, 0.1),
    (1 << 15, 512, 0.0, 16.0, 32, 0.02),
    (1 << 24, 64, 1.0, 16.0, 1024, 0.25),
    # three-pass with the tensor-core column pass (R2 = 2048): 8 sub-channel groups, inverted band
    (1 << 23, 32, 3.0, -16.0, 512, 0.11),
]


def _stream(p, seed, extra):
    spec = synth.StreamSpec(n=4 * p.S + p.nfft // 3 + extra, seed=seed, dm=p.dm, period=p.period,
                            snr=60.0, duty=0.05, bw=p.bw, rfi_duty=0.005)
    return synth.make_stream(spec)


@pytest.mark.parametrize("prec", PRECISIONS, ids=lambda v: PNAME[v])
@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: f"N{c[0]}_c{c[1]}_dm{c[2]}_bw{c[3]}")
def test_precision_matches_oracle(cfg, prec):
    nfft, nchan, dm, bw, nbins, period = cfg
    p = pcd.make_plan(326.5, bw, 32e6, dm, nfft, nchan, nbins, period)
    if nfft >= 1 << 24:
        spec = synth.StreamSpec(n=p.nfft + p.S // 2 + 7, seed=nfft + nchan, dm=dm, period=period, snr=40.0,
                                duty=0.05, rfi_duty=0.005)
        x = synth.make_stream(spec)
    else:
        x = _stream(p, seed=nfft + nchan, extra=17)
    r = pcd.run(p, x, want_voltages=True)
    check(run_engine(x, p, prec), r)


@pytest.mark.parametrize("prec", PRECISIONS, ids=lambda v: PNAME[v])
def test_precision_at_other_inverse_splits(prec):
    """The four-pass tensor-core inverse at splits other than the default (I1's
    columns of Q2 and I2's rows of Q1 as DFT-matrix stages of other lengths)
    against the oracle: nfft 2^16, 16 sub-channels (M 2^11, default split 2^6)."""
    p = pcd.make_plan(326.5, 16.0, 32e6, 0.3, 1 << 16, 16, 128, 0.033)
    x = _stream(p, seed=77, extra=3)
    r = pcd.run(p, x, want_voltages=True)
    for q in (3, 5, 7):
        check(run_engine(x, p, prec, schedule=pond.POND_SCHEDULE_FOUR_PASS, inv_split=q), r)


@pytest.mark.parametrize("prec", PRECISIONS, ids=lambda v: PNAME[v])
def test_precision_small_workload(prec):
    """2^23 samples, DM 3, P 0.253 s, S/N 50; nfft 2^21, 1 channel, 256 bins: the
    error of every output against the oracle, and the pushes split unevenly."""
    x = synth.make_stream(synth.SMALL)
    p = pcd.make_plan(326.5, 16.0, 32e6, 3.0, 1 << 21, 1, 256, 0.253)
    r = pcd.run(p, x, want_voltages=True)
    out = run_engine(x, p, prec, chunks=[1_000_003, 3_000_000, len(x) - 4_000_003])
    ev, ep, et = check(out, r)
    print(f"{PNAME[prec]}: voltages {ev:.3e}, profile {ep:.3e}, series {et:.3e}")


def test_tensor_path_signature():
    """The split-BF16 products leave a deviation far above FP32 rounding, and the
    five-term form is closer to the oracle than the three-term form."""
    p = pcd.make_plan(326.5, 16.0, 32e6, 0.5, 1 << 18, 1, 256, 0.0317)
    x = _stream(p, seed=11, extra=3)
    r = pcd.run(p, x, want_voltages=True)
    v = {prec: run_engine(x, p, prec)["V"] for prec in (pond.POND_FP32, *PRECISIONS)}
    e = {prec: rel(v[prec], r.voltages) for prec in v}
    assert e[pond.POND_FP32] < 1e-6
    assert rel(v[pond.POND_SPLIT_BF16], v[pond.POND_FP32]) > 1e-6
    assert e[pond.POND_SPLIT_BF16_5T] < e[pond.POND_SPLIT_BF16] <= TOL_V


def test_precision_repeatable_bitwise():
    p = pcd.make_plan(326.5, 16.0, 32e6, 1.0, 1 << 17, 64, 256, 0.05)
    x = _stream(p, seed=9, extra=3)
    a = run_engine(x, p, pond.POND_SPLIT_BF16)
    b = run_engine(x, p, pond.POND_SPLIT_BF16)
    for k in ("s", "h", "T", "C", "V"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("prec", PRECISIONS, ids=lambda v: PNAME[v])
def test_precision_batched_trials(prec):
    """A batched plan (one forward transform, per-trial chirps in the inverse
    column pass) on the tensor-core stages vs the oracle's batched form."""
    dms = [0.0, 0.05, 0.3, 0.15]
    nfft, nchan, t_dec = 1 << 16, 16, 8e-6
    x = synth.make_stream(synth.StreamSpec(n=5 * (1 << 16) + 999, seed=41, dm=0.2, period=0.011, snr=80.0,
                                           duty=0.05))
    with pond.Engine(326.5, 16.0, 32e6, 0.0, nfft, nchan, 1, 1.0, t_dec=t_dec, dms=dms, precision=prec) as e:
        e.push(x)
        e.flush()
        T, C, j0 = e.timeseries()
    base = pcd.make_plan(326.5, 16.0, 32e6, 0.0, nfft, nchan, 1, 1.0, t_dec)
    res = pcd.run_batched(base, [(dm, nfft, max(dms)) for dm in dms], x)
    for d, r in enumerate(res):
        assert j0 == r.ts_first and np.array_equal(C, r.ts_counts)
        assert rel(T[d], r.ts) <= TOL_P, (d, rel(T[d], r.ts))


def test_tensor_core_column_pass_three_pass_batched():
    """Batched trials in the three-pass geometry (nfft 2^23, 32 sub-channels,
    R2 = 2048) with three-term split-BF16 stages: the forward passes' radix-16
    stages and the column pass's two DFT-matrix factors run on the tensor
    cores, the row pass with each trial's chirp in FP32; every trial against
    the oracle, for several trials per launch and for per-trial launches."""
    dms = [0.0, 1.0, 2.0, 3.0, 4.0]
    nfft, nchan, t_dec = 1 << 23, 32, 16e-6
    p = pcd.make_plan(326.5, 16.0, 32e6, max(dms), nfft, nchan, 1, 1.0, t_dec)
    x = synth.make_stream(synth.StreamSpec(n=2 * p.S + nfft + 4321, seed=43, dm=2.0, period=0.011, snr=80.0,
                                           duty=0.05))
    base = pcd.make_plan(326.5, 16.0, 32e6, 0.0, nfft, nchan, 1, 1.0, t_dec)
    res = pcd.run_batched(base, [(dm, nfft, max(dms)) for dm in dms], x)
    for mode in (pond.POND_TRIALS_MULTI_TABLE, pond.POND_TRIALS_PER_TRIAL):
        with pond.Engine(326.5, 16.0, 32e6, 0.0, nfft, nchan, 1, 1.0, t_dec=t_dec, dms=dms,
                         precision=pond.POND_SPLIT_BF16, trial_mode=mode, trials_per_launch=3) as e:
            e.push(x)
            e.flush()
            T, C, j0 = e.timeseries()
        for d, r in enumerate(res):
            assert j0 == r.ts_first and np.array_equal(C, r.ts_counts)
            assert rel(T[d], r.ts) <= TOL_P, (mode, d, rel(T[d], r.ts))
