"""The full-rate and batched workloads at their full sizes, in the launch
configurations the benchmark times, against the oracle on sampled outputs and
on properties that hold at any size.

The 60 s stream (1.92e9 int8 samples, 326.5 MHz / 16 MHz, DM 26.8, nfft 2^24,
64 sub-channels, 1024 bins, 61.44 us series) goes through the engine as one
device push on two segment streams.  The oracle (FP64) then recomputes three
sampled stretches of the series (the first segment, one in the middle, the last
emitted samples) from the same input bytes, and the whole fold's hit counts
from its bin rule over every emitted channel sample.  The batched chunk (8 s,
128 DM trials 0..60, FFT lengths chosen by the autotuner) is checked on three
trials over a stretch of one segment.
"""
import numpy as np
import pytest

from oracle import pcd
from paper_1503_01405_gb300 import pond, synth

pytestmark = pytest.mark.gpu
TOL_P = 1e-4
PLAN = dict(f0=326.5, bw=16.0, fs=32e6, dm=26.8, nfft=1 << 24, nchan=64, nbins=1024, period=0.7145)


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1503_01405_gb300 import build as pbuild
    pbuild.build()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


@pytest.fixture(scope="module")
def full_run():
    import torch
    dev = torch.device("cuda", 0)
    x_dev = synth.make_stream_torch(synth.FULL_RATE, dev)
    with pond.Engine(PLAN["f0"], PLAN["bw"], PLAN["fs"], PLAN["dm"], PLAN["nfft"], PLAN["nchan"], PLAN["nbins"],
                     PLAN["period"], t_dec=61.44e-6) as e:
        e.push_tensor(x_dev)
        e.flush()
        s, h, meta = e.profile()
        T, C, j0 = e.timeseries(cap=1 << 21)
        st = e.stats()
    x = x_dev.cpu().numpy()
    del x_dev
    torch.cuda.empty_cache()
    p = pcd.make_plan(**PLAN, t_dec_s=61.44e-6)
    return dict(x=x, p=p, s=s, h=h, meta=meta, T=T, C=C, j0=j0, stats=st)


def test_full_size_geometry(full_run):
    """142 segments, every emitted channel sample folded and decimated once."""
    r, p = full_run, full_run["p"]
    g_first, g_end = pcd.emitted_range(p, len(r["x"]))
    assert r["stats"]["segments"] >= 142
    assert int(r["h"].sum()) == g_end - g_first
    assert int(r["C"].sum()) == g_end - g_first
    assert r["j0"] == (g_first * p.dec.denominator) // p.dec.numerator


@pytest.mark.parametrize("where", ["first", "middle", "last"])
def test_sampled_series_match_oracle(full_run, where):
    """Complete series samples of a stretch of about one segment, against the
    oracle run on the same input over that stretch alone: counts exact, values
    within the FP32 tolerance."""
    r, p = full_run, full_run["p"]
    g_first, g_end = pcd.emitted_range(p, len(r["x"]))
    span = p.S_c
    ga = {"first": g_first, "middle": g_first + 70 * p.S_c + 12345, "last": g_end - span}[where]
    gb = min(ga + span, g_end)
    o = pcd.run(p, r["x"], g_range=(ga, gb))
    num, den = p.dec.numerator, p.dec.denominator
    j_lo = -(-ga * den // num)           # first series sample whose channel samples start at or after ga
    j_hi = (gb * den) // num             # series samples below j_hi end at or before gb
    assert j_hi - j_lo > 5000
    eo = slice(j_lo - o.ts_first, j_hi - o.ts_first)
    ee = slice(j_lo - r["j0"], j_hi - r["j0"])
    assert np.array_equal(o.ts_counts[eo], r["C"][ee])
    assert rel(r["T"][ee], o.ts[eo]) <= TOL_P, (where, rel(r["T"][ee], o.ts[eo]))


def test_fold_hits_and_conservation(full_run):
    """The fold's hit counts equal the oracle's bin rule applied to every
    emitted channel sample (FP64, the same expression); the profile's sum
    equals the series' sum (both add every detected sample once); and the
    folded pulse peaks at the injected phase (0.5)."""
    r, p = full_run, full_run["p"]
    g_first, g_end = pcd.emitted_range(p, len(r["x"]))
    g = np.arange(g_first, g_end, dtype=np.float64)
    xg = g * p.inc
    b = np.minimum(((xg - np.floor(xg)) * p.nbins).astype(np.int64), p.nbins - 1)
    assert np.array_equal(np.bincount(b, minlength=p.nbins), r["h"])
    assert abs(r["s"].sum() - r["T"].astype(np.float64).sum()) <= 1e-5 * r["s"].sum()
    prof = r["s"] / np.maximum(r["h"], 1)
    assert abs(int(np.argmax(prof)) - p.nbins // 2) <= 20


# --- the batched workload at its full size: one 8 s chunk, 128 DM trials 0..60 ---

@pytest.fixture(scope="module")
def batched_run():
    import torch
    dev = torch.device("cuda", 0)
    spec = synth.BATCH_CHUNK
    pulses = synth.draw_pulses(spec.seed, 10, spec.n / spec.fs)
    x_dev = synth.make_chunk_torch(spec, pulses, dev)
    with pond.Engine(PLAN["f0"], PLAN["bw"], PLAN["fs"], 0.0, 1 << 24, 64, 1, 1.0, t_dec=32e-6,
                     dms=synth.BATCH_DMS, nfft_choices=(1 << 22, 1 << 23, 1 << 24), autotune=True) as e:
        e.push_tensor(x_dev)
        e.flush()
        T, C, j0 = e.timeseries(cap=1 << 19)
        dms, nf = e.trials()
    x = x_dev.cpu().numpy()
    del x_dev
    torch.cuda.empty_cache()
    return dict(x=x, T=T, C=C, j0=j0, dms=dms, nf=nf)


@pytest.mark.parametrize("d", [0, 64, 127])
def test_batched_chunk_sampled_trials_match_oracle(batched_run, d):
    """Trial d of the autotuned 128-trial chunk on a stretch of one segment in
    the middle of the chunk: the oracle runs the single-DM path at DM_d on the
    trial's group segmentation (its FFT length, the group's largest DM) over
    the stretch; complete series samples match (counts exact, FP32 tolerance)."""
    r = batched_run
    nf = r["nf"]
    dm = float(r["dms"][d])
    gmax = max(float(r["dms"][i]) for i in range(len(nf)) if nf[i] == nf[d])
    base = pcd.make_plan(PLAN["f0"], PLAN["bw"], PLAN["fs"], 0.0, int(nf[d]), 64, 1, 1.0, 32e-6)
    q = pcd.trial_plan(base, dm, gmax)
    g_lo, g_hi = pcd.batched_range(base, max(float(v) for v in r["dms"]), len(r["x"]))
    ga = (g_lo + g_hi) // 2
    gb = min(ga + q.S_c, g_hi)
    o = pcd.run(q, r["x"], g_range=(ga, gb))
    num, den = q.dec.numerator, q.dec.denominator
    j_lo, j_hi = -(-ga * den // num), (gb * den) // num
    assert j_hi - j_lo > 1000
    eo = slice(j_lo - o.ts_first, j_hi - o.ts_first)
    ee = slice(j_lo - r["j0"], j_hi - r["j0"])
    assert np.array_equal(o.ts_counts[eo], r["C"][ee])
    assert rel(r["T"][d][ee], o.ts[eo]) <= TOL_P, (d, rel(r["T"][d][ee], o.ts[eo]))
