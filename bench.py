"""Throughput of coherent dedispersion + detection + fold on GB300.

Workload (one "step"): the full-rate stream -- 60 s of 16 MHz band at 32 MS/s
(1.92e9 int8 real samples, seeded synthetic noise + DM 26.8 pulsar (P 0.7145 s,
5 % duty, S/N 20 per period) + 1 % impulsive RFI), dedispersed with nfft 2^24
overlap-save into 64 detected sub-channels, folded into 1024 bins and
decimated to 61.44 us.  Every step pushes the whole stream through the C ABI
and flushes; the stream (1.92 GB) is larger than L2, so no flush is needed.

JSON line fields: value = Msamples/s with the stream resident in HBM
(device push); e2e = the same through pond_push from pinned host memory (H2D
inside the timed region) plus the D2H read of the profile and series;
roofline = the dominant kernel's algorithmic FP32 operations / its CUDA-event
time against the FP32 ceiling (nominal, and measured by the library's FMA
probe), with the method's algorithmic bytes and the pass's own bytes against
measured HBM beside it, and the same for the whole path; cpu_baseline = the
FP64 oracle on the host cores (all of them, one process each, and one
thread); precision / batched = the split-BF16 tensor-core form beside the
FP32 path (speed and error against the oracle) and the 128-trial batched
form on one 8 s chunk.

``--impl reference`` times the FP64 CPU oracle (the only reference there is:
the paper publishes no code) on every host core over a bounded slice per step.
Multi-GPU: replicas only (one independent stream per rank, no collective).
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Msamples/s dedisperse+detect+fold (×real-time) and % HBM roofline vs plain FP32"
UNIT = "Msamples/s"
F0, BW, FS = 326.5, 16.0, 32e6
# kernel behind each stage name of pond_stats
KERNEL_OF_STAGE = {"fwd_cols_unpack": "k_fwd_cols", "fwd_rows_split": "k_fwd_rows",
                   "fwd_rows_chirp_inv": "k_fwd_rows_inv", "inv_rows_chirp": "k_inv_rows_chirp",
                   "inv_cols_chirp": "k_inv_cols",
                   "inv_rows_detect": "k_inv_rows", "inv_cols_detect": "k_inv_cols_det",
                   "fold": "k_fold_dec", "decimate": "k_decimate"}
PLAN = dict(dm=26.8, nfft=1 << 24, nchan=64, nbins=1024, period=0.7145, t_dec=61.44e-6)
REALTIME_MSPS = FS / 1e6


def workload_config(n_samples: int, channels: int = 1) -> dict:
    form = ("1.92e9 int8 samples" if channels == 1 else
            "1.92e9 interleaved N / S int8 pairs (3.84 GB) added in phase")
    return {"workload": f"full-rate 60 s stream: {form}, 326.5 MHz / 16 MHz, DM 26.8, "
                        "nfft 2^24 overlap-save, 64 sub-channels, 1024-bin fold, 61.44 us series",
            "samples_per_step": n_samples, "nfft": PLAN["nfft"], "nchan": PLAN["nchan"],
            "nbins": PLAN["nbins"], "dm": PLAN["dm"], "period_s": PLAN["period"],
            "t_dec_s": PLAN["t_dec"], "l2": "inputs larger than L2 (1.92 GB stream, 64 MB spectra)",
            "parallelism": "replicas"}


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "src": "measured"}
    return {"hbm_gbs": 6800.0, "src": "fallback"}


# FP32 lanes per SM of the Blackwell SM and the GB300's SM count and maximum SM
# clock: the nominal FP32 ceiling 152 x 128 x 2 x 2.07e9 = 80.5 TFLOP/s
FP32_LANES_PER_SM, N_SM, SM_MAX_HZ = 128, 152, 2.07e9
FP32_NOMINAL_TFLOPS = N_SM * FP32_LANES_PER_SM * 2 * SM_MAX_HZ / 1e12


def host_cpu() -> dict:
    """Host core count and CPU model of the machine the oracle runs on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"nproc": cores, "model": model}


def fp32_peak(pond, torch, dev, stream) -> dict:
    """FP32 FMA ceiling of this GPU, measured with the library's probe kernel
    (4 CTAs of 512 threads per SM, 8 independent chains per thread), best of 5
    launches of about 50 ms each, CUDA events on the launching stream."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = 4 * sms
    out = torch.empty(blocks * 512, dtype=torch.float32, device=dev)
    iters = 40000
    pond.probe_fp32_fma(out.data_ptr(), blocks, 100, stream.cuda_stream)     # warm-up
    best = None
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fl = pond.probe_fp32_fma(out.data_ptr(), blocks, iters, stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        t = fl / (e0.elapsed_time(e1) / 1e3) / 1e12
        best = t if best is None else max(best, t)
    assert torch.isfinite(out).all()
    return {"tflops": best, "sms": sms, "kernel": "k_fma_probe (pond_probe_fp32_fma)",
            "nominal_tflops": FP32_NOMINAL_TFLOPS}


def _oracle_worker_init():
    os.environ["OMP_NUM_THREADS"] = "1"
    from oracle import pcd  # noqa: F401  (import once per worker, outside the timed work)


def _oracle_worker(job):
    """Dedisperse whole segments of the shared stream with the FP64 oracle."""
    import numpy as np

    from oracle import pcd
    path, n, segs = job
    x = np.memmap(path, dtype=np.int8, mode="r", shape=(n,))
    p = pcd.make_plan(F0, BW, FS, PLAN["dm"], PLAN["nfft"], PLAN["nchan"], PLAN["nbins"], PLAN["period"],
                      PLAN["t_dec"])
    t0 = time.perf_counter()
    for s in segs:
        pcd.dedisperse_segment(p, np.asarray(x[s * p.S:s * p.S + p.nfft]))
    dt = time.perf_counter() - t0
    del x
    return len(segs), dt


class OraclePool:
    """The FP64 oracle on all host cores: worker processes (started with spawn,
    before any work is timed) each dedisperse whole segments of one stream,
    shared through a read-only file mapping.  Throughput = samples advanced /
    wall time of the round."""

    def __init__(self, x_host, workers: int | None = None):
        import concurrent.futures
        import multiprocessing as mp
        import tempfile

        import numpy as np
        self.cpu = host_cpu()
        self.workers = max(1, min(workers or self.cpu["nproc"], 64))
        self.S = int(x_host_seg_step())
        self.n = len(x_host)
        fd, self.path = tempfile.mkstemp(prefix="pond_oracle_", suffix=".i8")
        os.close(fd)
        self.ex = None
        try:
            np.asarray(x_host, dtype=np.int8).tofile(self.path)
            self.ex = concurrent.futures.ProcessPoolExecutor(self.workers, mp_context=mp.get_context("spawn"),
                                                             initializer=_oracle_worker_init)
            # start every worker (one short job each) before anything is timed
            list(self.ex.map(_oracle_worker, [(self.path, self.n, [])] * self.workers))
        except BaseException:
            self.close()
            raise
        self.max_seg = (self.n - PLAN["nfft"]) // self.S + 1

    def round(self, segs_per_worker: int, first: int = 0):
        """One timed round: worker w takes segments first + w, first + w + W, ...
        (modulo the segments the stream holds); returns (samples advanced, wall
        seconds, segments)."""
        total = self.workers * segs_per_worker
        segs = [(first + i) % self.max_seg for i in range(total)]
        jobs = [(self.path, self.n, segs[w::self.workers]) for w in range(self.workers)]
        t0 = time.perf_counter()
        done = list(self.ex.map(_oracle_worker, jobs))
        wall = time.perf_counter() - t0
        nseg = sum(d[0] for d in done)
        return nseg * self.S, wall, nseg

    def close(self):
        if self.ex is not None:
            self.ex.shutdown()
            self.ex = None
        if self.path and os.path.exists(self.path):
            os.unlink(self.path)
        self.path = None


def x_host_seg_step() -> int:
    """Real samples between segment starts of the full-rate plan (the oracle's geometry)."""
    from oracle import pcd
    return pcd.make_plan(F0, BW, FS, PLAN["dm"], PLAN["nfft"], PLAN["nchan"], PLAN["nbins"], PLAN["period"],
                         PLAN["t_dec"]).S


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, None
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend=backend)
    return rank, ws, dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, v: float) -> float:
    if dist is None:
        return v
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def quiet_gc():
    """Collect once and move every live object out of the collector's scans, so
    that a full collection of the harness's (torch / numpy) heap cannot land
    inside a timed region; collection stays enabled."""
    gc.collect()
    if hasattr(gc, "freeze"):
        gc.freeze()


def pass_sources_hash(root: str | None = None) -> str:
    """Hash of the pass sources (the kernels the traffic counters describe)."""
    import hashlib
    h = hashlib.sha256()
    for f in ("passes.cuh", "fft_block.cuh", "tc_dft.cuh"):
        with open(os.path.join(root or ROOT, "paper_1503_01405_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_from_profiles(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it is current."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    src = pass_sources_hash()
    rows = {}
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if len(parts) >= 3:
                rows[parts[0]] = (parts[1], float(parts[2]))
    if kernel in rows and rows[kernel][0] == src:
        return rows[kernel][1]
    return None


def oracle_rate(x_host, seconds_budget: float = 20.0):
    """FP64 oracle over whole segments of x_host, up to about seconds_budget."""
    from oracle import pcd
    p = pcd.make_plan(F0, BW, FS, PLAN["dm"], PLAN["nfft"], PLAN["nchan"], PLAN["nbins"], PLAN["period"],
                      PLAN["t_dec"])
    t0 = time.perf_counter()
    nseg = 0
    while True:
        a = nseg * p.S
        seg = x_host[a:a + p.nfft]
        if len(seg) < p.nfft:
            break
        pcd.dedisperse_segment(p, seg)
        nseg += 1
        if time.perf_counter() - t0 > seconds_budget * 0.5:
            break
    # fold + decimate of the same span's outputs (a small share of the oracle's time)
    dt_seg = time.perf_counter() - t0
    import numpy as np
    P = np.ones(nseg * p.S_c)
    t1 = time.perf_counter()
    pcd.fold(p, P, p.n_past)
    pcd.decimate(p, P, p.n_past)
    dt = dt_seg + (time.perf_counter() - t1)
    samples = nseg * p.S       # each segment advances the stream by S real samples
    return samples / dt / 1e6, nseg, samples, dt


def run_reference(args, rank, ws, dist):
    """The FP64 oracle on every host core (one process per core, whole segments
    of the full-rate plan); each step is one round of one segment per core."""
    if rank != 0:
        return
    from paper_1503_01405_gb300 import synth
    spec = synth.replace(synth.FULL_RATE, n=3 * (1 << 24))
    x = synth.make_stream(spec)
    pool = OraclePool(x)
    try:
        vals = []
        for i in range(args.warmup + args.steps):
            samples, wall, nseg = pool.round(1, first=i)
            if i >= args.warmup:
                vals.append((samples, wall))
    finally:
        pool.close()
    v = sum(a for a, _ in vals) / sum(d for _, d in vals) / 1e6
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(d for _, d in vals) / len(vals),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": workload_config(int(vals[0][0])),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": pool.workers, "kind": "oracle",
                             "host": pool.cpu,
                             "sample": f"{len(vals)} steps x {pool.workers} whole nfft-2^24 segments (one per "
                                       f"core, {pool.workers} processes) of a {spec.n}-sample slice of the "
                                       "full-rate workload, FP64 numpy"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batched_core(dev, local, stream, steps, warmup, seed_offset=0, samples=0, dist=None, precision=0):
    """Batched DM trials on one 8 s chunk: returns the timing and the plan's choices."""
    import torch

    from paper_1503_01405_gb300 import pond, synth
    spec = synth.replace(synth.BATCH_CHUNK, seed=synth.BATCH_CHUNK.seed + seed_offset)
    if samples:
        spec = synth.replace(spec, n=samples)
    pulses = synth.draw_pulses(spec.seed, 10, spec.n / spec.fs)
    x_dev = synth.make_chunk_torch(spec, pulses, dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    eng = pond.Engine(F0, BW, FS, 0.0, 1 << 24, 64, 1, 1.0, t_dec=32e-6, device=local,
                      dms=synth.BATCH_DMS, nfft_choices=(1 << 22, 1 << 23, 1 << 24), autotune=True,
                      precision=precision)
    plan_s = time.perf_counter() - t0
    _, nf = eng.trials()
    groups = {int(n): int((nf == n).sum()) for n in sorted(set(nf.tolist()))}

    def step():
        eng.reset()
        eng.push_tensor(x_dev, stream)
        eng.flush()

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    quiet_gc()
    barrier(dist)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(dist)
    ms = max_over_ranks(dist, ev0.elapsed_time(ev1))
    st1 = eng.stats()
    T, C, j0 = eng.timeseries()
    tuned = eng.tuning() if hasattr(eng, "tuning") else None
    eng.close()
    del x_dev
    return {"ms": ms, "n": spec.n, "groups": groups, "plan_s": plan_s, "series_shape": list(T.shape),
            "launches_per_step": int(st1["kernel_launches"]), "clocks": clk.summary(), "tuning": tuned}


def run_batched(args, rank, ws, dist):
    """Batched DM trials: an 8 s chunk (2.56e8 samples) with 10 injected single
    pulses, 128 trials DM_d = 60 d / 127, 64 sub-channels, 32 us series, FFT
    length per trial group chosen by the autotuner from {2^22, 2^23, 2^24}."""
    import torch

    from paper_1503_01405_gb300 import build as pbuild
    from paper_1503_01405_gb300 import synth

    local = int(os.environ.get("LOCAL_RANK", rank))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pbuild.build()
    stream = torch.cuda.current_stream(dev)
    prec = {"fp32": 0, "bf16x3": 1, "bf16x5": 2}[args.precision]
    r = batched_core(dev, local, stream, args.steps, args.warmup, seed_offset=rank, samples=args.samples, dist=dist,
                     precision=prec)
    value = ws * r["n"] * args.steps / (r["ms"] / 1e3) / 1e6
    if rank == 0:
        line = {"metric": METRIC + " [batched DM trials]", "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp32": "f32", "bf16x3": "bf16x3+f32acc", "bf16x5": "bf16x5+f32acc"}[args.precision],
                "data": "synthetic", "realtime_factor": value / REALTIME_MSPS,
                "trial_samples_per_s": value * 1e6 * len(synth.BATCH_DMS),
                "config": {"workload": BATCHED_WORKLOAD, "samples_per_step": r["n"],
                           "trials": len(synth.BATCH_DMS), "nfft_groups": r["groups"],
                           "plan_s_incl_autotune": r["plan_s"], "series_shape": r["series_shape"],
                           "tuning": r["tuning"], "l2": "inputs larger than L2"},
                "gpu_launches": r["launches_per_step"] * args.steps,
                "clocks": r["clocks"]}
        print(json.dumps(line), flush=True)


BATCHED_WORKLOAD = ("batched: 8 s chunk (2.56e8 int8 samples, 10 injected pulses), 128 DM trials 0..60, "
                    "64 sub-channels, 32 us series, autotuned nfft")


PREC_PLAN = dict(dm=3.0, nfft=1 << 21, nchan=1, nbins=256, period=0.253, t_dec=61.44e-6)


def precision_brief(dev, local, stream, steps=3, warmup=2):
    """The precision form beside the FP32 path, for the headline line: the
    2^23-sample stream (nfft 2^21, one channel; L2 flushed before each timed
    step) and the full-rate geometry on a 2^28-sample slice, in FP32 and with
    split-BF16 tensor-core radix-16 stages (three and five terms), plus the
    error of every output of each form against the FP64 oracle."""
    import numpy as np
    import torch

    from oracle import pcd
    from paper_1503_01405_gb300 import pond, synth
    P = PREC_PLAN
    xh = synth.make_stream(synth.SMALL)
    n = len(xh)
    x_dev = torch.from_numpy(xh).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    precs = {"fp32": pond.POND_FP32, "bf16x3": pond.POND_SPLIT_BF16, "bf16x5": pond.POND_SPLIT_BF16_5T}

    def engine(prec, plan, want_voltages=False):
        return pond.Engine(F0, BW, FS, plan["dm"], plan["nfft"], plan["nchan"], plan["nbins"], plan["period"],
                           t_dec=plan["t_dec"], want_voltages=want_voltages, device=local, precision=prec)

    def timed(eng, x, k, w, flush_l2):
        def step():
            eng.reset()
            eng.push_tensor(x, stream)
            eng.flush()
        for _ in range(w):
            step()
        torch.cuda.synchronize()
        total = 0.0
        for _ in range(k):
            if flush_l2:
                flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
        return total

    small, full = {}, {}
    for name, prec in precs.items():
        with engine(prec, P) as e:
            small[name] = n * steps / (timed(e, x_dev, steps, warmup, True) / 1e3) / 1e6
    fspec = synth.replace(synth.FULL_RATE, n=1 << 28)
    xf = synth.make_stream_torch(fspec, dev)
    for name, prec in precs.items():
        with engine(prec, PLAN) as e:
            full[name] = fspec.n * 2 / (timed(e, xf, 2, 1, False) / 1e3) / 1e6
    del xf, flush
    p = pcd.make_plan(F0, BW, FS, P["dm"], P["nfft"], P["nchan"], P["nbins"], P["period"], P["t_dec"])
    r = pcd.run(p, xh, want_voltages=True)

    def rel(a, b):
        return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))

    err = {}
    for name, prec in precs.items():
        with engine(prec, P, want_voltages=True) as e:
            e.push(xh)
            e.flush()
            s_, h_, _ = e.profile()
            T_, C_, _ = e.timeseries()
            V_, _ = e.voltages()
        err[name] = {"voltage": rel(V_, r.voltages), "profile": rel(s_, r.prof_sum), "series": rel(T_, r.ts),
                     "hits_exact": bool(np.array_equal(h_, r.prof_hits)),
                     "counts_exact": bool(np.array_equal(C_, r.ts_counts))}
    return {"workload": "2^23 int8 samples, DM 3, P 0.253 s, nfft 2^21, 1 channel, 256-bin fold (L2 flushed "
                        "before each step); full-rate geometry: 2^28 samples, nfft 2^24, 64 channels",
            "msps": small, "speedup_vs_fp32": {k: small[k] / small["fp32"] for k in ("bf16x3", "bf16x5")},
            "full_rate_geometry_msps": full,
            "full_rate_speedup_vs_fp32": {k: full[k] / full["fp32"] for k in ("bf16x3", "bf16x5")},
            "error_vs_oracle": err, "tolerance": {"voltage": 1e-5, "profile": 1e-4, "series": 1e-4}}


INCOH_PLAN = {"nchan": 1024, "nint": 1, "dm": 26.8, "nbins": 1024, "period": 0.7145}


def run_incoherent(args, rank, ws, dist):
    """Incoherent modes (Sec. 3.4) on the full-rate band: the two halves' 60 s
    streams (1.92e9 samples each, the second an independent stream of the same
    recipe) interleaved N / S (3.84 GB), through a 1024-channel FFT filterbank
    (64 us spectra, nint 1), detected as AID (added in phase) or CID (cross-power),
    shifted by the Eq. 3 delays at DM 26.8, summed and folded into 1024 bins.
    The input and the 3.84 GB filterbank are larger than L2."""
    import numpy as np
    import torch

    from oracle import incoherent as inc
    from paper_1503_01405_gb300 import build as pbuild
    from paper_1503_01405_gb300 import pond, synth

    local = int(os.environ.get("LOCAL_RANK", rank))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pbuild.build()
    P = INCOH_PLAN
    cid = args.incoh_mode == "cid"
    spec = synth.replace(synth.FULL_RATE, seed=synth.FULL_RATE.seed + rank)
    if args.samples:
        spec = synth.replace(spec, n=args.samples)
    n = spec.n
    a = synth.make_stream_torch(spec, dev)
    b = synth.make_stream_torch(synth.replace(spec, seed=spec.seed + 1000), dev)
    x_dev = torch.stack([a, b], dim=1).reshape(-1)
    del a, b
    torch.cuda.synchronize()
    eng = pond.Incoherent(F0, BW, FS, P["dm"], P["nchan"], P["nint"], P["nbins"], P["period"],
                          mode=pond.POND_INCOH_CID if cid else pond.POND_INCOH_AID, input_channels=2, device=local)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        eng.run_tensor(x_dev, stream)
    torch.cuda.synchronize()
    quiet_gc()
    barrier(dist)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            eng.run_tensor(x_dev, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(dist)
    ms = max_over_ranks(dist, ev0.elapsed_time(ev1))
    value = ws * n * args.steps / (ms / 1e3) / 1e6
    info = eng.info()   # the last timed run: CUDA events around each stage on its stream
    peaks = measured_peaks()
    stages = {"filterbank": (info["ms_filterbank"], info["algo_bytes_filterbank"], "k_fb_power"),
              "dedisperse": (info["ms_dedisperse"], info["algo_bytes_dedisperse"], "k_incoh_sum")}
    dom = max(stages, key=lambda k: stages[k][0])
    t_ms, nbytes, kname = stages[dom]
    achieved = nbytes / (t_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": None, "kernel": kname, "peak_src": peaks["src"],
            "stage_ms_per_step": {"filterbank": info["ms_filterbank"], "dedisperse": info["ms_dedisperse"],
                                  "fold": info["ms_fold"]},
            "stage_gbs": {k: v[1] / (v[0] / 1e3) / 1e9 for k, v in stages.items() if v[0] > 0}}

    # end to end: host int8 pairs in pinned memory through the binding's host call,
    # series and profile read back
    x_host = torch.empty(2 * n, dtype=torch.int8, pin_memory=True)
    x_host.copy_(x_dev)
    xh = x_host.numpy()
    del x_dev
    torch.cuda.synchronize()
    out = {}

    def step_host():
        eng.run(x_host)
        D, _ = eng.series()
        s_, h_ = eng.profile()
        out["bytes"] = D.nbytes + s_.nbytes + h_.nbytes

    for _ in range(max(1, args.warmup)):
        step_host()
    quiet_gc()
    barrier(dist)
    e2e_steps = max(args.steps, 10)
    t0 = time.perf_counter()
    marks = [t0]
    for _ in range(e2e_steps):
        step_host()
        marks.append(time.perf_counter())
    e2e_s = max_over_ranks(dist, marks[-1] - t0)
    step_ms = sorted(1e3 * (b_ - a_) for a_, b_ in zip(marks, marks[1:]))
    e2e = {"value": ws * n * e2e_steps / e2e_s / 1e6, "unit": UNIT, "steps": e2e_steps,
           "h2d_bytes_per_step": 2 * n, "d2h_bytes_per_step": out["bytes"],
           "step_ms_min_median_max": [step_ms[0], statistics.median(step_ms), step_ms[-1]]}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        p = inc.make_plan(F0, BW, FS, P["dm"], P["nchan"], P["nint"], inc.CID if cid else inc.AID, 2,
                          P["nbins"], P["period"])
        m = 1 << 22
        while True:
            t0 = time.perf_counter()
            inc.run(p, xh[:2 * m])
            dt = time.perf_counter() - t0
            if dt > 5.0 or 2 * m > len(xh) // 2:
                break
            m *= 2
        cpu = {"value": m / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"the first {m} pairs of the same input, {dt:.1f} s of FP64 numpy on 1 host thread"}
    clocks = clk.summary()
    if rank == 0:
        line = {"metric": "Msamples/s incoherent " + ("CID" if cid else "AID") +
                          " (1024-channel filterbank, Eq. 3 shifts, fold)",
                "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": "incoherent " + ("CID" if cid else "AID") + " on the full-rate band: "
                                       "1.92e9 interleaved N / S int8 pairs (3.84 GB), 1024 channels, 64 us "
                                       "spectra, DM 26.8, 1024-bin fold",
                           "samples_per_step": n, "nchan": P["nchan"], "nint": P["nint"], "dm": P["dm"],
                           "nbins": P["nbins"], "period_s": P["period"],
                           "l2": "inputs larger than L2 (3.84 GB input, 3.84 GB filterbank)",
                           "parallelism": "replicas"},
                "realtime_factor": value / REALTIME_MSPS, "e2e": e2e,
                "gpu_launches": int(info["launches"]) * args.steps, "roofline": roof, "cpu_baseline": cpu,
                "clocks": clocks}
        print(json.dumps(line), flush=True)
    eng.close()
    if dist is not None:
        dist.destroy_process_group()


def run_precision(args, rank, ws, dist):
    """Precision form: the 2^23-sample stream (DM 3, P 0.253 s, S/N 50 per fold;
    nfft 2^21, one channel, 256-bin fold) with every radix-16 FFT stage computed
    as split-BF16 16-point DFT-matrix products on the tensor cores (three product
    terms, FP32 accumulation).  The five-term form and the FP32 path run the same
    stream in the same process: value is the three-term throughput, the line
    carries the FP32 and five-term throughputs, the measured error of every
    output against the FP64 oracle, and the same comparison at the full-rate
    geometry (nfft 2^24, 64 channels) on a 2^28-sample slice of the full-rate
    stream.  The 8 MB stream fits in L2, so L2 is flushed (a 256 MB write)
    before every timed step and each step is timed alone with CUDA events."""
    import numpy as np
    import torch

    from oracle import pcd
    from paper_1503_01405_gb300 import build as pbuild
    from paper_1503_01405_gb300 import pond, synth

    local = int(os.environ.get("LOCAL_RANK", rank))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pbuild.build()
    P = PREC_PLAN
    spec = synth.replace(synth.SMALL, seed=synth.SMALL.seed + rank)
    xh = synth.make_stream(spec)
    n = len(xh)
    x_dev = torch.from_numpy(xh).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    precs = {"bf16x3": pond.POND_SPLIT_BF16, "bf16x5": pond.POND_SPLIT_BF16_5T, "fp32": pond.POND_FP32}

    def engine(prec, timing=False, want_voltages=False, plan=P):
        return pond.Engine(F0, BW, FS, plan["dm"], plan["nfft"], plan["nchan"], plan["nbins"], plan["period"],
                           t_dec=plan["t_dec"], timing=timing, want_voltages=want_voltages, device=local,
                           precision=prec)

    def timed(eng, x, steps, warmup, flush_l2):
        def step():
            eng.reset()
            eng.push_tensor(x, stream)
            eng.flush()
        for _ in range(warmup):
            step()
        st0 = eng.stats()
        torch.cuda.synchronize()
        quiet_gc()
        barrier(dist)
        total = 0.0
        for _ in range(steps):
            if flush_l2:
                flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
        barrier(dist)
        return max_over_ranks(dist, total), st0, eng.stats()

    res = {}
    with Clocks(local) as clk:
        for name, prec in precs.items():
            eng = engine(prec)
            ms, st0, st1 = timed(eng, x_dev, args.steps, args.warmup, True)
            res[name] = {"ms": ms, "st1": st1, "value": ws * n * args.steps / (ms / 1e3) / 1e6}
            eng.close()
    main = res["bf16x3"]
    # per-stage times from an engine with stage timing (segments serialized)
    eng = engine(pond.POND_SPLIT_BF16, timing=True)
    _, tst0, tst1 = timed(eng, x_dev, max(1, min(args.steps, 2)), 1, True)
    eng.close()
    stages = stage_deltas(tst0, tst1)
    roof = roofline(stages, max(1, min(args.steps, 2)), main["ms"] / args.steps, n, 1, main["st1"],
                    fp32_peak(pond, torch, dev, stream), measured_peaks())
    roof["kernel"] += " (tensor-core form)"
    roof["traffic"] = None

    # full-rate geometry on a 2^28-sample slice (larger than L2)
    full = {}
    fspec = synth.replace(synth.FULL_RATE, n=1 << 28, seed=synth.FULL_RATE.seed + rank)
    xf = synth.make_stream_torch(fspec, dev)
    for name, prec in precs.items():
        eng = engine(prec, plan=PLAN)
        ms, _, _ = timed(eng, xf, max(2, args.steps // 2), 1, False)
        full[name] = ws * fspec.n * max(2, args.steps // 2) / (ms / 1e3) / 1e6
        eng.close()
    del xf

    # end to end: pond_push from pinned host memory, results read back
    x_pin = torch.empty(n, dtype=torch.int8, pin_memory=True)
    x_pin.copy_(x_dev)
    xp = x_pin.numpy()
    eng_h = engine(pond.POND_SPLIT_BF16)
    nbytes = {}

    def step_host():
        eng_h.reset()
        eng_h.push(xp)
        eng_h.flush()
        s_, h_, _ = eng_h.profile()
        T_, C_, _ = eng_h.timeseries()
        nbytes["d2h"] = s_.nbytes + h_.nbytes + T_.nbytes + C_.nbytes

    for _ in range(max(1, args.warmup)):
        step_host()
    quiet_gc()
    barrier(dist)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_host()
    e2e_s = max_over_ranks(dist, time.perf_counter() - t0)
    launches = int(eng_h.stats()["kernel_launches"]) * args.steps
    eng_h.close()
    e2e = {"value": ws * n * args.steps / e2e_s / 1e6, "unit": UNIT, "h2d_bytes_per_step": n,
           "d2h_bytes_per_step": nbytes["d2h"]}

    line = None
    if rank == 0:
        # error of every output against the FP64 oracle (rank 0's stream)
        p = pcd.make_plan(F0, BW, FS, P["dm"], P["nfft"], P["nchan"], P["nbins"], P["period"], P["t_dec"])
        t1 = time.perf_counter()
        r = pcd.run(p, xh, want_voltages=True)
        oracle_s = time.perf_counter() - t1

        def rel(a, b):
            return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))

        err = {}
        for name, prec in precs.items():
            with engine(prec, want_voltages=True) as e:
                e.push(xh)
                e.flush()
                s_, h_, _ = e.profile()
                T_, C_, _ = e.timeseries()
                V_, _ = e.voltages()
            err[name] = {"voltage": rel(V_, r.voltages), "profile": rel(s_, r.prof_sum), "series": rel(T_, r.ts),
                         "hits_exact": bool(np.array_equal(h_, r.prof_hits)),
                         "counts_exact": bool(np.array_equal(C_, r.ts_counts))}
        cpu = None
        if not args.no_cpu_baseline:
            cpu = {"value": n / oracle_s / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"the whole {n}-sample stream (5 segments of 2^21), FP64 numpy on 1 host thread, "
                             f"{oracle_s:.1f} s, voltages kept"}
        line = {"metric": METRIC + " [precision form]", "value": main["value"], "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": main["ms"] / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3+f32acc",
                "data": "synthetic", "realtime_factor": main["value"] / REALTIME_MSPS,
                "config": {"workload": "precision form: 2^23 int8 samples, DM 3, P 0.253 s, nfft 2^21, 1 channel, "
                                       "256-bin fold; radix-16 stages as split-BF16 DFT-matrix products on tcgen05",
                           "samples_per_step": n, "l2": "flushed (256 MB write) before every timed step"},
                "fp32_value": res["fp32"]["value"], "bf16x5_value": res["bf16x5"]["value"],
                "speedup_vs_fp32": {"bf16x3": main["value"] / res["fp32"]["value"],
                                    "bf16x5": res["bf16x5"]["value"] / res["fp32"]["value"]},
                "full_rate_geometry_msps": full,
                "full_rate_speedup_vs_fp32": {k: full[k] / full["fp32"] for k in ("bf16x3", "bf16x5")},
                "error_vs_oracle": err, "e2e": e2e, "gpu_launches": launches, "roofline": roof,
                "cpu_baseline": cpu, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)


LEARNED_WORKLOAD = ("learned: DM-time patches (32 trials x 256 samples of 32 us) from the batched engine on "
                    "labelled 8 s chunks; pulse / DM-0 burst / narrowband / noise")


def learned_core(chunks: int, shifts: int, epochs: int) -> dict:
    """Classifier on DM-time patches: training chunks and disjoint held-out
    chunks (different seeds) through the batched engine; recall and false
    positive rate of the classifier and of the boxcar detector, the boxcar with
    the network's veto; inference rate."""
    import torch

    from paper_1503_01405_gb300 import learn, pond

    t0 = time.perf_counter()
    Xtr, Ytr, Ftr = learn.build_dataset(chunks, seed=1000, shifts=shifts)
    Xte, Yte, Fte = learn.build_dataset(max(2, chunks // 5), seed=2000, shifts=shifts)
    Xva, Yva, Fva = learn.build_dataset(max(2, chunks // 8), seed=3000, shifts=shifts)
    gen_s = time.perf_counter() - t0
    theta = learn.init_params(99)
    clf = pond.Classifier(theta, max_batch=512)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    hist = learn.train(clf, Xtr, Ytr, epochs=epochs, batch=256, lr=2e-3, seed=3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    pte = learn.predict(clf, Xte)
    res = learn.evaluate(pte, Yte, Fte)
    # the boxcar with the network's veto, at the operating point that keeps the
    # boxcar's recall on the validation chunks
    tau = learn.veto_threshold(learn.predict(clf, Xva), Yva, Fva, 0.0)
    veto = learn.evaluate_veto(pte, Yte, Fte, tau)
    rate = learn.inference_rate(clf, Xte)
    # the same trained network with room for large batches: inference throughput at 8192 patches per call
    clf_big = pond.Classifier(clf.params(), max_batch=8192)
    rate_big = learn.inference_rate(clf_big, Xte, batch=8192, reps=10)
    clf_big.close()
    clf.close()
    return {"value": rate, "unit": "candidates/s",
            "config": {"workload": LEARNED_WORKLOAD, "train_patches": int(len(Ytr)), "test_patches": int(len(Yte)),
                       "epochs": epochs, "shifts_per_event": shifts, "train_chunks": chunks, "batch": 256,
                       "lr": 2e-3},
            "inference_batch": 512, "value_batch_8192": rate_big,
            "inference_kernel": "k_cnn_infer_tc (tcgen05 implicit-GEMM convolutions, BF16, FP32 accumulators)",
            "evaluation": res, "boxcar_with_network_veto": veto, "validation_patches": int(len(Yva)),
            "train_loss_first_last": [hist[0], hist[-1]], "train_s": train_s, "dataset_s": gen_s}


def run_learned(args, rank):
    if rank != 0:
        return
    from paper_1503_01405_gb300 import build as pbuild

    pbuild.build()
    r = learned_core(args.chunks, args.shifts, args.epochs)
    line = {"metric": "single-pulse candidates classified per second (CNN inference)", "value": r.pop("value"),
            "unit": r.pop("unit"), "n_gpus": 1, "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
            "config": r.pop("config")}
    line.update(r)
    print(json.dumps(line), flush=True)


def stage_deltas(st0: dict, st1: dict) -> dict:
    """Per-stage time, launches, pass bytes and algorithmic flops between two pond_stats."""
    out = {}
    for name, d in st1["stages"].items():
        d0 = st0["stages"].get(name, {"ms": 0.0, "launches": 0})
        dl = d["launches"] - d0["launches"]
        if dl > 0:
            out[name] = {"ms": d["ms"] - d0["ms"], "launches": dl, "pass_bytes": d["pass_bytes"],
                         "algo_flops": d["algo_flops"]}
    return out


def algo_bytes_per_segment(st: dict, ch: int) -> float:
    """The method's algorithmic DRAM bytes per segment: the int8 input of one
    overlap-save segment read once (nfft bytes per channel of input, i.e. the
    1 B/sample input re-read over the overlap) plus the outputs (detected,
    folded and decimated power: 4 B per emitted channel sample, an upper bound)."""
    return float(st["nfft"]) * ch + 4.0 * (st["seg_step"] // (2 * st["nchan"]))


def roofline(stages: dict, t_steps: int, ms_step: float, n: int, ch: int, st: dict, fp32: dict,
             peaks: dict) -> dict:
    """Roofline of the dominant kernel (largest serialized time per step).

    The path's algorithmic arithmetic intensity is about 110 flop per DRAM byte,
    far above the GPU's balance (about 80 TFLOP/s / 6.8 TB/s = 12), so at its
    algorithmic minimum it is bound by the FP32 pipes: `achieved` is the
    kernel's algorithmic FP32 operations per launch over its mean CUDA-event
    duration, `peak` the nominal FP32 ceiling (152 SMs x 128 lanes x 2 x
    2.07 GHz) with the probe's measured ceiling beside it.  `algo_hbm_frac` is
    the same launch's share of the method's algorithmic bytes (one segment's
    input, one launch per segment) over its duration against measured HBM,
    `pass_bytes_frac` the bytes the pass itself must move (its input and output
    once) against measured HBM."""
    dom = max(stages, key=lambda k: stages[k]["ms"])
    d = stages[dom]
    avg_s = d["ms"] / d["launches"] / 1e3
    kname = KERNEL_OF_STAGE[dom]
    achieved = d["algo_flops"] / avg_s / 1e12
    seg_bytes = algo_bytes_per_segment(st, ch)
    segs_per_step = n / st["seg_step"]
    path_flops = sum(v["algo_flops"] * v["launches"] for v in stages.values()) / t_steps
    path_tflops = path_flops / (ms_step / 1e3) / 1e12
    path_gbs = seg_bytes * segs_per_step / (ms_step / 1e3) / 1e9
    return {"bound": "alu", "achieved": achieved, "peak": FP32_NOMINAL_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP32_NOMINAL_TFLOPS,
            "peak_src": "nominal FP32 (152 SMs x 128 lanes x 2 flop x 2.07 GHz)",
            "peak_measured": fp32["tflops"], "frac_of_measured": achieved / fp32["tflops"],
            # the committed counters are of the single-channel launches
            "traffic": traffic_from_profiles(kname) if ch == 1 else None,
            "kernel": kname, "algo_flops_per_launch": d["algo_flops"], "launch_us": avg_s * 1e6,
            "algo_hbm_gbs": seg_bytes / avg_s / 1e9, "algo_hbm_frac": seg_bytes / avg_s / 1e9 / peaks["hbm_gbs"],
            "pass_bytes_gbs": d["pass_bytes"] / avg_s / 1e9,
            "pass_bytes_frac": d["pass_bytes"] / avg_s / 1e9 / peaks["hbm_gbs"],
            "hbm_peak_gbs": peaks["hbm_gbs"], "hbm_peak_src": peaks["src"],
            "stage_ms_per_step_serialized": {k: v["ms"] / t_steps for k, v in stages.items()},
            "path": {"algo_flops_per_sample": path_flops / n, "tflops": path_tflops,
                     "alu_frac": path_tflops / FP32_NOMINAL_TFLOPS,
                     "alu_frac_of_measured": path_tflops / fp32["tflops"],
                     "algo_bytes_per_sample": seg_bytes / st["seg_step"], "algo_hbm_gbs": path_gbs,
                     "algo_hbm_frac": path_gbs / peaks["hbm_gbs"],
                     "pass_bytes_gbs": sum(v["pass_bytes"] * v["launches"] for v in stages.values()) / t_steps /
                                       (ms_step / 1e3) / 1e9},
            "fp32_probe": fp32}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--samples", type=int, default=0, help="override stream length (testing)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cufft-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="full-rate: skip the precision-form and batched-trials sub-measurements")
    ap.add_argument("--workload", default="full-rate", choices=["full-rate", "batched", "learned", "precision", "aip", "incoherent"],
                    help="full-rate: the headline stream; batched: 128 DM trials on 8 s chunks; "
                         "learned: classifier training and evaluation beside the boxcar detector; "
                         "precision: split-BF16 tensor-core FFT stages vs the FP32 path and the oracle")
    ap.add_argument("--chunks", type=int, default=40, help="learned: 8 s training chunks")
    ap.add_argument("--shifts", type=int, default=16, help="learned: time-shifted patches per event")
    ap.add_argument("--epochs", type=int, default=20, help="learned: training epochs")
    ap.add_argument("--incoh-mode", default="aid", choices=["aid", "cid"],
                    help="incoherent: adding in phase (AID) or correlation (CID)")
    ap.add_argument("--chirp", default="auto", choices=["auto", "anchors", "table"],
                    help="full-rate: chirp source of the fused forward row pass (POND_CHIRP_*)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16x3", "bf16x5"],
                    help="full-rate: arithmetic of the radix-16 FFT stages (FP32, or split-BF16 tensor-core "
                         "DFT products with three or five terms)")
    args = ap.parse_args()
    rank, ws, dist = dist_init()
    if args.impl == "reference":
        run_reference(args, rank, ws, dist)
        return
    if args.workload == "batched":
        run_batched(args, rank, ws, dist)
        return
    if args.workload == "learned":
        run_learned(args, rank)
        return
    if args.workload == "precision":
        run_precision(args, rank, ws, dist)
        return
    if args.workload == "incoherent":
        run_incoherent(args, rank, ws, dist)
        return
    import numpy as np
    import torch

    from paper_1503_01405_gb300 import build as pbuild
    from paper_1503_01405_gb300 import pond, synth

    local = int(os.environ.get("LOCAL_RANK", rank))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pbuild.build()
    spec = synth.replace(synth.FULL_RATE, seed=synth.FULL_RATE.seed + rank)
    if args.samples:
        spec = synth.replace(spec, n=args.samples)
    n = spec.n
    # "aip": the same plan fed the two halves' samples interleaved (N0 S0 N1 S1 ...),
    # added in phase by the engine's unpack; the halves are independent seeded streams
    # of the full-rate recipe
    ch = 2 if args.workload == "aip" else 1
    x_dev = synth.make_stream_torch(spec, dev)
    if ch == 2:
        s_half = synth.make_stream_torch(synth.replace(spec, seed=spec.seed + 1000), dev)
        x_dev = torch.stack([x_dev, s_half], dim=1).reshape(-1)
        del s_half
    torch.cuda.synchronize()
    prec = {"fp32": pond.POND_FP32, "bf16x3": pond.POND_SPLIT_BF16, "bf16x5": pond.POND_SPLIT_BF16_5T}[args.precision]
    # the timed engine runs consecutive segments on two streams (they overlap);
    # a second engine with per-stage timing runs them one after another, so its
    # CUDA events give each kernel's own duration for the roofline
    chirp = {"auto": pond.POND_CHIRP_AUTO, "anchors": pond.POND_CHIRP_ANCHORS, "table": pond.POND_CHIRP_TABLE}[args.chirp]
    eng = pond.Engine(F0, BW, FS, PLAN["dm"], PLAN["nfft"], PLAN["nchan"], PLAN["nbins"], PLAN["period"],
                      t_dec=PLAN["t_dec"], device=local, precision=prec, input_channels=ch, chirp=chirp)
    stream = torch.cuda.current_stream(dev)

    def step_device(e):
        e.reset()
        e.push_tensor(x_dev, stream)
        e.flush()

    for _ in range(args.warmup):
        step_device(eng)
    torch.cuda.synchronize()
    quiet_gc()
    barrier(dist)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step_device(eng)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(dist)
    ms = ev0.elapsed_time(ev1)
    ms = max_over_ranks(dist, ms)
    st1 = eng.stats()
    value = ws * n * args.steps / (ms / 1e3) / 1e6

    # dominant kernel from per-stage CUDA-event times of serialized steps
    eng_t = pond.Engine(F0, BW, FS, PLAN["dm"], PLAN["nfft"], PLAN["nchan"], PLAN["nbins"], PLAN["period"],
                        t_dec=PLAN["t_dec"], timing=True, device=local, precision=prec,
                        input_channels=ch, chirp=chirp)
    step_device(eng_t)
    tst0 = eng_t.stats()
    t_steps = max(1, min(args.steps, 2))
    for _ in range(t_steps):
        step_device(eng_t)
    tst1 = eng_t.stats()
    eng_t.close()
    stages = stage_deltas(tst0, tst1)
    fp32 = fp32_peak(pond, torch, dev, stream)
    roof = roofline(stages, t_steps, ms / args.steps, n, ch, st1, fp32, measured_peaks())

    # the cuFFT comparison path on the same device-resident stream (one warm-up, one timed step)
    cufft = None
    if rank == 0 and not args.no_cufft_baseline and ch == 1:
        from baseline.cufft_path import CufftPath
        cp = CufftPath(F0, BW, FS, PLAN["dm"], PLAN["nfft"], PLAN["nchan"], PLAN["nbins"], PLAN["period"],
                       PLAN["t_dec"], dev)
        cp.run(x_dev)
        torch.cuda.synchronize()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        cp.run(x_dev)
        c1.record(stream)
        torch.cuda.synchronize()
        cms = c0.elapsed_time(c1)
        cufft = {"value": n / (cms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": cms,
                 "kind": "cuFFT R2C + inverse-filter multiply + batched C2C inverse (torch.fft) + torch detect, "
                         "fold, decimate; same outputs (tests/test_gpu_cufft_baseline.py)",
                 "engine_speedup": (value / ws) / (n / (cms / 1e3) / 1e6)}
        del cp

    # end to end through pond_push from pinned host memory, results read back
    x_host = torch.empty(n * ch, dtype=torch.int8, pin_memory=True)
    x_host.copy_(x_dev)
    xh = x_host.numpy()
    torch.cuda.synchronize()
    # the host link's copy rate at this moment: the e2e step overlaps the copies with the
    # compute, so it is copy-bound only when this rate falls below n / device step time
    h2d_s = []
    for _ in range(4):
        t0 = time.perf_counter()
        x_dev.copy_(x_host, non_blocking=True)
        torch.cuda.synchronize()
        h2d_s.append(time.perf_counter() - t0)
    h2d_gbs = n * ch / min(h2d_s) / 1e9
    eng_h = pond.Engine(F0, BW, FS, PLAN["dm"], PLAN["nfft"], PLAN["nchan"], PLAN["nbins"], PLAN["period"],
                        t_dec=PLAN["t_dec"], device=local, precision=prec, input_channels=ch, chirp=chirp)
    prof = {}
    phases = []
    # the series lands in page-locked arrays the caller keeps across steps
    cap_ts = int(n / (PLAN["t_dec"] * FS)) + 4096      # series samples of one step, with room
    T_pin = torch.empty(cap_ts, dtype=torch.float32, pin_memory=True).numpy()
    C_pin = torch.empty(cap_ts, dtype=torch.int32, pin_memory=True).numpy()

    def step_host():
        a = time.perf_counter()
        eng_h.reset()
        b = time.perf_counter()
        eng_h.push(xh)
        c = time.perf_counter()
        eng_h.flush()
        d = time.perf_counter()
        s, h, _ = eng_h.profile()
        nt, _ = eng_h.timeseries_into(T_pin, C_pin)
        e = time.perf_counter()
        prof["bytes"] = s.nbytes + h.nbytes + nt * (T_pin.itemsize + C_pin.itemsize)
        phases.append((b - a, c - b, d - c, e - d))

    for _ in range(max(1, args.warmup)):
        step_host()
    quiet_gc()
    barrier(dist)
    torch.cuda.synchronize()
    phases.clear()
    # at least 20 steps (about 0.4 s): a single host-side stall of tens of ms (thread
    # scheduling, memory contention from other processes) stays in the figure but
    # weighs less; the step spread and the slowest step's phases below show it
    e2e_steps = max(args.steps, 20)
    t0 = time.perf_counter()
    marks = [t0]
    for _ in range(e2e_steps):
        step_host()
        marks.append(time.perf_counter())
    t1 = marks[-1]
    e2e_s = max_over_ranks(dist, t1 - t0)
    steps_ms = [1e3 * (b - a) for a, b in zip(marks, marks[1:])]
    step_ms = sorted(steps_ms)
    slow = max(range(len(steps_ms)), key=lambda k: steps_ms[k])
    e2e = {"value": ws * n * e2e_steps / e2e_s / 1e6, "unit": UNIT, "steps": e2e_steps, "h2d_bytes_per_step": n * ch,
           "d2h_bytes_per_step": prof["bytes"], "h2d_copy_gbs": h2d_gbs,
           "copy_bound_below_gbs": n * ch / (ms / args.steps / 1e3) / 1e9,
           "step_ms_min_median_max": [step_ms[0], statistics.median(step_ms), step_ms[-1]],
           "slowest_step": {"index": slow, "ms": steps_ms[slow],
                            "reset_push_flush_read_ms": [1e3 * v for v in phases[slow]]}}

    # the FP64 oracle on the host cores: one thread, then every core (one process per core)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline and ch == 1:
        host = host_cpu()
        v1, nseg1, samples1, dt1 = oracle_rate(xh[:16 * (1 << 24)], seconds_budget=10.0)
        pool = OraclePool(xh[:8 * x_host_seg_step() + PLAN["nfft"]])
        samples_all, wall_all, nseg_all = pool.round(2)
        pool.close()
        v_all = samples_all / wall_all / 1e6
        cpu = {"value": v_all, "unit": UNIT, "cores": pool.workers, "kind": "oracle", "host": host,
               "sample": f"{nseg_all} whole nfft-2^24 segments ({samples_all} samples advanced) of the same stream "
                         f"on {pool.workers} processes (two each), {wall_all:.1f} s wall, FP64 numpy",
               "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                                 "sample": f"{nseg1} whole segments ({samples1} samples advanced), "
                                           f"{dt1:.1f} s on 1 host thread"}}

    # the precision form and the batched trials on the same GPU, one short run each
    extra = {}
    if rank == 0 and not args.no_forms and ch == 1 and prec == pond.POND_FP32:
        eng.close()
        eng_h.close()
        eng = eng_h = None
        torch.cuda.empty_cache()
        extra["precision"] = precision_brief(dev, local, stream)
        del x_dev
        torch.cuda.empty_cache()
        b = batched_core(dev, local, stream, steps=2, warmup=1)
        bval = b["n"] * 2 / (b["ms"] / 1e3) / 1e6
        extra["batched"] = {"workload": BATCHED_WORKLOAD, "value": bval, "unit": UNIT,
                            "realtime_factor": bval / REALTIME_MSPS, "ms_per_step": b["ms"] / 2,
                            "trial_samples_per_s": bval * 1e6 * 128, "nfft_groups": b["groups"],
                            "plan_s_incl_autotune": b["plan_s"], "tuning": b["tuning"],
                            "gpu_launches_per_step": b["launches_per_step"], "clocks": b["clocks"]}
        # the learned form at the default scale (40 training chunks, 16 shifts per event)
        torch.cuda.empty_cache()
        lr_ = learned_core(40, 16, 20)
        lr_["metric"] = "single-pulse candidates classified per second (CNN inference)"
        extra["learned"] = lr_
    clocks = clk.summary()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp32": "f32", "bf16x3": "bf16x3+f32acc", "bf16x5": "bf16x5+f32acc"}[args.precision],
                "data": "synthetic", "config": dict(workload_config(n, ch), fft_stages=args.precision,
                              chirp={"auto": "table (default)", "anchors": "anchors", "table": "table"}[args.chirp]),
                "realtime_factor": value / REALTIME_MSPS,
                "e2e": e2e, "gpu_launches": int(st1["kernel_launches"]) * args.steps,
                "roofline": roof, "cpu_baseline": cpu, "cufft_baseline": cufft, "clocks": clocks}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if eng is not None:
        eng.close()
    if eng_h is not None:
        eng_h.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
