"""ctypes binding of libpond.so: the C ABI of include/pond.h, argument marshalling only.

Every computation runs in the library's CUDA kernels; this module converts
Python/numpy/torch arguments to pointers and sizes and raises ``PondError`` on
a negative return code.  It fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libpond.so")

POND_OK = 0
POND_E_ARG = -1
POND_E_NFFT = -2
POND_E_NCHAN = -3
POND_E_OOM = -4
POND_E_CUDA = -5
POND_E_STATE = -6
POND_E_OVERRUN = -7
POND_E_TIMEOUT = -8
POND_E_UNIMPLEMENTED = -9
POND_FP32 = 0
POND_SPLIT_BF16 = 1
POND_SPLIT_BF16_5T = 2
POND_SCHEDULE_AUTO = 0
POND_SCHEDULE_FOUR_PASS = 1
POND_CHIRP_AUTO = 0
POND_CHIRP_ANCHORS = 1
POND_CHIRP_TABLE = 2
POND_TRIALS_AUTO = 0
POND_TRIALS_PER_TRIAL = 1
POND_TRIALS_MULTI_ANCHOR = 2
POND_TRIALS_MULTI_TABLE = 3
POND_TRIALS_FOUR_PASS = 4
TRIAL_MODE_NAMES = {POND_TRIALS_PER_TRIAL: "per-trial", POND_TRIALS_MULTI_ANCHOR: "multi-anchor",
                    POND_TRIALS_MULTI_TABLE: "multi-table", POND_TRIALS_FOUR_PASS: "four-pass"}
POND_NSTAGE = 9
POND_NOALLOC_MAX_NBINS = 1024
POND_STACK_ROTATION = 0
POND_STACK_SUBINT = 1
POND_INCOH_AID = 0
POND_INCOH_CID = 1

CODE_NAMES = {POND_E_ARG: "ARG", POND_E_NFFT: "NFFT", POND_E_NCHAN: "NCHAN", POND_E_OOM: "OOM",
              POND_E_CUDA: "CUDA", POND_E_STATE: "STATE", POND_E_OVERRUN: "OVERRUN",
              POND_E_TIMEOUT: "TIMEOUT", POND_E_UNIMPLEMENTED: "UNIMPLEMENTED"}

# Functions declared in include/pond.h.
EXPORTS = ["pond_plan", "pond_plan_ex", "pond_push", "pond_push_device", "pond_flush", "pond_sync",
           "pond_reset",
           "pond_profile", "pond_timeseries", "pond_voltages", "pond_stats", "pond_strerror",
           "pond_last_error", "pond_destroy", "pond_fold_noalloc", "pond_trials",
           "pond_boxcar", "pond_candidates", "pond_candidates_scored", "pond_check_bounded_wait", "pond_cnn_create", "pond_cnn_set_params", "pond_cnn_params",
           "pond_cnn_forward", "pond_cnn_gradient", "pond_cnn_train_step", "pond_cnn_destroy", "pond_patches",
           "pond_incoh_create", "pond_incoh_run", "pond_incoh_info_get", "pond_incoh_filterbank",
           "pond_incoh_series", "pond_incoh_profile", "pond_incoh_delays", "pond_incoh_destroy", "pond_incoh_ips",
           "pond_stack_rows", "pond_fold_stack", "pond_probe_fp32_fma", "pond_tuning"]


class PondError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{CODE_NAMES.get(code, code)}: {msg}")
        self.code = code
        self.name = CODE_NAMES.get(code, str(code))


class pond_opts(ctypes.Structure):
    _fields_ = [("f0_mhz", ctypes.c_double), ("bw_mhz", ctypes.c_double), ("fs_hz", ctypes.c_double),
                ("dm", ctypes.c_double), ("nfft", ctypes.c_int64), ("nchan", ctypes.c_int32),
                ("nbins", ctypes.c_int32), ("period_s", ctypes.c_double), ("t_dec_s", ctypes.c_double),
                ("epoch_mjd_day", ctypes.c_int32), ("epoch_mjd_sec", ctypes.c_double),
                ("precision", ctypes.c_int32), ("want_voltages", ctypes.c_int32),
                ("timing", ctypes.c_int32), ("device", ctypes.c_int32),
                ("ndm", ctypes.c_int32), ("dm_list", ctypes.POINTER(ctypes.c_double)),
                ("nfft_choices", ctypes.c_int64 * 4), ("autotune", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("input_channels", ctypes.c_int32),
                ("trial_mode", ctypes.c_int32), ("trials_per_launch", ctypes.c_int32),
                ("chirp", ctypes.c_int32), ("inv_split", ctypes.c_int32), ("phase_ncoef", ctypes.c_int32),
                ("phase_tref_s", ctypes.c_double), ("phase_coef", ctypes.c_double * 8)]


POND_TUNE_MAXCAND = 12


class pond_lane_info(ctypes.Structure):
    _fields_ = [("nfft", ctypes.c_int64), ("ntrials", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("trials_per_launch", ctypes.c_int32), ("ncand", ctypes.c_int32), ("inv_split", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("dm_step", ctypes.c_double),
                ("cand_mode", ctypes.c_int32 * POND_TUNE_MAXCAND), ("cand_kt", ctypes.c_int32 * POND_TUNE_MAXCAND),
                ("cand_split", ctypes.c_int32 * POND_TUNE_MAXCAND), ("cand_us", ctypes.c_double * POND_TUNE_MAXCAND)]


class pond_meta(ctypes.Structure):
    _fields_ = [("epoch_mjd_day", ctypes.c_int32), ("epoch_mjd_sec", ctypes.c_double),
                ("period_s", ctypes.c_double), ("dm", ctypes.c_double), ("dtc_s", ctypes.c_double),
                ("first_g", ctypes.c_int64), ("nsamples", ctypes.c_int64), ("nbins", ctypes.c_int32)]


class pond_cand(ctypes.Structure):
    _fields_ = [("trial", ctypes.c_int32), ("width", ctypes.c_int32), ("index", ctypes.c_int64),
                ("snr", ctypes.c_double), ("dm", ctypes.c_double), ("score", ctypes.c_float),
                ("reserved", ctypes.c_int32)]


class pond_stats_t(ctypes.Structure):
    _fields_ = [("samples_in", ctypes.c_int64), ("segments", ctypes.c_int64), ("outputs", ctypes.c_int64),
                ("n_past", ctypes.c_int64), ("n_fut", ctypes.c_int64), ("seg_step", ctypes.c_int64),
                ("nfft", ctypes.c_int32), ("nchan", ctypes.c_int32), ("kernel_launches", ctypes.c_int32),
                ("flushed", ctypes.c_int32), ("stage_ms", ctypes.c_double * POND_NSTAGE),
                ("stage_launches", ctypes.c_int64 * POND_NSTAGE),
                ("pass_bytes", ctypes.c_double * POND_NSTAGE),
                ("stage_name", ctypes.c_char_p * POND_NSTAGE),
                ("algo_flops", ctypes.c_double * POND_NSTAGE), ("push_enqueue_ms", ctypes.c_double),
                ("push_wait_ms", ctypes.c_double)]


_lib = None


class pond_incoh_opts(ctypes.Structure):
    _fields_ = [("f0_mhz", ctypes.c_double), ("bw_mhz", ctypes.c_double), ("fs_hz", ctypes.c_double),
                ("dm", ctypes.c_double), ("period_s", ctypes.c_double), ("nchan", ctypes.c_int32),
                ("nint", ctypes.c_int32), ("mode", ctypes.c_int32), ("input_channels", ctypes.c_int32),
                ("nbins", ctypes.c_int32), ("device", ctypes.c_int32), ("ips_len", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 5)]


class pond_incoh_info(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int64), ("t_first", ctypes.c_int64), ("n_out", ctypes.c_int64),
                ("ips_chunks", ctypes.c_int64), ("d_min", ctypes.c_int32), ("d_max", ctypes.c_int32),
                ("ts", ctypes.c_double), ("ms_filterbank", ctypes.c_double), ("ms_dedisperse", ctypes.c_double),
                ("ms_fold", ctypes.c_double), ("ms_ips", ctypes.c_double), ("algo_bytes_filterbank", ctypes.c_double),
                ("algo_bytes_dedisperse", ctypes.c_double), ("launches", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]


def lib() -> ctypes.CDLL:
    """Load libpond.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built: run __graft_entry__.build() first")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    sig = {
        "pond_plan": [P(vp), ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                      ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_double],
        "pond_plan_ex": [P(vp), P(pond_opts)],
        "pond_push": [vp, vp, ctypes.c_size_t],
        "pond_push_device": [vp, vp, ctypes.c_size_t, vp],
        "pond_flush": [vp],
        "pond_sync": [vp],
        "pond_reset": [vp],
        "pond_profile": [vp, vp, vp, P(pond_meta)],
        "pond_timeseries": [vp, vp, vp, ctypes.c_size_t, P(ctypes.c_size_t), P(ctypes.c_int64)],
        "pond_voltages": [vp, vp, ctypes.c_size_t, P(ctypes.c_size_t), P(ctypes.c_int64)],
        "pond_stats": [vp, P(pond_stats_t)],
        "pond_strerror": [ctypes.c_int],
        "pond_last_error": [],
        "pond_destroy": [vp],
        "pond_fold_noalloc": [vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                              ctypes.c_int32, vp, vp, vp],
        "pond_trials": [vp, vp, vp, ctypes.c_int32, P(ctypes.c_int32)],
        "pond_boxcar": [vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_double, vp,
                        ctypes.c_size_t, P(ctypes.c_size_t), vp],
        "pond_candidates": [vp, ctypes.c_double, vp, ctypes.c_size_t, P(ctypes.c_size_t)],
        "pond_candidates_scored": [vp, vp, ctypes.c_double, vp, ctypes.c_size_t, P(ctypes.c_size_t)],
        "pond_check_bounded_wait": [ctypes.c_double, ctypes.c_int32, P(ctypes.c_double)],
        "pond_cnn_create": [P(vp), vp, ctypes.c_int32, ctypes.c_int32],
        "pond_cnn_set_params": [vp, vp],
        "pond_cnn_params": [vp, vp],
        "pond_cnn_forward": [vp, vp, ctypes.c_int32, vp, vp],
        "pond_cnn_gradient": [vp, vp, vp, ctypes.c_int32, vp, vp, vp],
        "pond_cnn_train_step": [vp, vp, vp, ctypes.c_int32, ctypes.c_float, vp, vp],
        "pond_cnn_destroy": [vp],
        "pond_patches": [vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, vp, ctypes.c_int32, vp, vp],
        "pond_incoh_create": [P(vp), P(pond_incoh_opts)],
        "pond_incoh_run": [vp, vp, ctypes.c_size_t, vp],
        "pond_incoh_info_get": [vp, P(pond_incoh_info)],
        "pond_incoh_filterbank": [vp, vp, ctypes.c_size_t, P(ctypes.c_int64)],
        "pond_incoh_series": [vp, vp, ctypes.c_size_t, P(ctypes.c_int64), P(ctypes.c_int64)],
        "pond_incoh_profile": [vp, vp, vp],
        "pond_incoh_delays": [vp, vp],
        "pond_incoh_ips": [vp, vp, P(ctypes.c_int64)],
        "pond_stack_rows": [ctypes.c_int64, ctypes.c_int64, ctypes.c_double, vp, ctypes.c_int32, ctypes.c_double,
                            ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, P(ctypes.c_int64), P(ctypes.c_int64)],
        "pond_fold_stack": [vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_double, vp, ctypes.c_int32, ctypes.c_double,
                            ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, vp, vp, ctypes.c_int64,
                            P(ctypes.c_int64), P(ctypes.c_int64), vp],
        "pond_incoh_destroy": [vp],
        "pond_probe_fp32_fma": [vp, ctypes.c_int32, ctypes.c_int32, vp, P(ctypes.c_double)],
        "pond_tuning": [vp, vp, ctypes.c_int32, P(ctypes.c_int32)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_char_p if name in ("pond_strerror", "pond_last_error") else ctypes.c_int
    _lib = L
    return L


def _check(rc: int) -> None:
    if rc != POND_OK:
        msg = lib().pond_last_error().decode(errors="replace")
        raise PondError(rc, msg or lib().pond_strerror(rc).decode())


def cand_dict(c) -> dict:
    return {"trial": c.trial, "width": c.width, "index": c.index, "snr": c.snr, "dm": c.dm, "score": c.score}


def check_bounded_wait(limit_s: float = 0.05, device: int = 0) -> tuple[int, float]:
    """Run the bounded-wait self-check: (return code, seconds waited).  The
    expected code is POND_E_TIMEOUT (the wait gave up by itself)."""
    w = ctypes.c_double()
    rc = lib().pond_check_bounded_wait(limit_s, device, ctypes.byref(w))
    return rc, w.value


def probe_fp32_fma(d_out_ptr: int, blocks: int, iters: int, stream: int = 0) -> float:
    """Enqueue the FP32 FMA ceiling probe on `stream`; returns the FP32 operations enqueued."""
    fl = ctypes.c_double()
    _check(lib().pond_probe_fp32_fma(d_out_ptr, blocks, iters, stream, ctypes.byref(fl)))
    return fl.value


def boxcar(d_series_ptr: int, ndm: int, n: int, stride: int, threshold: float = 6.0, cap: int = 1 << 16,
           stream: int = 0):
    """pond_boxcar over a device series block [ndm][stride]: list of candidate dicts."""
    out = (pond_cand * cap)()
    nf = ctypes.c_size_t()
    _check(lib().pond_boxcar(d_series_ptr, ndm, n, stride, threshold, out, cap, ctypes.byref(nf), stream))
    return [cand_dict(out[i]) for i in range(nf.value)]


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data if a is not None else 0


class Engine:
    """One coherent-dedispersion stream (a ``pond_t`` handle)."""

    def __init__(self, f0: float, bw: float, fs: float, dm: float, nfft: int, nchan: int, nbins: int,
                 period: float, t_dec: float = 61.44e-6, want_voltages: bool = False,
                 timing: bool = False, device: int = 0, epoch_mjd: tuple[int, float] = (0, 0.0),
                 precision: int = POND_FP32, dms=None, nfft_choices=(), autotune: bool = False,
                 schedule: int = POND_SCHEDULE_AUTO, input_channels: int = 1, trial_mode: int = POND_TRIALS_AUTO,
                 trials_per_launch: int = 0, chirp: int = POND_CHIRP_AUTO, inv_split: int = 0,
                 phase_model=None):
        """A single-DM plan, or with ``dms`` a batched plan over those DM trials.
        ``phase_model`` = (t_ref seconds, coefficients): fold with that polynomial
        phase instead of the constant period (single-DM plans)."""
        o = pond_opts()
        o.f0_mhz, o.bw_mhz, o.fs_hz, o.dm = f0, bw, fs, dm
        o.nfft, o.nchan, o.nbins, o.period_s = nfft, nchan, nbins, period
        o.t_dec_s = t_dec
        o.epoch_mjd_day, o.epoch_mjd_sec = int(epoch_mjd[0]), float(epoch_mjd[1])
        o.precision = precision
        o.want_voltages = int(bool(want_voltages))
        o.timing = int(bool(timing))
        o.device = device
        o.schedule = schedule
        o.input_channels = input_channels
        o.trial_mode = trial_mode
        o.trials_per_launch = trials_per_launch
        o.chirp = chirp
        o.inv_split = inv_split
        if phase_model is not None:
            t_ref, coef = phase_model
            coef = [float(c) for c in coef]
            o.phase_ncoef = len(coef)
            o.phase_tref_s = float(t_ref)
            for i, c in enumerate(coef[:8]):
                o.phase_coef[i] = c
        self._dms = None
        if dms is not None:
            self._dms = (ctypes.c_double * len(dms))(*[float(d) for d in dms])
            o.ndm = len(dms)
            o.dm_list = ctypes.cast(self._dms, ctypes.POINTER(ctypes.c_double))
            o.autotune = int(bool(autotune))
            for i, n in enumerate(list(nfft_choices)[:4]):
                o.nfft_choices[i] = int(n)
        self.ndm = len(dms) if dms is not None else 0
        self.nbins = nbins
        self.nchan = nchan
        h = ctypes.c_void_p()
        _check(lib().pond_plan_ex(ctypes.byref(h), ctypes.byref(o)))
        self._h = h

    @property
    def handle(self) -> int:
        return self._h.value

    def push(self, x: np.ndarray) -> None:
        """Append host int8 samples (copied before return)."""
        x = np.ascontiguousarray(x, dtype=np.int8)
        _check(lib().pond_push(self._h, _ptr(x), x.size))

    def push_device(self, ptr: int, n: int, stream: int = 0) -> None:
        """Append n int8 samples at device address ptr, ordered on ``stream``."""
        _check(lib().pond_push_device(self._h, ptr, n, stream))

    def push_tensor(self, t, stream=None) -> None:
        """Append a CUDA int8 tensor, ordered on ``stream`` (default: torch's current)."""
        import torch
        assert t.is_cuda and t.dtype == torch.int8 and t.is_contiguous()
        s = stream if stream is not None else torch.cuda.current_stream(t.device)
        self.push_device(t.data_ptr(), t.numel(), s.cuda_stream)

    def flush(self) -> None:
        _check(lib().pond_flush(self._h))

    def sync(self) -> None:
        _check(lib().pond_sync(self._h))

    def reset(self) -> None:
        """Start a new stream with the same plan."""
        _check(lib().pond_reset(self._h))

    def profile(self):
        s = np.zeros(self.nbins, dtype=np.float64)
        h = np.zeros(self.nbins, dtype=np.int64)
        m = pond_meta()
        _check(lib().pond_profile(self._h, _ptr(s), _ptr(h), ctypes.byref(m)))
        meta = {f: getattr(m, f) for f, _ in pond_meta._fields_}
        return s, h, meta

    def timeseries(self, cap: int = 1 << 20):
        """Drain every completed time-series sample: (T float32, counts int32, first index).

        T is 1-D for a single-DM plan and [ndm, n] for a batched plan."""
        rows = max(1, self.ndm)
        parts, cparts, first = [], [], None
        while True:
            out = np.empty((rows, cap), dtype=np.float32)   # the library fills [:, :n]
            cnt = np.empty(cap, dtype=np.int32)
            n = ctypes.c_size_t()
            j0 = ctypes.c_int64()
            _check(lib().pond_timeseries(self._h, _ptr(out), _ptr(cnt), cap, ctypes.byref(n),
                                         ctypes.byref(j0)))
            if first is None:
                first = j0.value
            if n.value == 0:
                break
            parts.append(out[:, :n.value])
            cparts.append(cnt[:n.value])
            if n.value < cap:
                break
        if len(parts) == 1:   # a single drain: no concatenation (rows of a batched plan made contiguous)
            T, C = (parts[0] if rows == 1 else np.ascontiguousarray(parts[0])), cparts[0]
        else:
            T = np.concatenate(parts, axis=1) if parts else np.zeros((rows, 0), np.float32)
            C = np.concatenate(cparts) if cparts else np.zeros(0, np.int32)
        return (T if self.ndm else T[0]), C, first

    def timeseries_into(self, T: np.ndarray, C: np.ndarray) -> tuple[int, int]:
        """Drain completed series samples into caller arrays: T float32 ([ndm, cap]
        for a batched plan, [cap] otherwise), C int32 [cap].  Returns (samples
        written, index of the first).  Arrays in page-locked memory (e.g. a
        pinned torch tensor's numpy view) receive the device's rows directly."""
        rows = max(1, self.ndm)
        cap = C.shape[0]
        assert T.dtype == np.float32 and C.dtype == np.int32 and T.size == rows * cap
        assert T.flags.c_contiguous and C.flags.c_contiguous
        n = ctypes.c_size_t()
        j0 = ctypes.c_int64()
        _check(lib().pond_timeseries(self._h, _ptr(T), _ptr(C), cap, ctypes.byref(n), ctypes.byref(j0)))
        return n.value, j0.value

    def candidates(self, threshold: float = 6.0, cap: int = 1 << 16, classifier=None):
        """Boxcar candidates over the completed, undrained series: list of dicts.
        With ``classifier`` (a Classifier on the same device) each candidate's
        score is the network's dispersed-pulse probability for its patch."""
        out = (pond_cand * cap)()
        n = ctypes.c_size_t()
        if classifier is None:
            _check(lib().pond_candidates(self._h, threshold, out, cap, ctypes.byref(n)))
        else:
            _check(lib().pond_candidates_scored(self._h, classifier.handle, threshold, out, cap, ctypes.byref(n)))
        return [cand_dict(out[i]) for i in range(n.value)]

    def trials(self):
        """(DM, FFT length) of every trial, in the order the plan was given."""
        n = ctypes.c_int32()
        _check(lib().pond_trials(self._h, None, None, 0, ctypes.byref(n)))
        dm = np.zeros(n.value, np.float64)
        nf = np.zeros(n.value, np.int64)
        _check(lib().pond_trials(self._h, _ptr(dm), _ptr(nf), n.value, ctypes.byref(n)))
        return dm, nf

    def tuning(self) -> list:
        """How each lane runs its trials: FFT length, trials, mode, trials per
        launch, the four-pass inverse split (log2 Q1), DM step of the table form,
        and the autotuner's timed candidates."""
        n = ctypes.c_int32()
        _check(lib().pond_tuning(self._h, None, 0, ctypes.byref(n)))
        arr = (pond_lane_info * max(1, n.value))()
        _check(lib().pond_tuning(self._h, arr, n.value, ctypes.byref(n)))
        out = []
        for r in arr[:n.value]:
            out.append({"nfft": r.nfft, "ntrials": r.ntrials, "mode": TRIAL_MODE_NAMES.get(r.mode, r.mode),
                        "trials_per_launch": r.trials_per_launch, "inv_split": r.inv_split,
                        "dm_step": r.dm_step,
                        "candidates_us_per_trial": [
                            {"mode": TRIAL_MODE_NAMES.get(r.cand_mode[c], r.cand_mode[c]),
                             "trials_per_launch": r.cand_kt[c], "inv_split": r.cand_split[c],
                             "us": r.cand_us[c]} for c in range(r.ncand)]})
        return out

    def voltages(self, cap: int = 1 << 22):
        """Drain every kept dedispersed voltage: (complex64 [nchan, n], first g)."""
        parts, first = [], None
        while True:
            out = np.zeros((self.nchan, cap, 2), dtype=np.float32)
            n = ctypes.c_size_t()
            g0 = ctypes.c_int64()
            _check(lib().pond_voltages(self._h, _ptr(out), cap, ctypes.byref(n), ctypes.byref(g0)))
            if first is None:
                first = g0.value
            if n.value:
                parts.append((out[:, :n.value, 0] + 1j * out[:, :n.value, 1]).astype(np.complex64))
            if n.value < cap:
                break
        v = np.concatenate(parts, axis=1) if parts else np.zeros((self.nchan, 0), np.complex64)
        return v, first

    def stats(self) -> dict:
        s = pond_stats_t()
        _check(lib().pond_stats(self._h, ctypes.byref(s)))
        d = {f: getattr(s, f) for f, _ in pond_stats_t._fields_ if f not in
             ("stage_ms", "stage_launches", "pass_bytes", "stage_name", "algo_flops")}
        d["stages"] = {}
        for i in range(POND_NSTAGE):
            name = s.stage_name[i]
            if name:
                d["stages"][name.decode()] = {"ms": s.stage_ms[i], "launches": s.stage_launches[i],
                                              "pass_bytes": s.pass_bytes[i], "algo_flops": s.algo_flops[i]}
        return d

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().pond_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


CNN_NPARAM = 21732


class Classifier:
    """The single-pulse candidate classifier (a ``pond_cnn_t``)."""

    def __init__(self, params: np.ndarray, max_batch: int = 512, device: int = 0):
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == CNN_NPARAM
        h = ctypes.c_void_p()
        _check(lib().pond_cnn_create(ctypes.byref(h), _ptr(p), max_batch, device))
        self._h = h
        self.max_batch = max_batch

    @property
    def handle(self) -> int:
        return self._h.value

    def params(self) -> np.ndarray:
        out = np.zeros(CNN_NPARAM, np.float32)
        _check(lib().pond_cnn_params(self._h, _ptr(out)))
        return out

    def set_params(self, params: np.ndarray) -> None:
        p = np.ascontiguousarray(params, dtype=np.float32)
        _check(lib().pond_cnn_set_params(self._h, _ptr(p)))

    def forward(self, x, stream: int = 0):
        """Probabilities [B, 4] (torch CUDA tensor) of BF16 patches x [B, 32, 256]."""
        import torch
        prob = torch.empty((x.shape[0], 4), dtype=torch.float32, device=x.device)
        _check(lib().pond_cnn_forward(self._h, x.data_ptr(), x.shape[0], prob.data_ptr(), stream))
        return prob

    def gradient(self, x, labels, stream: int = 0):
        g = np.zeros(CNN_NPARAM, np.float32)
        loss = ctypes.c_float()
        _check(lib().pond_cnn_gradient(self._h, x.data_ptr(), labels.data_ptr(), x.shape[0], _ptr(g),
                                       ctypes.byref(loss), stream))
        return float(loss.value), g

    def train_step(self, x, labels, lr: float, stream: int = 0, want_loss: bool = False):
        loss = ctypes.c_float()
        _check(lib().pond_cnn_train_step(self._h, x.data_ptr(), labels.data_ptr(), x.shape[0], lr,
                                         ctypes.byref(loss) if want_loss else None, stream))
        return float(loss.value) if want_loss else None

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().pond_cnn_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def patches(series, corners, stream: int = 0):
    """BF16 patches [P, 32, 256] from a device series block [ndm, n] and int32 corners [P, 2]."""
    import torch
    assert series.dtype == torch.float32 and series.is_cuda and corners.dtype == torch.int32
    out = torch.empty((corners.shape[0], 32, 256), dtype=torch.bfloat16, device=series.device)
    _check(lib().pond_patches(series.data_ptr(), series.shape[0], series.shape[1], series.stride(0),
                              corners.data_ptr(), corners.shape[0], out.data_ptr(), stream))
    return out


class Incoherent:
    """Incoherent dedispersion (PONDER Sec. 3.4): FFT filterbank, AID or CID
    detection, integration, Eq. 3 channel shifts with the channel sum, fold.
    One ``run`` processes one whole buffer of int8 input."""

    def __init__(self, f0: float, bw: float, fs: float, dm: float, nchan: int, nint: int, nbins: int,
                 period: float, mode: int = POND_INCOH_AID, input_channels: int = 1, device: int = 0,
                 ips_len: int = 0):
        o = pond_incoh_opts()
        o.f0_mhz, o.bw_mhz, o.fs_hz, o.dm, o.period_s = f0, bw, fs, dm, period
        o.nchan, o.nint, o.mode, o.input_channels, o.nbins, o.device = nchan, nint, mode, input_channels, nbins, device
        o.ips_len = ips_len
        h = ctypes.c_void_p()
        _check(lib().pond_incoh_create(ctypes.byref(h), ctypes.byref(o)))
        self._h = h
        self.nchan, self.nbins, self.channels, self.ips_len = nchan, nbins, input_channels, ips_len
        self.device = device

    def run_device(self, ptr: int, nbytes: int, stream: int = 0) -> None:
        """Enqueue the mode over nbytes of int8 at device address ptr on ``stream``."""
        _check(lib().pond_incoh_run(self._h, ptr, nbytes, stream))

    def run_tensor(self, t, stream=None) -> None:
        """Enqueue the mode over a CUDA int8 tensor (default: torch's current stream)."""
        import torch
        assert t.is_cuda and t.dtype == torch.int8 and t.is_contiguous()
        s = stream if stream is not None else torch.cuda.current_stream(t.device)
        self.run_device(t.data_ptr(), t.numel(), s.cuda_stream)

    def run(self, x, stream=None) -> None:
        """Copy host int8 input (a numpy array, or a CPU int8 tensor, ideally in pinned
        memory) to the device and run."""
        import torch
        dev = torch.device("cuda", self.device)
        if isinstance(x, torch.Tensor):
            assert x.device.type == "cpu" and x.dtype == torch.int8
            src = x.contiguous()
        else:
            src = torch.from_numpy(np.ascontiguousarray(x, dtype=np.int8))
        if not src.is_pinned():
            src = src.pin_memory()
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        with torch.cuda.stream(s):      # the buffer belongs to the stream that copies and reads it
            d = torch.empty(src.numel(), dtype=torch.int8, device=dev)
            d.copy_(src, non_blocking=True)
        self.run_tensor(d, s)
        self._keep = (src, d)      # alive until the next run or a result read

    def info(self) -> dict:
        i = pond_incoh_info()
        _check(lib().pond_incoh_info_get(self._h, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in pond_incoh_info._fields_ if f != "reserved"}

    def filterbank(self) -> np.ndarray:
        """The integrated filterbank of the last run, [T][nchan] (time-major)."""
        T = ctypes.c_int64()
        rc = lib().pond_incoh_filterbank(self._h, None, 0, ctypes.byref(T))
        if rc not in (POND_OK, POND_E_OVERRUN):
            _check(rc)
        out = np.empty((T.value, self.nchan), np.float32)
        _check(lib().pond_incoh_filterbank(self._h, _ptr(out) if out.size else None, out.size, ctypes.byref(T)))
        return out

    def series(self):
        """(D, t_first): the dedispersed series of the last run and its first sample index."""
        n, t0 = ctypes.c_int64(), ctypes.c_int64()
        rc = lib().pond_incoh_series(self._h, None, 0, ctypes.byref(n), ctypes.byref(t0))
        if rc not in (POND_OK, POND_E_OVERRUN):
            _check(rc)
        out = np.empty(n.value, np.float32)
        _check(lib().pond_incoh_series(self._h, _ptr(out) if out.size else None, out.size, ctypes.byref(n),
                                       ctypes.byref(t0)))
        return out, t0.value

    def profile(self):
        s = np.empty(self.nbins, np.float64)
        h = np.empty(self.nbins, np.int64)
        _check(lib().pond_incoh_profile(self._h, _ptr(s), _ptr(h)))
        return s, h

    def ips(self):
        """(A, J): the accumulated fluctuation spectrum (ips_len / 2 + 1 bins) of the
        last run's series and the number of chunks in it (Sec. 3.5)."""
        out = np.empty(max(self.ips_len, 2) // 2 + 1, np.float64)
        j = ctypes.c_int64()
        _check(lib().pond_incoh_ips(self._h, _ptr(out), ctypes.byref(j)))
        return out, j.value

    def delays(self) -> np.ndarray:
        d = np.empty(self.nchan, np.int32)
        _check(lib().pond_incoh_delays(self._h, _ptr(d)))
        return d

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().pond_incoh_destroy(self._h)
            self._h = None
        self._keep = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stack_rows(n: int, g0: int, dt: float, coef, t_ref: float, nbins: int, mode: int = POND_STACK_ROTATION,
               n_sub: int = 0):
    """(rows, first rotation) of the stack pond_fold_stack fills (host arithmetic only)."""
    c = np.ascontiguousarray(coef, dtype=np.float64)
    rows, q0 = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().pond_stack_rows(n, g0, dt, _ptr(c), c.size, t_ref, nbins, mode, n_sub, ctypes.byref(rows),
                                 ctypes.byref(q0)))
    return rows.value, q0.value


def fold_stack(series, g0: int, dt: float, coef, t_ref: float, nbins: int, mode: int = POND_STACK_ROTATION,
               n_sub: int = 0, stream=None):
    """Fold a CUDA FP32 series with a polynomial phase model into a pulse stack:
    (S [rows][nbins] FP64, H [rows][nbins] int64, first rotation), on the host."""
    import torch
    assert series.is_cuda and series.dtype == torch.float32 and series.is_contiguous()
    n = series.numel()
    rows, _ = stack_rows(n, g0, dt, coef, t_ref, nbins, mode, n_sub)
    S = torch.empty((max(rows, 1), nbins), dtype=torch.float64, device=series.device)
    H = torch.empty((max(rows, 1), nbins), dtype=torch.int64, device=series.device)
    c = np.ascontiguousarray(coef, dtype=np.float64)
    s = stream if stream is not None else torch.cuda.current_stream(series.device)
    r, q0 = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().pond_fold_stack(series.data_ptr(), n, g0, dt, _ptr(c), c.size, t_ref, nbins, mode, n_sub,
                                 S.data_ptr(), H.data_ptr(), rows, ctypes.byref(r), ctypes.byref(q0), s.cuda_stream))
    s.synchronize()
    return S[:r.value].cpu().numpy(), H[:r.value].cpu().numpy(), q0.value
