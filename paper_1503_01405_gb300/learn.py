"""The candidate classifier's data, training and evaluation (orchestration only).

Labelled chunks come from ``synth.make_labelled_chunk_torch``; the batched
engine dedisperses them into DM-trial series; patches are cut around each
event with ``pond_patches``; the network trains with ``pond_cnn_train_step``
and is compared with the boxcar detector (``pond_candidates``), which flags a
patch when a candidate with S/N >= 6 at a trial with DM > 0 lies inside it.
Every numerical step runs in the library's kernels; this module moves
pointers, shuffles indices and counts outcomes.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import pond, synth

DT = 32e-6                    # series sample time
ROWS, COLS = 32, 256          # patch: DM trials x series samples
F0, BW, FS = 326.5, 16.0, 32e6


CONV_C, CONV_K, NCLASS = 32, 7, 4   # the network's width, kernel length and classes (pond.h)


def init_params(seed: int) -> np.ndarray:
    """Seeded starting parameters in the flat layout of pond_cnn_create.

    Conv weights w[co][ci][k] uniform in +-sqrt(6 / fan_in) with fan_in =
    CONV_C * CONV_K (He et al. 2015, uniform form, for ReLU layers); conv
    biases zero; the final linear layer's weights uniform in
    +-0.5 sqrt(6 / CONV_C) and its biases zero.  The uniforms are the
    counter-based generator's words of stream 0 of ``seed``."""
    n_conv = CONV_C * CONV_C * CONV_K
    theta = np.zeros(pond.CNN_NPARAM, np.float64)
    u = synth.uniform(seed, 0, 0, pond.CNN_NPARAM)
    lim = math.sqrt(6.0 / (CONV_C * CONV_K))
    off = 0
    for _layer in range(3):
        theta[off:off + n_conv] = lim * (2.0 * u[off:off + n_conv] - 1.0)
        off += n_conv + CONV_C
    n_fc = NCLASS * CONV_C
    theta[off:off + n_fc] = 0.5 * math.sqrt(6.0 / CONV_C) * (2.0 * u[off:off + n_fc] - 1.0)
    assert off + n_fc + NCLASS == pond.CNN_NPARAM
    return theta.astype(np.float32)


def trial_grid(ndm: int = 128, dm_max: float = 60.0) -> list[float]:
    return [dm_max * d / (ndm - 1) for d in range(ndm)]


def make_engine(dms, nfft: int = 1 << 24, nchan: int = 64, device: int = 0) -> pond.Engine:
    return pond.Engine(F0, BW, FS, 0.0, nfft, nchan, 1, 1.0, t_dec=DT, dms=dms, device=device)


def chunk_patches(engine: pond.Engine, dms, x_dev, events, shifts_per_event: int, rng, stream=None):
    """Dedisperse one chunk and cut patches around its events.

    Returns (BF16 patches [P, 32, 256] on the device, labels [P], boxcar flags [P])."""
    import torch
    engine.reset()
    engine.push_tensor(x_dev, stream)
    engine.flush()
    cands = engine.candidates(6.0)
    T, _, j0 = engine.timeseries()
    ndm, n = T.shape
    ddm = dms[1] - dms[0]
    corners, labels = [], []
    for ev in events:
        dc = int(round(ev.dm / ddm))
        d0 = min(max(dc - ROWS // 2, 0), ndm - ROWS)
        tc = int(round(ev.t0 / DT)) - j0
        for _ in range(shifts_per_event):
            t0 = tc - COLS // 2 + int(rng.integers(-COLS // 4, COLS // 4 + 1))
            if t0 < 0 or t0 + COLS > n:
                continue
            corners.append((d0, t0))
            labels.append(ev.kind)
    if not corners:
        return None, np.zeros(0, np.int32), np.zeros(0, bool)
    cn = np.asarray(corners, np.int32)
    series = torch.from_numpy(np.ascontiguousarray(T, dtype=np.float32)).to(x_dev.device)
    X = pond.patches(series, torch.from_numpy(cn).to(x_dev.device))
    ct = np.array([[c["trial"], c["index"] - j0] for c in cands if c["trial"] > 0], np.int64).reshape(-1, 2)
    flags = np.zeros(len(cn), bool)
    for i, (d0, t0) in enumerate(cn):
        inside = ((ct[:, 0] >= d0) & (ct[:, 0] < d0 + ROWS) & (ct[:, 1] >= t0) & (ct[:, 1] < t0 + COLS))
        flags[i] = bool(inside.any())
    return X, np.asarray(labels, np.int32), flags


def build_dataset(n_chunks: int, seed: int, chunk_s: float = 8.0, ndm: int = 128, shifts: int = 4,
                  device=None):
    """Patches, labels and boxcar flags from n_chunks labelled chunks."""
    import torch
    device = device or torch.device("cuda", torch.cuda.current_device())
    dms = trial_grid(ndm)
    eng = make_engine(dms, device=device.index or 0)
    rng = np.random.default_rng(seed)
    Xs, Ys, Fs = [], [], []
    n_events = int((chunk_s - 0.55) / 0.3) + 1
    for c in range(n_chunks):
        spec = synth.StreamSpec(n=int(chunk_s * FS), seed=seed * 100003 + c, dm=0.0, period=0.0, snr=0.0)
        events = synth.draw_events(spec.seed, n_events, chunk_s, dm_max=dms[-1])
        x = synth.make_labelled_chunk_torch(spec, events, device)
        X, Y, F = chunk_patches(eng, dms, x, events, shifts, rng)
        if X is not None:
            Xs.append(X)
            Ys.append(Y)
            Fs.append(F)
        del x
    eng.close()
    return torch.cat(Xs), np.concatenate(Ys), np.concatenate(Fs)


def train(clf: pond.Classifier, X, Y: np.ndarray, epochs: int, batch: int, lr: float, seed: int):
    """Mini-batch Adam over shuffled patches; returns the mean loss of each epoch."""
    import torch
    rng = np.random.default_rng(seed)
    yt = torch.from_numpy(Y.astype(np.int32)).to(X.device)
    hist = []
    for ep in range(epochs):
        order = torch.from_numpy(rng.permutation(len(Y))).to(X.device)
        losses = []
        for s in range(0, len(Y) - batch + 1, batch):
            idx = order[s:s + batch]
            losses.append(clf.train_step(X[idx].contiguous(), yt[idx].contiguous(), lr, want_loss=True))
        hist.append(float(np.mean(losses)) if losses else float("nan"))
    return hist


def predict(clf: pond.Classifier, X, batch: int = 512) -> np.ndarray:
    batch = min(batch, clf.max_batch)
    out = []
    for s in range(0, X.shape[0], batch):
        out.append(clf.forward(X[s:s + batch].contiguous()).cpu().numpy())
    return np.concatenate(out)


def threshold_for_recall(prob: np.ndarray, Y: np.ndarray, recall: float) -> float:
    """The largest threshold on the pulse-class probability whose recall on
    (prob, Y) reaches `recall` (an operating point chosen on a validation set)."""
    p = np.sort(prob[Y == synth.EV_PULSE, synth.EV_PULSE])[::-1]
    if len(p) == 0:
        return 0.5
    k = min(len(p) - 1, max(0, int(np.ceil(recall * len(p))) - 1))
    return float(p[k])


def veto_threshold(prob: np.ndarray, Y: np.ndarray, flags: np.ndarray, max_recall_loss: float) -> float:
    """Operating point of the boxcar + network detector (a patch is flagged when
    the boxcar flags it and the network's pulse probability is >= tau): the
    largest tau whose recall on (prob, Y, flags) stays within max_recall_loss
    of the boxcar's own (chosen on a validation set)."""
    pos = Y == synth.EV_PULSE
    if not pos.any():
        return 0.0
    need = flags[pos].mean() - max_recall_loss
    p = np.sort(prob[pos & flags, synth.EV_PULSE])[::-1]   # pulse patches the boxcar flags
    k = int(np.ceil(need * pos.sum())) - 1
    if k < 0:
        return float(p[0]) if len(p) else 0.0
    return float(p[min(k, len(p) - 1)]) if len(p) else 0.0


def evaluate_veto(prob: np.ndarray, Y: np.ndarray, flags: np.ndarray, tau: float) -> dict:
    """Recall and false-positive rate of the boxcar alone and of the boxcar with
    the network's veto (flag and pulse probability >= tau)."""
    pos = Y == synth.EV_PULSE
    neg = ~pos
    both = flags & (prob[:, synth.EV_PULSE] >= tau)
    return {"tau": tau, "n_pulse": int(pos.sum()), "n_other": int(neg.sum()),
            "boxcar_recall": float(flags[pos].mean()), "boxcar_fpr": float(flags[neg].mean()),
            "boxcar_cnn_recall": float(both[pos].mean()), "boxcar_cnn_fpr": float(both[neg].mean())}


def evaluate(prob: np.ndarray, Y: np.ndarray, flags: np.ndarray, threshold: float | None = None) -> dict:
    """Recall on dispersed pulses and false-positive rate on the other classes,
    for the classifier (argmax = pulse, or pulse probability >= threshold) and
    for the boxcar flag."""
    if threshold is None:
        pred_pulse = prob.argmax(1) == synth.EV_PULSE
    else:
        pred_pulse = prob[:, synth.EV_PULSE] >= threshold
    pos = Y == synth.EV_PULSE
    neg = ~pos
    res = {"n_test": int(len(Y)), "n_pulse": int(pos.sum()),
           "cnn_recall": float(pred_pulse[pos].mean()) if pos.any() else None,
           "cnn_fpr": float(pred_pulse[neg].mean()) if neg.any() else None,
           "boxcar_recall": float(flags[pos].mean()) if pos.any() else None,
           "boxcar_fpr": float(flags[neg].mean()) if neg.any() else None,
           "cnn_accuracy_4class": float((prob.argmax(1) == Y).mean())}
    for k, name in ((synth.EV_BURST, "burst"), (synth.EV_NARROW, "narrowband"), (synth.EV_NOISE, "noise")):
        m = Y == k
        if m.any():
            res[f"cnn_fpr_{name}"] = float(pred_pulse[m].mean())
            res[f"boxcar_fpr_{name}"] = float(flags[m].mean())
    return res


def inference_rate(clf: pond.Classifier, X, batch: int = 512, reps: int = 20) -> float:
    """Patches classified per second (CUDA events around repeated batches)."""
    import torch
    batch = min(batch, clf.max_batch)
    xb = X[:batch].contiguous()
    if xb.shape[0] < batch:
        xb = xb.repeat((math.ceil(batch / xb.shape[0]), 1, 1))[:batch].contiguous()
    clf.forward(xb)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        clf.forward(xb)
    e1.record()
    torch.cuda.synchronize()
    return reps * batch / (e0.elapsed_time(e1) / 1e3)
