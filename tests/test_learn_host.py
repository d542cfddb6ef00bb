"""Host-side pieces of the learned form that need no GPU: the package's own
seeded parameter initialiser (the layout of pond_cnn_create) and the outcome
counting of the evaluation."""
import math

import numpy as np

from oracle import cnn
from paper_1503_01405_gb300 import learn, pond, synth


def test_init_params_layout_and_bounds():
    th = learn.init_params(7)
    assert th.dtype == np.float32 and th.size == pond.CNN_NPARAM == cnn.n_params()
    layers, fw, fb = cnn.unpack(th)
    lim = math.sqrt(6.0 / (32 * 7))
    for w, b in layers:
        assert w.shape == (32, 32, 7) and not b.any()
        assert np.abs(w).max() <= lim and np.abs(w).max() > 0.9 * lim
        assert abs(float(w.mean())) < 0.02 * lim          # 7168 uniforms: mean near zero
    assert fw.shape == (4, 32) and not fb.any() and np.abs(fw).max() <= 0.5 * math.sqrt(6.0 / 32)
    # the same draw as the oracle's initialiser given the same uniforms (stream 0 of the seed)
    ref = cnn.init_params(synth.uniform(7, 0, 0, cnn.n_params())).astype(np.float32)
    assert np.array_equal(th, ref)
    assert not np.array_equal(th, learn.init_params(8))


def test_evaluate_counts_outcomes():
    Y = np.array([synth.EV_PULSE, synth.EV_PULSE, synth.EV_BURST, synth.EV_NOISE, synth.EV_NARROW])
    prob = np.zeros((5, 4))
    prob[[0, 2, 3, 4], [0, 0, 3, 2]] = 1.0      # pulse, missed pulse, burst called pulse, noise, narrowband
    prob[1, 3] = 1.0
    flags = np.array([True, True, False, False, True])
    r = learn.evaluate(prob, Y, flags)
    assert r["cnn_recall"] == 0.5 and math.isclose(r["cnn_fpr"], 1 / 3)
    assert r["boxcar_recall"] == 1.0 and math.isclose(r["boxcar_fpr"], 1 / 3)
    assert r["cnn_fpr_burst"] == 1.0 and r["boxcar_fpr_narrowband"] == 1.0
