"""The learned form end to end on a small scale: labelled chunks through the
batched engine, patches, training on the GPU, evaluation beside the boxcar."""
import numpy as np
import pytest

from oracle import cnn
from paper_1503_01405_gb300 import learn, pond, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1503_01405_gb300 import build as pbuild
    pbuild.build()


def test_events_and_labels():
    ev = synth.draw_events(3, 20, 8.0)
    assert len(ev) == 20 and all(0.25 <= e.t0 <= 7.75 for e in ev)
    assert {e.kind for e in ev} <= {0, 1, 2, 3}
    assert all(e.dm == 0.0 for e in ev if e.kind == synth.EV_BURST)


def test_learned_pipeline_small():
    X, Y, F = learn.build_dataset(n_chunks=3, seed=5, chunk_s=3.0, shifts=4)
    assert X.shape[1:] == (32, 256) and len(Y) == X.shape[0] == len(F)
    # patches are normalised: zero mean, unit standard deviation
    xf = X.float()
    assert abs(float(xf.mean())) < 0.02 and abs(float(xf.std()) - 1) < 0.02
    # the boxcar finds most bright dispersed pulses in their patches
    assert F[Y == synth.EV_PULSE].mean() > 0.5
    theta = cnn.init_params(synth.uniform(17, 0, 0, cnn.n_params())).astype(np.float32)
    clf = pond.Classifier(theta, max_batch=64)
    hist = learn.train(clf, X, Y, epochs=15, batch=32, lr=2e-3, seed=1)
    prob = learn.predict(clf, X)
    res = learn.evaluate(prob, Y, F)
    clf.close()
    assert hist[-1] < hist[0]
    assert res["cnn_accuracy_4class"] > 0.5, res
