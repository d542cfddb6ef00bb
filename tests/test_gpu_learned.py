"""The learned form end to end on a small scale: labelled chunks through the
batched engine, patches, training on the GPU, evaluation beside the boxcar,
and what the trained network gains over the boxcar detector alone."""
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


def test_scored_candidates_match_patches_and_forward():
    """pond_candidates_scored = the boxcar candidates, each scored by the network
    on its patch of the same series block: bit-identical to cutting the patches
    with pond_patches and running pond_cnn_forward separately."""
    import torch
    dev = torch.device("cuda", 0)
    dms = learn.trial_grid(48, 30.0)
    spec = synth.StreamSpec(n=int(3.0 * learn.FS), seed=77, dm=0.0, period=0.0, snr=0.0)
    events = [e for e in synth.draw_events(78, 8, 3.0, dm_max=dms[-1])]
    x = synth.make_labelled_chunk_torch(spec, events, dev)
    theta = cnn.init_params(synth.uniform(19, 0, 0, cnn.n_params())).astype(np.float32)
    clf = pond.Classifier(theta, max_batch=7)          # several batches
    with learn.make_engine(dms) as e:
        e.push_tensor(x)
        e.flush()
        scored = e.candidates(6.0, classifier=clf)
        plain = e.candidates(6.0)
        T, _, j0 = e.timeseries()
    assert len(scored) == len(plain) > 0
    for a, b in zip(scored, plain):
        assert (a["trial"], a["index"], a["width"], a["snr"]) == (b["trial"], b["index"], b["width"], b["snr"])
        assert b["score"] == -1.0 and 0.0 <= a["score"] <= 1.0
    ndm = T.shape[0]
    corners = np.array([[min(max(c["trial"] - 16, 0), max(ndm - 32, 0)), c["index"] - j0 - 128] for c in plain],
                       np.int32)
    series = torch.from_numpy(np.ascontiguousarray(T, dtype=np.float32)).to(dev)
    X = pond.patches(series, torch.from_numpy(corners).to(dev))
    prob = learn.predict(clf, X)
    clf.close()
    assert np.array_equal(np.array([c["score"] for c in scored], np.float32), prob[:, 0].astype(np.float32))


def test_network_veto_gains_over_boxcar():
    """What the trained network adds to the method without it.  The boxcar S/N >= 6
    detector flags narrowband RFI (a 2-sigma sinusoid integrated over ms widths
    reaches S/N 6 at every trial); the network, trained on the GPU by the
    library's kernels, vetoes the boxcar's flags whose pulse probability is
    below tau, with tau chosen on a validation set (disjoint seeds) as the
    largest that keeps the boxcar's validation recall.  On held-out chunks
    (disjoint seeds again) the combination keeps the boxcar's recall within
    0.03 and cuts its false-positive rate at least fourfold."""
    Xtr, Ytr, _ = learn.build_dataset(16, seed=1000, shifts=16)
    Xva, Yva, Fva = learn.build_dataset(4, seed=3000, shifts=16)
    Xte, Yte, Fte = learn.build_dataset(6, seed=2000, shifts=16)
    clf = pond.Classifier(learn.init_params(99), max_batch=512)
    learn.train(clf, Xtr, Ytr, epochs=15, batch=256, lr=2e-3, seed=3)
    tau = learn.veto_threshold(learn.predict(clf, Xva), Yva, Fva, 0.0)
    r = learn.evaluate_veto(learn.predict(clf, Xte), Yte, Fte, tau)
    clf.close()
    assert r["n_pulse"] > 300 and r["n_other"] > 1000, r
    assert r["boxcar_fpr"] > 0.03, r                  # the boxcar alone is fooled by RFI ...
    assert r["boxcar_cnn_recall"] >= r["boxcar_recall"] - 0.03, r
    assert r["boxcar_cnn_fpr"] <= 0.25 * r["boxcar_fpr"], r   # ... and the network removes most of it
