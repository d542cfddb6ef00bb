"""The classifier's CUDA kernels vs the FP64 oracle, through the C ABI.

The GPU network keeps BF16 weights and activations with FP32 accumulation; the
oracle runs in FP64 on the same BF16-rounded weights and inputs.  The BF16
rounding of the hidden activations bounds the agreement: relative L2 <= 2e-2
on gradients, <= 1e-2 on probabilities and the loss.
"""
import numpy as np
import pytest

from oracle import cnn
from paper_1503_01405_gb300 import pond, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1503_01405_gb300 import build as pbuild
    pbuild.build()


def bf16_round(a):
    import torch
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def gpu_weights_view(theta):
    """The parameters as the GPU uses them: BF16 weights, FP32 biases."""
    t = np.asarray(theta, np.float32).astype(np.float64)
    out = bf16_round(t)
    o = 0
    for _ in range(3):
        o += cnn.CONV
        out[o:o + cnn.C] = t[o:o + cnn.C]
        o += cnn.C
    out[-cnn.NCLS:] = t[-cnn.NCLS:]
    return out


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def setup(B, seed):
    import torch
    theta = cnn.init_params(synth.uniform(seed, 0, 0, cnn.n_params())).astype(np.float32)
    theta[cnn.CONV:cnn.CONV + 32] = 0.02
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((B, 32, 256)).astype(np.float32)
    x[:, 10:14, 100:120] += 3.0
    xt = torch.from_numpy(x).to(torch.bfloat16).cuda()
    y = rng.integers(0, 4, B).astype(np.int32)
    yt = torch.from_numpy(y).cuda()
    return theta, xt, y, yt


def test_forward_and_gradient_match_oracle():
    import torch
    theta, xt, y, yt = setup(6, 3)
    net = pond.Classifier(theta, max_batch=8)
    prob = net.forward(xt).cpu().numpy()
    loss, g = net.gradient(xt, yt)
    net.close()
    xo = xt.float().cpu().numpy().astype(np.float64)
    th = gpu_weights_view(theta)
    lo, go, po = cnn.backward(th, xo, y)
    assert np.max(np.abs(prob - po)) < 1e-2
    assert abs(loss - lo) < 1e-2 * abs(lo)
    assert rel(g, go) < 2e-2, rel(g, go)
    # every layer's block of the gradient agrees, not just the total
    o = 0
    for size in (cnn.CONV, 32, cnn.CONV, 32, cnn.CONV, 32, 128, 4):
        assert rel(g[o:o + size], go[o:o + size]) < 5e-2, (o, rel(g[o:o + size], go[o:o + size]))
        o += size


def test_adam_step_matches_oracle():
    theta, xt, y, yt = setup(4, 5)
    net = pond.Classifier(theta, max_batch=4)
    _, g = net.gradient(xt, yt)
    net.train_step(xt, yt, 1e-3)
    after = net.params()
    net.close()
    want, _, _ = cnn.adam_step(theta.astype(np.float64), 0, 0, g.astype(np.float64), 1, 1e-3)
    assert np.max(np.abs(after - want)) < 2e-6


def test_gradient_is_deterministic():
    theta, xt, y, yt = setup(8, 7)
    net = pond.Classifier(theta, max_batch=8)
    a = net.gradient(xt, yt)[1]
    b = net.gradient(xt, yt)[1]
    net.close()
    assert np.array_equal(a, b)


def test_patches_match_oracle():
    import torch
    rng = np.random.default_rng(9)
    block = (100 + 5 * rng.standard_normal((40, 3000))).astype(np.float32)
    corners = np.array([[0, 0], [8, 1000], [20, 2900], [-3, -10], [39, 5]], np.int32)
    out = pond.patches(torch.from_numpy(block).cuda(), torch.from_numpy(corners).cuda()).float().cpu().numpy()
    for p, (d0, t0) in enumerate(corners):
        want = cnn.patch(block, int(d0), int(t0))
        assert np.max(np.abs(out[p] - want)) < 2 ** -7 * np.max(np.abs(want))


def test_training_learns_a_separable_task():
    """Class = which of four row bands carries a bright box: loss must fall and
    training accuracy rise well above chance."""
    import torch
    rng = np.random.default_rng(11)
    B = 256
    y = rng.integers(0, 4, B).astype(np.int32)
    x = rng.standard_normal((B, 32, 256)).astype(np.float32)
    for i in range(B):
        t = rng.integers(20, 200)
        x[i, 8 * y[i]:8 * y[i] + 8, t:t + 30] += 2.0
    xt = torch.from_numpy(x).to(torch.bfloat16).cuda()
    yt = torch.from_numpy(y).cuda()
    theta = cnn.init_params(synth.uniform(13, 0, 0, cnn.n_params())).astype(np.float32)
    net = pond.Classifier(theta, max_batch=B)
    first = net.train_step(xt, yt, 3e-3, want_loss=True)
    for _ in range(150):
        last = net.train_step(xt, yt, 3e-3, want_loss=True)
    acc = float((net.forward(xt).argmax(1).cpu().numpy() == y).mean())
    net.close()
    assert last < 0.5 * first and acc > 0.9, (first, last, acc)


def oracle_prob(th, x):
    logits, _ = cnn.forward(th, x)
    z = np.exp(logits - logits.max(axis=1, keepdims=True))
    return z / z.sum(axis=1, keepdims=True)


@pytest.mark.parametrize("B", [1, 5, 333, 700])
def test_tensor_core_inference_matches_oracle(B):
    """pond_cnn_forward runs the convolutions as implicit GEMMs on the tensor
    cores (several samples per CTA when the batch exceeds two CTAs per SM):
    probabilities against the FP64 oracle on the same BF16 weights and inputs,
    for batches of one sample, a few, and more than the grid."""
    theta, xt, y, yt = setup(B, 7 + B)
    net = pond.Classifier(theta, max_batch=B)
    prob = net.forward(xt).cpu().numpy()
    net.close()
    xo = xt.float().cpu().numpy().astype(np.float64)
    th = gpu_weights_view(theta)
    po = np.concatenate([oracle_prob(th, xo[i:i + 1]) for i in range(0, B, max(1, B // 40))])
    pg = prob[::max(1, B // 40)]
    assert np.all(np.isfinite(prob)) and np.allclose(prob.sum(1), 1.0, atol=1e-5)
    assert np.max(np.abs(pg - po)) < 1e-2, np.max(np.abs(pg - po))


def test_tensor_core_inference_follows_training():
    """After Adam steps the inference kernel uses the updated weights: its
    probabilities agree with the oracle's forward of the trained parameters."""
    theta, xt, y, yt = setup(16, 21)
    net = pond.Classifier(theta, max_batch=16)
    for _ in range(5):
        net.train_step(xt, yt, 1e-2)
    th_new = net.params()
    prob = net.forward(xt).cpu().numpy()
    net.close()
    xo = xt.float().cpu().numpy().astype(np.float64)
    po = oracle_prob(gpu_weights_view(th_new), xo)
    assert np.max(np.abs(prob - po)) < 1e-2, np.max(np.abs(prob - po))
