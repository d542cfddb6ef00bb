"""The FP32 ceiling probe the benchmark's roofline divides by: its operation
count, a finite output per thread, and a measured rate in the plausible range
for this GPU (below the nominal FP32 ceiling of its SMs at their maximum clock,
above a quarter of it)."""
import numpy as np
import pytest

from paper_1503_01405_gb300 import pond

pytestmark = pytest.mark.gpu


def test_fp32_probe_counts_and_rate():
    import torch
    dev = torch.device("cuda", 0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, iters = 4 * sms, 4000
    out = torch.full((blocks * 512,), float("nan"), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    pond.probe_fp32_fma(out.data_ptr(), blocks, 10, stream.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fl = pond.probe_fp32_fma(out.data_ptr(), blocks, iters, stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    assert fl == 2.0 * blocks * 512 * iters * 16 * 8
    assert bool(torch.isfinite(out).all())
    tflops = fl / (e0.elapsed_time(e1) / 1e3) / 1e12
    nominal = sms * 128 * 2 * 2.07e9 / 1e12
    assert 0.25 * nominal < tflops < 1.05 * nominal, (tflops, nominal)


def test_fp32_probe_rejects_bad_arguments():
    import torch
    out = torch.zeros(512, dtype=torch.float32, device="cuda")
    with pytest.raises(pond.PondError) as ei:
        pond.probe_fp32_fma(out.data_ptr(), 0, 10)
    assert ei.value.name == "ARG"
    with pytest.raises(pond.PondError):
        pond.probe_fp32_fma(0, 1, 10)
    assert np.isfinite(out.cpu().numpy()).all()
