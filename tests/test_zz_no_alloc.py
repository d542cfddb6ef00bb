"""pond_fold_noalloc: folding for callers that cannot allocate device memory.

Some callers may not call cudaMalloc: a real-time acquisition thread that must
never stall (allocation and release can synchronise the whole device), or a
host application whose memory manager owns every device allocation.  They fold
detected power with pond_fold_noalloc, which uses a fixed device array as its
scratch instead of allocating.  Its profile, built over two calls in a row that
share that array, is checked against the FP64 oracle's fold of the same power
series (hits exactly, sums to the profile tolerance of the other GPU tests) and
against the engine's own fold (pond_push + pond_profile) of the same stream.
"""
import ctypes

import numpy as np
import pytest

from oracle import pcd
from paper_1503_01405_gb300 import pond, synth

pytestmark = pytest.mark.gpu

TOL_P = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1503_01405_gb300 import build as pbuild
    pbuild.build()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_noalloc_fold_matches_oracle_and_engine():
    import torch
    p = pcd.make_plan(326.5, 16.0, 32e6, 0.3, 1 << 16, 16, 128, 0.033)
    x = synth.make_stream(synth.StreamSpec(n=60 * p.S + 4321, seed=21, dm=p.dm, period=p.period,
                                           snr=60.0, duty=0.05))
    with pond.Engine(p.f0, p.bw, p.fs, p.dm, p.nfft, p.nchan, p.nbins, p.period, want_voltages=True) as e:
        e.push(x)
        e.flush()
        s_eng, h_eng, _ = e.profile()
        V, g0 = e.voltages()
    # detected power of the emitted channel samples, summed over sub-channels
    P = (V.real.astype(np.float64) ** 2 + V.imag.astype(np.float64) ** 2).sum(axis=0).astype(np.float32)
    s_ora, h_ora = pcd.fold(p, P.astype(np.float64), g0)
    dP = torch.from_numpy(P).cuda()
    d_sum = torch.zeros(p.nbins, dtype=torch.float64, device="cuda")
    d_hits = torch.zeros(p.nbins, dtype=torch.int64, device="cuda")
    L = pond.lib()
    stream = torch.cuda.current_stream().cuda_stream
    k = len(P) // 3
    for start, count in ((0, k), (k, len(P) - k)):          # two calls in a row, one scratch array
        rc = L.pond_fold_noalloc(dP.data_ptr() + 4 * start, count, g0 + start, p.dtc, p.period, p.nbins,
                                 d_sum.data_ptr(), d_hits.data_ptr(), stream)
        assert rc == pond.POND_OK, L.pond_last_error()
    torch.cuda.synchronize()
    s = d_sum.cpu().numpy()
    h = d_hits.cpu().numpy()
    assert np.array_equal(h, h_ora)
    assert rel(s, s_ora) <= TOL_P
    # the engine's fold of the same stream: same bins, same sums
    assert np.array_equal(h, h_eng)
    assert rel(s, s_eng) <= TOL_P
    # and the whole FP64 path from the int8 stream: the bins, and the profile within tolerance
    r = pcd.run(p, x)
    assert np.array_equal(h, r.prof_hits)
    assert rel(s, r.prof_sum) <= TOL_P


def test_noalloc_fold_rejects_too_many_bins():
    import torch
    L = pond.lib()
    d = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = L.pond_fold_noalloc(d.data_ptr(), 4, 0, 4e-6, 0.1, pond.POND_NOALLOC_MAX_NBINS + 1, d.data_ptr(),
                             d.data_ptr(), ctypes.c_void_p(None))
    assert rc == pond.POND_E_ARG
    assert b"exceeds the limit" in L.pond_last_error()
