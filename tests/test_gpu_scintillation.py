"""GPU parity of the interplanetary scintillation mode (PONDER Sec. 3.5) against
the FP64 oracle, through the C ABI: the band-collapsed cross-power series (the
CID series at DM 0) and its accumulated fluctuation spectrum.  The halves share
a common component whose intensity is modulated at a known rate (a scintillating
source) over independent receiver noise.  Tolerance: relative L2 1e-5 over all
bins (the spectrum of an FP32 series from FP32 FFTs), and 1e-3 over the bins
above DC alone (their norm is a tenth to a fifth of the DC bin's in these cases,
so rounding that is small against DC may weigh more there); the modulation's
bin exactly."""
import numpy as np
import pytest

from oracle import incoherent as inc
from oracle import ips
from paper_1503_01405_gb300 import pond

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _halves(n, fmod_hz, seed):
    """N / S int8 pairs: g(t) w + n_N and g(t) w + n_S, g = 1 + 0.5 cos(2 pi fmod t)."""
    rng = np.random.default_rng(seed)
    t = np.arange(n) / 32e6
    w = rng.normal(0.0, 10.0, n) * (1.0 + 0.5 * np.cos(2 * np.pi * fmod_hz * t))
    q = lambda v: np.clip(np.rint(v), -127, 127).astype(np.int8)
    inter = np.empty(2 * n, np.int8)
    inter[0::2] = q(w + rng.normal(0.0, 10.0, n))
    inter[1::2] = q(w + rng.normal(0.0, 10.0, n))
    return inter


CASES = [  # nchan, nint, mode, L, input pairs, modulation Hz
    (256, 16, inc.CID, 256, 1 << 23, 46.0),
    (1024, 4, inc.CID, 64, (1 << 22) + 999, 120.0),
    (64, 64, inc.AID, 128, 1 << 22, 30.0),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"nch{c[0]}_nint{c[1]}_{'CID' if c[2] else 'AID'}_L{c[3]}")
def test_scintillation_spectrum_matches_oracle(case):
    import torch
    nchan, nint, mode, L, n, fmod = case
    p = inc.make_plan(326.5, 16.0, 32e6, 0.0, nchan, nint, mode, 2, 16, 0.5)
    raw = _halves(n, fmod, seed=21)
    r = inc.run(p, raw)
    A_ref, J_ref = ips.accumulated_spectrum(r.D, L)
    if mode == inc.CID:
        assert np.array_equal(ips.collapsed_series(p, raw), r.D)
    with pond.Incoherent(326.5, 16.0, 32e6, 0.0, nchan, nint, 16, 0.5, mode=mode, input_channels=2,
                         ips_len=L) as e:
        e.run_tensor(torch.from_numpy(raw).cuda())
        D, t_first = e.series()
        A, J = e.ips()
        info = e.info()
    assert t_first == 0 and len(D) == len(r.D) and rel(D, r.D) <= 1e-5
    assert J == J_ref == info["ips_chunks"] and J >= 4
    assert rel(A, A_ref) <= 1e-5
    assert rel(A[1:], A_ref[1:]) <= 1e-3
    f_mod = int(round(fmod * L * p.ts))
    assert int(np.argmax(A[1:])) + 1 == int(np.argmax(A_ref[1:])) + 1 == f_mod
    assert info["launches"] == 5


def test_scintillation_without_complete_chunk_and_state_errors():
    """Fewer series samples than one chunk: a zero spectrum and J = 0; a handle
    without ips_len refuses pond_incoh_ips."""
    import torch
    raw = _halves(1 << 20, 50.0, seed=3)
    with pond.Incoherent(326.5, 16.0, 32e6, 0.0, 256, 64, 16, 0.5, mode=pond.POND_INCOH_CID, input_channels=2,
                         ips_len=4096) as e:
        e.run_tensor(torch.from_numpy(raw).cuda())
        A, J = e.ips()
        assert J == 0 and not A.any() and A.shape == (2049,)
    with pond.Incoherent(326.5, 16.0, 32e6, 0.0, 256, 64, 16, 0.5, mode=pond.POND_INCOH_CID,
                         input_channels=2) as e:
        e.run_tensor(torch.from_numpy(raw).cuda())
        with pytest.raises(pond.PondError) as ei:
            e.ips()
        assert ei.value.name == "STATE"
