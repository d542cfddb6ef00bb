"""GPU parity of the phase-model fold and pulse stacks (PONDER Sec. 3.4 fold with a
predicted period, Sec. 4 single-pulse stack) against the FP64 oracle, through the
C ABI.  Phases, rotations and bins are decided with the same FP64 operations on
both sides and every cell adds its samples in sample order, so sums and hits are
compared bit for bit."""
import numpy as np
import pytest

from oracle import stack as st
from paper_1503_01405_gb300 import pond

pytestmark = pytest.mark.gpu

MODELS = [  # (t_ref, coefficients), dt, g0, nbins
    (st.spin_model(0.7145, 4e-6, 0.0123, 0.3), 61.44e-6, 12345, 256),
    ((2.5, np.array([0.3, 7.0, -0.02, 1e-4])), 1e-4, 0, 64),
    (st.spin_model(0.0331, 0.0, 0.0, 0.0), 4e-6, 777, 1024),
]


@pytest.mark.parametrize("model", MODELS, ids=["spin_down", "cubic", "crab_like"])
@pytest.mark.parametrize("mode,n_sub", [(st.ROTATION, 0), (st.SUBINT, 9973), (st.SUBINT, 1 << 22)],
                         ids=["rotation", "subint", "one_subint"])
def test_stack_matches_oracle_bit_for_bit(model, mode, n_sub):
    import torch
    (t_ref, c), dt, g0, nbins = model
    y = np.random.default_rng(7).normal(10.0, 3.0, 300_001).astype(np.float32)
    S_ref, H_ref, q0_ref = st.stack(y, g0, dt, c, t_ref, nbins, mode, n_sub)
    S, H, q0 = pond.fold_stack(torch.from_numpy(y).cuda(), g0, dt, c, t_ref, nbins, mode, n_sub)
    assert q0 == q0_ref and S.shape == S_ref.shape
    assert np.array_equal(H, H_ref)
    assert np.array_equal(S, S_ref)


def test_stack_errors_and_empty_series():
    import torch
    y = torch.ones(1000, dtype=torch.float32, device="cuda")
    with pytest.raises(pond.PondError) as ei:           # phase running backwards
        pond.fold_stack(y, 0, 1e-3, [0.0, 5.0, -10.0], 0.0, 16)
    assert ei.value.name == "ARG"
    S, H, _ = pond.fold_stack(y[:0], 0, 1e-3, [0.0, 5.0], 0.0, 16)
    assert S.shape == (0, 16) and H.shape == (0, 16)
    import ctypes
    rows, q0 = ctypes.c_int64(), ctypes.c_int64()
    c = np.array([0.0, 5.0])
    rc = pond.lib().pond_fold_stack(y.data_ptr(), 1000, 0, 1e-3, c.ctypes.data, 2, 0.0, 16, 0, 0, None, None, 2,
                                    ctypes.byref(rows), ctypes.byref(q0), None)
    assert rc == pond.POND_E_OVERRUN and rows.value == 5
