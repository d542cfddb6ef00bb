"""The C ABI on a machine without a GPU: symbols, argument checks, error codes.

No compute call runs here; plan validation happens on the host before any
CUDA call, so bad plans return their code without a device.
"""
import ctypes
import os
import re

import pytest

from oracle import pcd
from paper_1503_01405_gb300 import build as pbuild
from paper_1503_01405_gb300 import pond

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    pbuild.build()


def _header_functions():
    src = open(os.path.join(ROOT, "include", "pond.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pond_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    names = _header_functions()
    assert len(names) >= 13
    L = pond.lib()
    for n in names:
        assert hasattr(L, n), n
    assert sorted(pond.EXPORTS) == names


def test_strerror_covers_codes():
    L = pond.lib()
    for code in range(0, -10, -1):
        assert L.pond_strerror(code)
    assert L.pond_strerror(-999) == b"unknown error"


ORT = dict(f0=326.5, bw=16.0, fs=32e6)
CASES = [
    dict(nfft=3000),
    dict(nfft=1 << 10, dm=3.0),
    dict(nchan=3),
    dict(nchan=1 << 12, nfft=1 << 12),
    dict(dm=-1.0),
    dict(period=0.0),
    dict(fs=31e6),
    dict(nbins=0),
    dict(bw=0.0),
]


@pytest.mark.parametrize("kw", CASES)
def test_plan_errors_match_oracle_rules(kw):
    args = dict(**ORT, dm=0.5, nfft=1 << 16, nchan=4, nbins=64, period=0.1)
    args.update(kw)
    with pytest.raises(pcd.PlanError) as oe:
        pcd.make_plan(**args)
    with pytest.raises(pond.PondError) as ce:
        pond.Engine(args["f0"], args["bw"], args["fs"], args["dm"], args["nfft"], args["nchan"],
                    args["nbins"], args["period"])
    assert ce.value.name == oe.value.code, (ce.value, oe.value)


def test_engine_limits():
    with pytest.raises(pond.PondError) as e:
        pond.Engine(326.5, 16.0, 32e6, 0.1, 1 << 16, 4, 5000, 0.1)
    assert e.value.name == "ARG"
    with pytest.raises(pond.PondError) as e:
        pond.Engine(326.5, 16.0, 32e6, 0.1, 1 << 16, 4, 64, 0.1, precision=7)
    assert e.value.name == "ARG"
    with pytest.raises(pond.PondError) as e:
        pond.Engine(326.5, 16.0, 32e6, 0.1, 1 << 16, 4, 64, 0.1, schedule=2)
    assert e.value.name == "ARG"


def test_null_handle_and_pointers():
    L = pond.lib()
    assert L.pond_flush(None) == pond.POND_E_ARG
    assert L.pond_destroy(None) == pond.POND_OK
    assert L.pond_plan_ex(None, None) == pond.POND_E_ARG
    h = ctypes.c_void_p()
    assert L.pond_plan_ex(ctypes.byref(h), None) == pond.POND_E_ARG
    assert h.value is None


def test_valid_plan_without_gpu_reports_cuda():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(pond.PondError) as e:
        pond.Engine(326.5, 16.0, 32e6, 0.1, 1 << 16, 4, 64, 0.1)
    assert e.value.name == "CUDA"


def test_batched_plan_validation():
    base = dict(f0=326.5, bw=16.0, fs=32e6, dm=0.0, nfft=1 << 16, nchan=4, nbins=1, period=1.0)
    with pytest.raises(pond.PondError) as e:
        pond.Engine(**base, dms=[0.1, -1.0])
    assert e.value.name == "ARG"
    with pytest.raises(pond.PondError) as e:
        pond.Engine(**base, dms=[0.1], want_voltages=True)
    assert e.value.name == "ARG"
    with pytest.raises(pond.PondError) as e:
        pond.Engine(**base, dms=[0.1], nfft_choices=(3000,), autotune=True)
    assert e.value.name == "NFFT"
    with pytest.raises(pond.PondError) as e:        # the fixed nfft cannot carry DM 30
        pond.Engine(**base, dms=[0.1, 30.0])
    assert e.value.name == "NFFT"
    for kw in (dict(trial_mode=5), dict(trial_mode=-1), dict(trials_per_launch=129), dict(trials_per_launch=-2),
               dict(inv_split=-1), dict(inv_split=13), dict(inv_split=1), dict(inv_split=8), dict(inv_split=12)):
        with pytest.raises(pond.PondError) as e:
            pond.Engine(**base, dms=[0.1, 0.2], **kw)
        assert e.value.name == "ARG", kw


def test_phase_model_errors():
    """A fold phase model is checked on the host: at most 8 finite coefficients,
    a finite reference time, single-DM plans only."""
    base = dict(f0=326.5, bw=16.0, fs=32e6, dm=0.1, nfft=1 << 16, nchan=4, nbins=64, period=0.1)
    for pm in ((0.0, [0.0] * 9), (float("nan"), [0.0, 10.0]), (0.0, [0.0, float("inf")])):
        with pytest.raises(pond.PondError) as e:
            pond.Engine(**base, phase_model=pm)
        assert e.value.name == "ARG", pm
    with pytest.raises(pond.PondError) as e:
        pond.Engine(326.5, 16.0, 32e6, 0.0, 1 << 16, 4, 1, 1.0, dms=[0.1, 0.2], phase_model=(0.0, [0.0, 10.0]))
    assert e.value.name == "ARG"


@pytest.mark.parametrize("nfft,nchan,bad", [(1 << 16, 4, (1, 8, 11)),      # M 2^13, R2 2^7: q in 2..7
                                            (1 << 21, 16, (3, 10)),        # M 2^16, R2 2^10: q in 4..9
                                            (1 << 24, 64, (4, 8))])        # M 2^17: q in 5..7 (nchan Q1 <= 8192)
def test_inverse_split_admissibility(nfft, nchan, bad):
    """Inverse splits outside the kernels' tile limits are refused on the host
    (single-DM four-pass plans here), before any CUDA call."""
    for q in bad:
        with pytest.raises(pond.PondError) as e:
            pond.Engine(326.5, 16.0, 32e6, 0.1, nfft, nchan, 64, 0.1, schedule=pond.POND_SCHEDULE_FOUR_PASS,
                        inv_split=q)
        assert e.value.name == "ARG", q


INCOH_CASES = [  # (options changed from a valid incoherent plan, expected code)
    (dict(mode=pond.POND_INCOH_CID, input_channels=1), "ARG"),
    (dict(input_channels=3), "ARG"),
    (dict(mode=2), "ARG"),
    (dict(nchan=32), "NCHAN"),
    (dict(nchan=4096), "NCHAN"),
    (dict(nchan=96), "NCHAN"),
    (dict(nint=3), "ARG"),
    (dict(nint=1 << 17), "ARG"),
    (dict(nbins=0), "ARG"),
    (dict(nbins=4097), "ARG"),
    (dict(dm=-1.0), "ARG"),
    (dict(period=0.0), "ARG"),
    (dict(fs=31e6), "ARG"),
    (dict(bw=0.0), "ARG"),
    (dict(ips_len=32), "ARG"),
    (dict(ips_len=8192), "ARG"),
    (dict(ips_len=100), "ARG"),
]


@pytest.mark.parametrize("kw,code", INCOH_CASES)
def test_incoherent_plan_errors(kw, code):
    """Incoherent-mode options are checked on the host before any CUDA call."""
    a = dict(f0=326.5, bw=16.0, fs=32e6, dm=1.0, nchan=1024, nint=1, nbins=64, period=0.5,
             mode=pond.POND_INCOH_AID, input_channels=1)
    a.update(kw)
    with pytest.raises(pond.PondError) as ei:
        pond.Incoherent(**a)
    assert ei.value.name == code


def test_incoherent_reserved_fields_rejected():
    o = pond.pond_incoh_opts()
    o.f0_mhz, o.bw_mhz, o.fs_hz, o.dm, o.period_s = 326.5, 16.0, 32e6, 1.0, 0.5
    o.nchan, o.nint, o.mode, o.input_channels, o.nbins = 1024, 1, 0, 1, 64
    o.reserved[2] = 1
    h = ctypes.c_void_p()
    assert pond.lib().pond_incoh_create(ctypes.byref(h), ctypes.byref(o)) == pond.POND_E_ARG
    assert pond.lib().pond_incoh_create(None, ctypes.byref(o)) == pond.POND_E_ARG
    assert pond.lib().pond_incoh_destroy(None) == pond.POND_OK


def test_stack_rows_match_the_oracle():
    """The host's row count and first rotation are the oracle's, bit for bit, for
    spin-down and cubic models, both row modes (pond_stack_rows needs no GPU)."""
    import numpy as np
    from oracle import stack as st
    y = np.zeros(200_001)
    for (t_ref, c), dt, g0 in (((0.0123, st.spin_model(0.7145, 4e-6, 0.0123, 0.3)[1]), 61.44e-6, 12345),
                               ((2.5, np.array([0.3, 7.0, -0.02, 1e-4])), 1e-4, 0),
                               ((-1.0, np.array([-5.2, 1.0 / 0.0331])), 4e-6, 777)):
        for mode, n_sub in ((st.ROTATION, 0), (st.SUBINT, 4097)):
            S, _, q0 = st.stack(y, g0, dt, c, t_ref, 64, mode, n_sub)
            rows, first = pond.stack_rows(len(y), g0, dt, c, t_ref, 64, mode, n_sub)
            assert rows == S.shape[0]
            assert first == q0


@pytest.mark.parametrize("kw", [dict(dt=0.0), dict(coef=[]), dict(coef=[0.0] * 9), dict(nbins=0),
                                dict(mode=1, n_sub=0), dict(mode=5), dict(n=-1), dict(coef=[float("nan"), 1.0])])
def test_stack_argument_errors(kw):
    a = dict(n=1000, g0=0, dt=1e-3, coef=[0.0, 2.0], t_ref=0.0, nbins=16, mode=0, n_sub=0)
    a.update(kw)
    with pytest.raises(pond.PondError) as ei:
        pond.stack_rows(**a)
    assert ei.value.name == "ARG"


def test_struct_layouts_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the C header's field offsets and
    size (a C program compiled against include/pond.h prints them)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"pond_opts": pond.pond_opts, "pond_meta": pond.pond_meta, "pond_cand": pond.pond_cand,
               "pond_stats_t": pond.pond_stats_t, "pond_incoh_opts": pond.pond_incoh_opts,
               "pond_incoh_info": pond.pond_incoh_info, "pond_lane_info": pond.pond_lane_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pond.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} . %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {(a, b): int(c) for a, b, c in (l.split() for l in out if l.strip())}
    for cname, cls in structs.items():
        assert got[(cname, ".")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)
