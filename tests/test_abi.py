"""The C-ABI library loads and exports every entry point include/lc.h declares;
host-side argument checks answer without a GPU (no compute call is made)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1502_02294_gb300 as lc
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "lc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lc_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    lc.build()
    return lc._lib()


def test_every_declared_symbol_is_exported_and_bound(lib):
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    bound = {s[0] for s in lc.SIGNATURES}
    assert set(names) <= bound, set(names) - bound


def test_status_strings_and_argument_checks(lib):
    assert lib.lc_status_string(0) == b"ok"
    assert b"step" in lib.lc_status_string(3)
    st, keep = lc._steps_struct(synth.config("c1").steps)
    c = lc._Cosmology(0.31, 0.68)
    out = ctypes.c_void_p()
    # unsupported grid size and bad arguments are rejected before any device work
    assert lib.lc_plan_create(100, 100.0, ctypes.byref(c), ctypes.byref(st), None, ctypes.byref(out)) == 2
    assert lib.lc_plan_create(32, -1.0, ctypes.byref(c), ctypes.byref(st), None, ctypes.byref(out)) == 1
    bad = lc._Cosmology(0.0, 0.68)
    assert lib.lc_plan_create(32, 100.0, ctypes.byref(bad), ctypes.byref(st), None, ctypes.byref(out)) == 1
    assert lib.lc_push_sources(None, 0, 0, None, None) == 1
    assert lib.lc_retarded_field(None, 0, None) == 1
    assert lib.lc_plan_destroy(None) == 1
    st.subsamples = 3
    assert lib.lc_plan_create(32, 100.0, ctypes.byref(c), ctypes.byref(st), None, ctypes.byref(out)) == 1


def test_plan_estimate_is_host_only(lib):
    w = synth.config("c3")
    base, table = lc.estimate_bytes(w.n, w.steps, w.omega_m, w.h, history=lc.HISTORY_BF16)
    # 256^3 BF16 ring of 128 slots: 256*256*136*4 B * 128 ~ 4.6 GB
    assert 4.0e9 < base < 6.0e9
    assert 1.5e8 < table < 2.5e8  # one step's wedge table: 366145 * 128 * 4 B


def test_no_cpu_fallback_without_device(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    st, keep = lc._steps_struct(synth.config("c1").steps)
    c = lc._Cosmology(0.31, 0.68)
    out = ctypes.c_void_p()
    assert lib.lc_plan_create(32, 100.0, ctypes.byref(c), ctypes.byref(st), None, ctypes.byref(out)) == lc.LC_ERR_CUDA
    with pytest.raises(lc.LCError):
        lc.Plan.from_workload(synth.config("c1"))


def test_static_fft_wrapper_rejects_bad_arguments_before_the_library():
    import torch

    with pytest.raises(ValueError):
        lc.fft_r2c_static(torch.zeros((8, 8, 8)))  # not a CUDA tensor
    if torch.cuda.is_available():
        with pytest.raises(ValueError):
            lc.fft_r2c_static(torch.zeros((8, 8, 4), device="cuda"))  # not cubic
        with pytest.raises(ValueError):
            lc.fft_r2c_static(torch.zeros((8, 8, 8), device="cuda"),
                              out=torch.zeros((8, 8, 4), dtype=torch.complex64, device="cuda"))
        with pytest.raises(ValueError):
            lc.fft_r2c_static(torch.zeros((8, 8, 8), device="cuda"),
                              out=torch.zeros((8, 8, 5), dtype=torch.complex128, device="cuda"))


def test_step_options_are_checked_on_the_host(lib):
    c = lc._Cosmology(0.31, 0.68)
    out = ctypes.c_void_p()
    spec = synth.config("c1").steps

    def create(**kw):
        st, keep = lc._steps_struct(spec, **kw)
        return lib.lc_plan_create(32, 100.0, ctypes.byref(c), ctypes.byref(st), None, ctypes.byref(out))

    # the sub-cell near field is built on NGP cells; the rough horizon belongs to the LW kernel
    assert create(deposit=lc.DEPOSIT_CIC, near_mode=lc.NEAR_SUBCELL) == lc.LC_ERR_INVALID_ARG
    assert create(horizon_mode=lc.HORIZON_ROUGH, kernel=(lc.KERNEL_EXP, 30.0, 80.0)) == lc.LC_ERR_INVALID_ARG
    assert create(deposit=2) == lc.LC_ERR_INVALID_ARG
    assert create(horizon_mode=2) == lc.LC_ERR_INVALID_ARG
    assert create(n_shell_max=-1) == lc.LC_ERR_INVALID_ARG
    # the cap bounds the ring depth in the host-only estimate
    w = synth.config("c3")
    b_full, t_full = lc.estimate_bytes(w.n, w.steps, w.omega_m, w.h, history=lc.HISTORY_BF16)
    b_cap, t_cap = lc.estimate_bytes(w.n, w.steps, w.omega_m, w.h, history=lc.HISTORY_BF16, n_shell_max=16)
    assert b_cap < b_full / 4 and t_cap < t_full / 6
