"""A plain C caller compiled against include/lc.h and linked to liblc.so: the
struct layouts the header defines (lc_steps, lc_cosmology, lc_plan_info_t)
agree field by field with the ones the Python binding declares, and a
host-only call (lc_plan_estimate) gives the same answer from C as through the
binding, so every field of lc_steps reaches the library where the header puts
it.  No GPU is used."""
import ctypes
import os
import shutil
import subprocess

import pytest

import paper_1502_02294_gb300 as lc
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SRC = r"""
#include <stddef.h>
#include <stdio.h>
#include <string.h>
#include "lc.h"

#define OFF(T, f) printf("%s.%s %zu\n", #T, #f, offsetof(T, f))

int main(void) {
    printf("sizeof.lc_steps %zu\n", sizeof(lc_steps));
    printf("sizeof.lc_cosmology %zu\n", sizeof(lc_cosmology));
    printf("sizeof.lc_plan_info_t %zu\n", sizeof(lc_plan_info_t));
    OFF(lc_steps, n_steps); OFF(lc_steps, spacing); OFF(lc_steps, z_edges); OFF(lc_steps, z_start);
    OFF(lc_steps, z_end); OFF(lc_steps, n_shell); OFF(lc_steps, subsamples); OFF(lc_steps, history);
    OFF(lc_steps, normalise); OFF(lc_steps, out_unit); OFF(lc_steps, kernel); OFF(lc_steps, kernel_length);
    OFF(lc_steps, kernel_rmax); OFF(lc_steps, near_mode); OFF(lc_steps, deposit); OFF(lc_steps, horizon_mode);
    OFF(lc_steps, n_shell_max);
    OFF(lc_cosmology, omega_m); OFF(lc_cosmology, h);
    OFF(lc_plan_info_t, n); OFF(lc_plan_info_t, n_steps); OFF(lc_plan_info_t, n_ring);
    OFF(lc_plan_info_t, history); OFF(lc_plan_info_t, wedge_size); OFF(lc_plan_info_t, spectrum_row);
    OFF(lc_plan_info_t, box_mpc); OFF(lc_plan_info_t, z_edges);

    lc_steps st;
    memset(&st, 0, sizeof st);
    st.n_steps = 24;
    st.spacing = LC_STEPS_EQUAL_TIME;
    st.z_start = 20.0;
    st.z_end = 15.0;
    st.subsamples = 4;
    st.history = LC_HISTORY_BF16;
    st.normalise = 1;
    st.out_unit = 1.0;
    st.kernel = LC_KERNEL_LW;
    st.near_mode = LC_NEAR_NGP;
    st.deposit = LC_DEPOSIT_CIC;
    st.horizon_mode = LC_HORIZON_ROUGH;
    st.n_shell_max = 3;
    lc_cosmology c = {0.31, 0.68};
    size_t b = 0, t = 0;
    lc_status s = lc_plan_estimate(64, &st, &c, &b, &t);
    printf("estimate %d %zu %zu\n", (int)s, b, t);
    st.n_shell_max = 0;
    s = lc_plan_estimate(64, &st, &c, &b, &t);
    printf("estimate_nocap %d %zu %zu\n", (int)s, b, t);
    st.deposit = 7;
    s = lc_plan_estimate(64, &st, &c, &b, &t);
    printf("bad_deposit %d\n", (int)s);
    st.deposit = LC_DEPOSIT_NGP;
    st.horizon_mode = 9;
    s = lc_plan_estimate(64, &st, &c, &b, &t);
    printf("bad_horizon %d\n", (int)s);
    printf("status %s\n", lc_status_string(LC_ERR_INVALID_ARG));
    return 0;
}
"""


@pytest.fixture(scope="module")
def c_output(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lc.build()
    d = tmp_path_factory.mktemp("abi_c")
    src = d / "caller.c"
    src.write_text(C_SRC)
    exe = d / "caller"
    libdir = os.path.dirname(os.path.abspath(lc.__file__))
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", libdir, "-llc", "-Wl,-rpath," + libdir], check=True, capture_output=True)
    r = subprocess.run([str(exe)], check=True, capture_output=True, text=True)
    out = {}
    for line in r.stdout.splitlines():
        k, v = line.split(" ", 1)
        out[k] = v
    return out


@pytest.mark.parametrize("cname,pyclass", [("lc_steps", lc._Steps), ("lc_cosmology", lc._Cosmology),
                                           ("lc_plan_info_t", lc._Info)])
def test_struct_layout_matches_binding(c_output, cname, pyclass):
    assert int(c_output["sizeof." + cname]) == ctypes.sizeof(pyclass)
    for name, _ in pyclass._fields_:
        assert int(c_output[cname + "." + name]) == getattr(pyclass, name).offset, name


def test_host_call_from_c_equals_binding(c_output):
    spec = synth.StepSpec(synth.STEPS_EQUAL_TIME, 24, z_start=20.0, z_end=15.0)
    lib = lc._lib()
    cos = lc._Cosmology(0.31, 0.68)
    for key, cap in (("estimate", 3), ("estimate_nocap", 0)):
        st, keep = lc._steps_struct(spec, 4, lc.HISTORY_BF16, 1, 1.0, None, lc.NEAR_NGP, lc.DEPOSIT_CIC,
                                    lc.HORIZON_ROUGH, cap)
        b, t = ctypes.c_size_t(), ctypes.c_size_t()
        rc = lib.lc_plan_estimate(64, ctypes.byref(st), ctypes.byref(cos), ctypes.byref(b), ctypes.byref(t))
        assert c_output[key].split() == [str(rc), str(b.value), str(t.value)]
        assert rc == 0 and b.value > 0 and t.value > 0
    # the cap shrinks the ring and the per-step table
    capped = [int(x) for x in c_output["estimate"].split()[1:]]
    free = [int(x) for x in c_output["estimate_nocap"].split()[1:]]
    assert capped[0] < free[0] and capped[1] < free[1]
    assert int(c_output["bad_deposit"]) == 1 and int(c_output["bad_horizon"]) == 1
    assert c_output["status"] == lib.lc_status_string(1).decode()
