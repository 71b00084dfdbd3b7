"""The innermost shell's near-field scatter on extra CTAs of the inverse plane
kernel (grids up to 192^3, and 256^3 with the four-CTA cluster plane kernels;
short lists) against its own launch: the same fields, one launch fewer per
field.  LC_NEAR_CTAS and LC_FFT_VARIANT are read once per process, so each
setting runs in a child process."""
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = (
    "import sys, numpy as np, paper_1502_02294_gb300 as lc, synth\n"
    "name, steps = sys.argv[2], int(sys.argv[3])\n"
    "if name == 'c2':\n"
    "    w = synth.config('c2')\n"
    "elif name == 'c2cic':\n"
    "    import dataclasses\n"
    "    w = dataclasses.replace(synth.config('c2'), deposit=1)\n"
    "elif name == 'g256p4':\n"
    "    w = synth.small(n=256, box=200.0, n_steps=steps, n_src=600, seed=4411, clustered=True)\n"
    "else:\n"
    "    w = synth.small(n=192, box=150.0, n_steps=steps, n_src=600, seed=4409, clustered=True)\n"
    "p = lc.Plan.from_workload(w)\n"
    "outs, launches = [], []\n"
    "for s in range(steps):\n"
    "    pos, lum = w.cat.active(s)\n"
    "    p.push(s, pos, lum)\n"
    "    k0 = lc.kernel_launches()\n"
    "    outs.append(p.field(s, np.empty((w.n,) * 3, dtype=np.float32)))\n"
    "    launches.append(lc.kernel_launches() - k0)\n"
    "np.savez(sys.argv[1], f=np.stack(outs), k=np.array(launches))\n")


def _run(name, steps, fuse, d):
    env = dict(os.environ, PYTHONPATH=ROOT)
    if not fuse:
        env["LC_NEAR_CTAS"] = "0"
    if name.endswith("p4"):
        env["LC_FFT_VARIANT"] = "plane4"
    path = os.path.join(d, f"{name}_{int(fuse)}.npz")
    subprocess.run([sys.executable, "-c", CHILD, path, name, str(steps)], check=True, env=env, cwd=ROOT,
                   timeout=900)
    r = np.load(path)
    return r["f"], r["k"]


@pytest.mark.parametrize("name,steps,fused", [("c2", 6, True), ("g192", 4, True), ("g256p4", 4, True),
                                              ("c2cic", 4, False)])
def test_near_on_plane_ctas_equals_own_launch(name, steps, fused):
    # c2: 142-418 sources a step at 128^3 (24 idle SMs); 192^3: the extra
    # CTAs follow the 40 planes of the second wave; 256^3 with the cluster
    # plane kernels: whole clusters after the plane CTAs; c2 with cloud in cell:
    # 8 entries a source, beyond the short-list bound, so both runs launch
    # the scatter on its own
    with tempfile.TemporaryDirectory() as d:
        fa, ka = _run(name, steps, True, d)
        fb, kb = _run(name, steps, False, d)
    assert np.isfinite(fa).all() and np.abs(fa).max() > 0
    # the FP64 sums of a cell may be added in another order: the folded
    # values agree to FP32 rounding
    for s in range(steps):
        ref = fb[s]
        assert np.allclose(fa[s], ref, rtol=2.5e-7, atol=1e-7 * np.abs(ref).max()), s
    if fused:
        assert (ka == kb - 1).all(), (ka, kb)
    else:
        assert (ka == kb).all(), (ka, kb)
