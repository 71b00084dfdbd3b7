"""The z pass skips grid rows that hold no share of the current push (rows
stamped by the deposit with the push counter): the fields equal those of a
process that reads every row (LC_ROW_STAMPS=0, read once per process), bit
for bit up to the sign of exact zeros.  No near split here, so that no FP64
atomic order differs between the processes."""
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = (
    "import sys, dataclasses, numpy as np, paper_1502_02294_gb300 as lc, synth\n"
    "name, steps = sys.argv[2], int(sys.argv[3])\n"
    "if name == 'c2':\n"
    "    w = synth.config('c2')\n"
    "elif name == 'cic64':\n"
    "    w = dataclasses.replace(synth.small(n=64, box=80.0, n_steps=steps, n_src=300, seed=5503, clustered=True),\n"
    "                            deposit=1)\n"
    "else:\n"
    "    w = synth.small(n=256, box=200.0, n_steps=steps, n_src=3000, seed=5507, clustered=True,\n"
    "                    history=lc.HISTORY_BF16)\n"
    "p = lc.Plan.from_workload(w, near_mode=lc.NEAR_NONE)\n"
    "outs = []\n"
    "for s in range(steps):\n"
    "    pos, lum = w.cat.active(s)\n"
    "    p.push(s, pos, lum)\n"
    "    outs.append(p.field(s, np.empty((w.n,) * 3, dtype=np.float32)))\n"
    "np.save(sys.argv[1], np.stack(outs))\n")


def _run(name, steps, stamps, d):
    env = dict(os.environ, PYTHONPATH=ROOT)
    if not stamps:
        env["LC_ROW_STAMPS"] = "0"
    if name.endswith("p4"):
        env["LC_FFT_VARIANT"] = "plane4"
    path = os.path.join(d, f"{name}_{int(stamps)}.npy")
    subprocess.run([sys.executable, "-c", CHILD, path, name, str(steps)], check=True, env=env, cwd=ROOT,
                   timeout=900)
    return np.load(path)


@pytest.mark.parametrize("name,steps", [("c2", 6), ("cic64", 5), ("bf16_256", 3), ("bf16_256p4", 3)])
def test_sparse_z_pass_equals_dense(name, steps):
    # c2: 128^3 plane kernels, FP32 history; 64^3 cloud in cell (up to four
    # rows a source); 256^3 BF16 history through the autotuned form and
    # through the four-CTA cluster plane kernels, which also clear the grid
    # rows they read
    with tempfile.TemporaryDirectory() as d:
        a = _run(name, steps, True, d)
        b = _run(name, steps, False, d)
    assert np.isfinite(a).all() and np.abs(a).max() > 0
    assert np.array_equal(a, b)
