"""bench.py's command line on CPU: the reference arm (the oracle) runs the
workload variants and names them in its config, and keeps the JSON line's
contract keys."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*extra):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "c1",
                        "--steps", "1", "--warmup", "0", *extra], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_reference_arm_default_and_variants():
    base = _run()
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in base
    assert base["impl"] == "reference" and base["value"] > 0
    assert "radial_kernel" not in base["config"] and "near_field" not in base["config"]
    v = _run("--kernel", "exp", "--near", "subcell", "--fdiff")
    assert v["config"]["radial_kernel"].startswith("exp(")
    assert "sub-cell" in v["config"]["near_field"]
    assert "f_diff" in v["config"]["step_adds"]
    assert v["value"] > 0


def test_mac_source_hash_finds_the_kernel_texts():
    # the roofline's captured DRAM traffic is tied to a hash over the MAC
    # kernels' sources; the helper must find every function it hashes
    import sys

    sys.path.insert(0, ROOT)
    import bench

    h = bench.mac_sources_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    for name, t in bench.MAC_TRAFFIC.items():
        assert t["bytes"] > 0 and t["from"].startswith("profiles/")
        assert os.path.exists(os.path.join(ROOT, t["from"].split(" ")[0]))
    t = bench.MAC512_TRAFFIC
    assert t["bytes"] > t["algorithmic"] > 0 and os.path.exists(os.path.join(ROOT, t["from"]))
    # the captures belong to the kernels as they stand: a change to them
    # must come with new captures (and a new hash), else `traffic` goes null
    assert t["sources"] == h and all(x["sources"] == h for x in bench.MAC_TRAFFIC.values())
