"""Checkpoint / resume of a plan's history: a plan restored from a checkpoint
continues with the same fields as the plan it was taken from, and both match
the FP64 oracle; mismatched or truncated checkpoints are refused."""
import numpy as np
import pytest

import oracle
import paper_1502_02294_gb300 as lc
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    lc.build()
    oracle.build()


def _push(plan, cat, s):
    pos, lum = cat.active(s)
    plan.push(s, torch.from_numpy(pos).cuda(), torch.from_numpy(lum).cuda())


def _close_ulps(a, b, k=2.0):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    ulp = np.exp2(np.floor(np.log2(np.maximum(np.abs(b), np.finfo(np.float32).tiny))) - 23)
    return bool(np.all(np.abs(a - b) <= k * ulp))


@pytest.mark.parametrize("history", [synth.HISTORY_FP32, synth.HISTORY_BF16])
@pytest.mark.parametrize("device_buf", [False, True])
def test_resume_continues_identically(history, device_buf):
    w = synth.small(n=32, box=60.0, n_steps=10, n_src=150, seed=31, clustered=True, history=history)
    a = lc.Plan.from_workload(w)
    for s in range(5):
        _push(a, w.cat, s)
        a.field(s)
    n = a.checkpoint_bytes()
    buf = torch.empty(n, dtype=torch.uint8, device="cuda") if device_buf else None
    buf = a.save(buf)
    b = lc.Plan.from_workload(w)
    b.load(buf)
    P = oracle.Problem.from_workload(w)
    for s in range(5, 10):
        _push(a, w.cat, s)
        _push(b, w.cat, s)
        ja = a.field(s).cpu().numpy()
        jb = b.field(s).cpu().numpy()
        assert _close_ulps(jb, ja), s
        if s == 9:
            ref = oracle.field_for(P, w.cat, s)
            rel = np.linalg.norm(jb - ref) / np.linalg.norm(ref)
            assert rel <= (1e-5 if history == synth.HISTORY_FP32 else 5e-3), rel
    a.close()
    b.close()


def test_checkpoint_between_push_and_field():
    # the innermost slice's near-field list travels with the checkpoint
    w = synth.small(n=32, box=60.0, n_steps=6, n_src=150, seed=32, clustered=True)
    a = lc.Plan.from_workload(w)
    for s in range(4):
        _push(a, w.cat, s)
    buf = a.save()
    b = lc.Plan.from_workload(w)
    b.load(buf)
    ja = a.field(3).cpu().numpy()
    jb = b.field(3).cpu().numpy()
    assert _close_ulps(jb, ja)
    with pytest.raises(lc.LCError):
        _push(b, w.cat, 3)  # steps stay ordered after a restore
    a.close()
    b.close()


def test_mismatched_and_truncated_checkpoints_refused():
    w = synth.small(n=32, box=60.0, n_steps=6, n_src=100, seed=33)
    a = lc.Plan.from_workload(w)
    for s in range(3):
        _push(a, w.cat, s)
    buf = a.save()
    other_box = lc.Plan.from_workload(w, box=61.0)
    with pytest.raises(lc.LCError):
        other_box.load(buf)
    other_unit = lc.Plan.from_workload(w, out_unit=2.0)
    with pytest.raises(lc.LCError):
        other_unit.load(buf)
    same = lc.Plan.from_workload(w)
    with pytest.raises(lc.LCError):
        same.load(buf[: buf.size - 1])
    bad = buf.copy()
    bad[0] ^= 0xFF
    with pytest.raises(lc.LCError):
        same.load(bad)
    # a refused load leaves the plan usable from its own state
    _push(same, w.cat, 0)
    same.field(0)
    with pytest.raises(lc.LCError):
        a.save(np.empty(16, dtype=np.uint8))
    for p in (a, other_box, other_unit, same):
        p.close()
