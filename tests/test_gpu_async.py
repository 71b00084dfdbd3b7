"""Asynchronous host output: lc_retarded_field_async returns once the field
and its device-to-host copy are enqueued, the copy overlapping the next
steps; lc_plan_wait makes the output readable.  Fields equal the waiting
call's, with pinned and pageable host buffers, across stage reuse."""
import time

import numpy as np
import pytest

import paper_1502_02294_gb300 as lc
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    lc.build()


def test_async_outputs_equal_waiting_outputs():
    w = synth.small(n=32, box=60.0, n_steps=8, n_src=150, seed=2718, clustered=True)
    a = lc.Plan.from_workload(w)
    b = lc.Plan.from_workload(w)
    want = []
    pinned = [torch.empty((w.n,) * 3, dtype=torch.float32).pin_memory() for _ in range(3)]
    tickets = []
    for s in range(8):
        pos, lum = w.cat.active(s)
        a.push(s, pos, lum)
        want.append(a.field(s, np.empty((w.n,) * 3, dtype=np.float32)))
        b.push(s, pos, lum)
        tickets.append(b.field_async(s, pinned[s % 3]))
        assert tickets[-1] == s + 1
        if s >= 1:  # the previous step's copy, while this one computes
            b.wait(tickets[s - 1])
            got = pinned[(s - 1) % 3].numpy()
            assert np.allclose(got, want[s - 1], rtol=1e-6, atol=1e-6 * np.abs(want[s - 1]).max()), s - 1
    b.wait(tickets[-1])
    assert np.allclose(pinned[7 % 3].numpy(), want[7], rtol=1e-6, atol=1e-6 * np.abs(want[7]).max())
    b.wait(tickets[0])  # an old ticket returns at once
    with pytest.raises(lc.LCError):
        b.wait(tickets[-1] + 5)  # never issued
    a.close()
    b.close()


def test_async_pageable_and_device_outputs():
    w = synth.small(n=16, box=40.0, n_steps=4, n_src=60, seed=2719)
    p = lc.Plan.from_workload(w)
    ref = lc.Plan.from_workload(w)
    for s in range(4):
        pos, lum = w.cat.active(s)
        p.push(s, pos, lum)
        ref.push(s, pos, lum)
        want = ref.field(s).cpu().numpy()
        host = np.empty((w.n,) * 3, dtype=np.float32)  # pageable
        t = p.field_async(s, host)
        p.wait(t)
        assert np.allclose(host, want, rtol=1e-6, atol=1e-6 * np.abs(want).max())
    dev = torch.empty((w.n,) * 3, dtype=torch.float32, device="cuda")
    assert p.field_async(3, dev) == 0  # a device output is stream-ordered
    p.wait(0)
    assert np.allclose(dev.cpu().numpy(), want, rtol=1e-6, atol=1e-6 * np.abs(want).max())
    p.close()
    ref.close()


def test_waiting_field_into_page_locked_host_memory():
    # a page-locked output is written by the SMs through its device view
    w = synth.small(n=32, box=60.0, n_steps=4, n_src=100, seed=2720)
    a = lc.Plan.from_workload(w)
    b = lc.Plan.from_workload(w)
    pinned = torch.empty((w.n,) * 3, dtype=torch.float32).pin_memory()
    for s in range(4):
        pos, lum = w.cat.active(s)
        a.push(s, pos, lum)
        b.push(s, pos, lum)
        want = a.field(s).cpu().numpy()
        b.field(s, pinned)
        assert np.array_equal(pinned.numpy(), want), s
    a.close()
    b.close()


def test_page_locked_host_inputs():
    # page-locked sources give the fields of device inputs, and bad values
    # still fail on the host
    w = synth.small(n=32, box=60.0, n_steps=4, n_src=120, seed=2721, clustered=True)
    a = lc.Plan.from_workload(w)
    b = lc.Plan.from_workload(w)
    for s in range(4):
        pos, lum = w.cat.active(s)
        a.push(s, torch.from_numpy(pos).cuda(), torch.from_numpy(lum).cuda())
        pp, lp = torch.from_numpy(pos).pin_memory(), torch.from_numpy(lum).pin_memory()
        b.push(s, pp, lp)
        assert np.array_equal(b.field(s).cpu().numpy(), a.field(s).cpu().numpy()), s
    bad = torch.from_numpy(w.cat.active(3)[1].copy()).pin_memory()
    if bad.numel():
        bad[0] = -1.0
        b.reset()
        with pytest.raises(lc.LCError) as e:
            b.push(0, torch.from_numpy(w.cat.active(3)[0]).pin_memory(), bad)
        assert e.value.status == lc.LC_ERR_INVALID_ARG
    a.close()
    b.close()


def test_poll_completes_each_ticket_in_order_over_many_tickets():
    # more tickets than the stages and than the per-ticket event ring: each
    # ticket reports done once its own copy has finished, completions are
    # monotone in ticket order, and every output equals the waiting call's
    w = synth.small(n=64, box=90.0, n_steps=24, n_src=200, seed=2720, clustered=True)
    a = lc.Plan.from_workload(w)
    b = lc.Plan.from_workload(w)
    nbuf = 5
    pinned = [torch.empty((w.n,) * 3, dtype=torch.float32).pin_memory() for _ in range(nbuf)]
    tickets, want = [], []
    for s in range(24):
        pos, lum = w.cat.active(s)
        a.push(s, pos, lum)
        want.append(a.field(s, np.empty((w.n,) * 3, dtype=np.float32)))
        if s >= nbuf:  # the buffer is free again once its ticket is done
            t_end = time.monotonic() + 60.0
            while not b.poll(tickets[s - nbuf]):
                assert time.monotonic() < t_end, "ticket never completed"
            got = pinned[(s - nbuf) % nbuf].numpy()
            ref = want[s - nbuf]
            assert np.allclose(got, ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max()), s - nbuf
        b.push(s, pos, lum)
        tickets.append(b.field_async(s, pinned[s % nbuf]))
        # newest first: a ticket seen done implies every earlier ticket done
        done = [b.poll(t) for t in reversed(tickets)][::-1]
        assert all(done[i] or not done[i + 1] for i in range(len(done) - 1)), done
    b.wait(tickets[-1])
    assert all(b.poll(t) for t in tickets)
    for s in range(24 - nbuf, 24):
        ref = want[s]
        assert np.allclose(pinned[s % nbuf].numpy(), ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max()), s
    a.close()
    b.close()


def test_copy_engine_path_equals_copy_kernel_path():
    # page-locked outputs go through a small copy kernel by default and
    # through the copy engine with LC_D2H=ce (read once per process): a
    # child process with each setting gives the same bytes (no near split,
    # whose FP64 atomics may sum in another order in another process)
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import sys, numpy as np, torch, paper_1502_02294_gb300 as lc, synth\n"
        "w = synth.small(n=32, box=60.0, n_steps=6, n_src=120, seed=2721, clustered=True)\n"
        "p = lc.Plan.from_workload(w, near_mode=lc.NEAR_NONE)\n"
        "outs = [torch.empty((32,) * 3, dtype=torch.float32).pin_memory() for _ in range(6)]\n"
        "ts = []\n"
        "for s in range(6):\n"
        "    pos, lum = w.cat.active(s)\n"
        "    p.push(s, pos, lum)\n"
        "    ts.append(p.field_async(s, outs[s]))\n"
        "p.wait(ts[-1])\n"
        "np.save(sys.argv[1], np.stack([o.numpy() for o in outs]))\n")
    import tempfile

    res = {}
    with tempfile.TemporaryDirectory() as d:
        for mode in ("sm", "ce"):
            env = dict(os.environ, LC_D2H=mode, PYTHONPATH=root)
            path = os.path.join(d, f"{mode}.npy")
            subprocess.run([sys.executable, "-c", code, path], check=True, env=env, cwd=root, timeout=600)
            res[mode] = np.load(path)
    assert np.isfinite(res["sm"]).all() and np.abs(res["sm"]).max() > 0
    assert np.array_equal(res["sm"], res["ce"])
