"""Host-side scheduling logic of the continuous-batching server, on the CPU
with a stand-in plan and a stand-in of the few torch calls it makes:
requests of one simulation run in step order whatever their arrival order;
at most `slots` requests of a simulation are in flight, and a slot (with its
page-locked source buffers) is reused only after its request completed;
latency is split into the wait for admission and the rest; rewind() serves
the same steps again from a refilled history."""
import contextlib
import types

import numpy as np

import paper_1502_02294_gb300.serve as sv


class _Event:
    """Completes after `after` queries (0: at once)."""
    after = 0

    def __init__(self, enable_timing=False):
        self.left = _Event.after

    def record(self, s):
        pass

    def query(self):
        if self.left > 0:
            self.left -= 1
            return False
        return True

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return 2.0


class _Stream:
    cuda_stream = 0

    def __init__(self, priority=0):
        self.priority = priority

    def synchronize(self):
        pass

    def wait_event(self, e):
        pass

    @staticmethod
    def priority_range():
        return (0, -5)


class _Tensor:
    def __init__(self, a):
        self.a = a

    def pin_memory(self):
        return self

    @property
    def shape(self):
        return self.a.shape

    def __getitem__(self, k):
        return _Tensor(self.a[k])

    def numpy(self):
        return self.a


class _Torch:
    float32, float64 = np.float32, np.float64

    class cuda:
        Event = _Event
        Stream = _Stream

        @staticmethod
        def stream(s):
            return contextlib.nullcontext()

        @staticmethod
        def current_stream():
            return _Stream()

        @staticmethod
        def synchronize():
            pass

    @staticmethod
    def empty(shape, dtype=None, device=None):
        return _Tensor(np.zeros(shape, dtype=dtype or np.float32))


class _Plan:
    def __init__(self, log):
        self.log = log
        self.pushed = []

    def push(self, s, p, l):
        self.log.append(s)
        self.pushed.append((s, p.numpy().copy(), l.numpy().copy()))

    def field(self, s, o):
        pass

    def field_async(self, s, o):
        return s + 1

    def poll(self, t):
        return True

    def reset(self):
        self.log.append("reset")

    def close(self):
        pass


def _server(budget, slots=4, retain=False, host_outputs=False):
    srv = sv.Server.__new__(sv.Server)
    srv.torch, srv.budget, srv.used = _Torch, budget, 0
    srv.sims, srv.waiting, srv.completed, srv.keep_outputs = {}, sv.collections.deque(), [], False
    srv.host_outputs, srv.n_slots, srv.table_steps, srv.retain, srv.priorities = host_outputs, slots, None, retain, False
    return srv


def _sim(srv, name, first, last, log, n=8, fill=None):
    sim = sv.Simulation(name, types.SimpleNamespace(n=n), first, last, fill=fill, plan=_Plan(log),
                        stream=_Stream(), next_step=first, remaining=last - first + 1)
    sim.slots = [sv.Slot() for _ in range(srv.n_slots)]
    srv.sims[name] = sim
    return sim


def test_out_of_order_arrivals_run_in_step_order():
    _Event.after = 0
    srv = _server(1 << 40)
    log = []
    _sim(srv, "a", 2, 5, log)
    reqs = [sv.Request("a", s, np.zeros((0, 3)), np.zeros(0)) for s in (5, 3, 2, 4)]
    st = srv.run_stream(reqs, [0.0, 0.0, 0.0, 0.0], limit_s=5)
    assert st["requests"] == 4 and log == [2, 3, 4, 5]
    assert st["device_seconds"] == 0.002 and st["fields_per_s"] == 2000.0
    assert srv.sims["a"].plan is None  # released after its last step


def test_duplicate_step_is_refused():
    srv = _server(1 << 40)
    _sim(srv, "a", 0, 3, [])
    srv.submit(sv.Request("a", 1, None, None))
    try:
        srv.submit(sv.Request("a", 1, None, None))
        raise AssertionError("accepted twice")
    except ValueError:
        pass


def test_slots_bound_requests_in_flight_and_stage_each_requests_sources():
    _Event.after = 3  # every request completes only on its 4th poll
    srv = _server(1 << 40, slots=2)
    log = []
    sim = _sim(srv, "a", 0, 5, log)
    plan = sim.plan  # released (set to None) after the last request
    rng = np.random.default_rng(0)
    reqs = [sv.Request("a", s, rng.uniform(size=(s + 1, 3)), rng.uniform(size=s + 1)) for s in range(6)]
    for r in reqs:
        srv.submit(r)
    srv.pump()
    assert len(sim.inflight) == 2 and log == [0, 1]  # two slots, two launched
    inflight_max = 2
    while sim.remaining:
        srv.pump()
        inflight_max = max(inflight_max, len(sim.inflight))
    assert inflight_max <= 2 and log == list(range(6))
    # each push saw its own request's sources (staged into the slot's page-locked buffers)
    for (s, p, l), r in zip(plan.pushed, reqs):
        assert np.array_equal(p, r.pos) and np.array_equal(l, r.lum)
    _Event.after = 0


def test_admission_wait_is_reported_apart():
    _Event.after = 0
    srv = _server(1 << 40)
    sim = _sim(srv, "a", 0, 1, [])
    r0, r1 = sv.Request("a", 0, np.zeros((0, 3)), np.zeros(0)), sv.Request("a", 1, np.zeros((0, 3)), np.zeros(0))
    # both arrive at t = 1 s; the simulation is admitted half a second later
    r0.arrival = r1.arrival = 1.0
    sim.admitted_at = 1.5
    srv.submit(r0)
    srv.submit(r1)
    srv.pump()
    srv.pump()
    st = srv.stats(1.0, 1.0)
    assert st["requests"] == 2 and all(r.admitted == 1.5 for r in srv.completed)
    assert abs(st["p50_ms"] - st["p50_ms_without_admission_wait"] - 500.0) < 1e-6
    assert abs(st["p99_ms"] - st["p99_ms_without_admission_wait"] - 500.0) < 1e-6


def test_rewind_serves_the_same_steps_from_a_refilled_history():
    _Event.after = 0
    srv = _server(1 << 40, retain=True, host_outputs=True)
    log = []
    _sim(srv, "a", 2, 3, log, fill=lambda p: p.log.extend(["fill"]))
    for rnd in range(2):
        reqs = [sv.Request("a", s, np.zeros((0, 3)), np.zeros(0)) for s in (2, 3)]
        st = srv.run_stream(reqs, [0.0, 0.0], limit_s=5)
        assert st["requests"] == 2 and srv.sims["a"].plan is not None  # retained
        srv.rewind()
    assert log == [2, 3, "reset", "fill", 2, 3, "reset", "fill"]
    assert st["by_grid"][8]["requests"] == 2


def test_stream_priority_by_grid_size():
    srv = _server(1 << 40)
    got = {}
    for pr in (True, False):
        srv.priorities = pr
        for n in (128, 192, 256, 384, 512):
            sim = sv.Simulation("s%d" % n, types.SimpleNamespace(n=n), 0, 0, fill=None, plan=None, stream=None,
                                next_step=0, remaining=1)
            got[pr, n] = srv._stream_for(sim).priority
    # CUDA: a lower number is a higher priority; range (0, -5) in the stand-in
    assert got[True, 128] == got[True, 192] == -5
    assert -5 < got[True, 256] < got[True, 384] < got[True, 512] == 0
    assert all(got[False, n] == 0 for n in (128, 192, 256, 384, 512))
