"""Host-side scheduling logic of the continuous-batching server, on the CPU
with a stand-in plan: requests of one simulation run in step order whatever
their arrival order, HBM-budget admission waits for memory to be released."""
import contextlib
import types

import numpy as np

import paper_1502_02294_gb300.serve as sv


class _Event:
    def record(self, s):
        pass

    def query(self):
        return True


class _Stream:
    def synchronize(self):
        pass


class _Torch:
    float32 = None

    class cuda:
        Event = _Event
        Stream = _Stream

        @staticmethod
        def stream(s):
            return contextlib.nullcontext()

    @staticmethod
    def from_numpy(x):
        t = types.SimpleNamespace(to=lambda *a, **k: x)
        t.pin_memory = lambda: t
        return t

    @staticmethod
    def empty(*a, **k):
        return None


class _Plan:
    def __init__(self, log):
        self.log = log

    def push(self, s, p, l):
        self.log.append(s)

    def field(self, s, o):
        pass

    def close(self):
        pass


def _server(budget):
    srv = sv.Server.__new__(sv.Server)
    srv.torch, srv.budget, srv.used = _Torch, budget, 0
    srv.sims, srv.waiting, srv.completed, srv.keep_outputs = {}, sv.collections.deque(), [], False
    return srv


def test_out_of_order_arrivals_run_in_step_order():
    srv = _server(1 << 40)
    log = []
    srv.sims["a"] = sv.Simulation("a", types.SimpleNamespace(n=8), 2, 5, plan=_Plan(log), stream=_Stream(),
                                  next_step=2, remaining=4)
    reqs = [sv.Request("a", s, np.zeros((0, 3)), np.zeros(0)) for s in (5, 3, 2, 4)]
    st = srv.run_stream(reqs, [0.0, 0.0, 0.0, 0.0], limit_s=5)
    assert st["requests"] == 4 and log == [2, 3, 4, 5]
    assert srv.sims["a"].plan is None  # released after its last step


def test_duplicate_step_is_refused():
    srv = _server(1 << 40)
    srv.sims["a"] = sv.Simulation("a", types.SimpleNamespace(n=8), 0, 3, plan=_Plan([]), stream=_Stream(),
                                  next_step=0, remaining=4)
    srv.submit(sv.Request("a", 1, None, None))
    try:
        srv.submit(sv.Request("a", 1, None, None))
        raise AssertionError("accepted twice")
    except ValueError:
        pass
