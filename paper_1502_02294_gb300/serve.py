"""Continuous-batching server for retarded-field evaluations of many simulations.

Each admitted simulation owns a Plan: its Green's function tables and its
device-resident history ring stay on the GPU for as long as it is served.
Requests (simulation, step, sources) arrive over time; the loop

  * admits waiting simulations while the HBM budget allows (host estimate of
    the plan's bytes plus the tables it keeps, `lc_plan_estimate`), and frees
    a simulation's memory when its last request completes (unless told to
    retain it for another pass over the same steps);
  * launches every request whose step is the simulation's next one as soon
    as it arrives and one of the simulation's request slots is free, each
    simulation on its own CUDA stream, so the work of requests that arrive
    while others are running overlaps on the device (requests of one
    simulation stay ordered by its stream);
  * stages each request's host sources through the slot's page-locked
    buffers (allocated once per simulation and slot, grown when a request
    needs more room), so the library's host-to-device copy is asynchronous
    and nothing is allocated or page-locked per request;
  * writes each field to the slot's device buffer, or, with host outputs,
    to the slot's page-locked host buffer through the library's asynchronous
    output path (the copy overlaps the next steps' work);
  * records per-request times on the host clock: arrival, admission of the
    simulation, launch, completion (seen through a CUDA event or the output
    ticket), and brackets the whole stream with CUDA events on the device.

The arithmetic is entirely in liblc; this module only schedules.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Deque, Dict, List, Optional

import numpy as np

from . import Plan, estimate_bytes


@dataclasses.dataclass
class Request:
    sim: str
    step: int
    pos: object  # host numpy (n, 3) float64
    lum: object  # host numpy (n,) float64
    arrival: float = 0.0
    admitted: float = 0.0  # when the request could first run: max(arrival, its simulation's admission)
    launched: float = 0.0
    done: float = 0.0
    out: Optional[object] = None  # the field (device, or page-locked host with host outputs) once launched
    event: Optional[object] = None
    ticket: int = 0
    slot: int = -1


@dataclasses.dataclass
class Slot:
    """One in-flight request's buffers: page-locked sources, and the output."""
    pos: Optional[object] = None  # page-locked torch (cap, 3) float64
    lum: Optional[object] = None  # page-locked torch (cap,) float64
    out: Optional[object] = None  # device or page-locked host (N, N, N) float32
    busy: bool = False


@dataclasses.dataclass
class Simulation:
    name: str
    workload: object
    first_step: int
    last_step: int
    fill: object = None
    plan: Optional[Plan] = None
    stream: Optional[object] = None
    next_step: int = 0
    bytes: int = 0
    pending: Dict[int, Request] = dataclasses.field(default_factory=dict)  # by step
    inflight: List[Request] = dataclasses.field(default_factory=list)
    remaining: int = 0
    admitted_at: float = 0.0
    slots: List[Slot] = dataclasses.field(default_factory=list)


class Server:
    """hbm_budget_bytes: device bytes the admitted simulations may hold.
    keep_outputs: each request gets its own output buffer, kept on the
    Request (else the slot's buffer is reused).  host_outputs: fields go to
    page-locked host memory.  slots: requests in flight per simulation.
    table_steps: None to build every served step's Green's-function table at
    admission (the tables the paper precomputes); k to keep at most k steps'
    tables (lc_plan_set_table_budget), building later ones when their step
    is served.  retain: keep simulations admitted after their last request
    (rewind() then serves the same steps again).  priorities: each
    simulation's stream gets a CUDA stream priority by grid size (four
    tiers: up to 192^3, 256^3, 384^3, larger), so short
    requests of small grids are not queued behind the blocks of large ones;
    False gives every stream the default priority."""

    def __init__(self, hbm_budget_bytes: int, keep_outputs: bool = False, host_outputs: bool = False,
                 slots: int = 4, table_steps: Optional[int] = None, retain: bool = False, priorities: bool = True):
        import torch

        self.torch = torch
        self.budget = int(hbm_budget_bytes)
        self.used = 0
        self.sims: Dict[str, Simulation] = {}
        self.waiting: Deque[str] = collections.deque()
        self.completed: List[Request] = []
        self.keep_outputs = keep_outputs
        self.host_outputs = host_outputs
        self.n_slots = max(1, int(slots))
        self.table_steps = table_steps
        self.retain = retain
        self.priorities = priorities

    # -------------------------------------------------------------- admission
    @staticmethod
    def plan_bytes(w, first_step: int, last_step: int, table_steps: Optional[int] = None) -> int:
        base, per_step = estimate_bytes(w.n, w.steps, w.omega_m, w.h, history=w.history,
                                        kernel=getattr(w, "kernel", None),
                                        horizon_mode=getattr(w, "horizon_mode", 0),
                                        n_shell_max=getattr(w, "n_shell_max", 0))
        served = last_step - first_step + 1
        kept = served if table_steps is None else min(served, int(table_steps))
        return int(base + per_step * kept)

    def add_simulation(self, name: str, workload, first_step: int, last_step: int, fill=None):
        """Register a simulation that will be served for steps [first_step, last_step].
        `fill(plan)` pushes the history before first_step (untimed)."""
        sim = Simulation(name, workload, first_step, last_step, fill=fill, next_step=first_step,
                         bytes=self.plan_bytes(workload, first_step, last_step, self.table_steps),
                         remaining=last_step - first_step + 1)
        self.sims[name] = sim
        self.waiting.append(name)
        self._admit()

    def _stream_for(self, sim: Simulation):
        if not self.priorities:
            return self.torch.cuda.Stream()
        # smaller grids first: their requests are short, so they should not
        # queue behind the blocks of large grids
        lo, hi = self.torch.cuda.Stream.priority_range() if hasattr(self.torch.cuda.Stream, "priority_range") \
            else (0, -1)
        n = sim.workload.n
        # four tiers by grid size, i.e. by service time: up to 192^3, 256^3,
        # 384^3, larger (CUDA: the lower number is the higher priority)
        tier = 0 if n <= 192 else 1 if n <= 256 else 2 if n <= 384 else 3
        prio = hi + int(round((lo - hi) * tier / 3))
        return self.torch.cuda.Stream(priority=prio)

    def _admit(self):
        while self.waiting:
            sim = self.sims[self.waiting[0]]
            if self.used + sim.bytes > self.budget and self.used > 0:
                return  # wait for memory to free up
            self.waiting.popleft()
            sim.stream = self._stream_for(sim)
            with self.torch.cuda.stream(sim.stream):
                sim.plan = Plan.from_workload(sim.workload, stream=sim.stream)
                if self.table_steps is None:
                    sim.plan.prepare(sim.first_step, sim.last_step + 1)
                else:
                    _, per_step = estimate_bytes(sim.workload.n, sim.workload.steps, sim.workload.omega_m,
                                                 sim.workload.h, history=sim.workload.history,
                                                 kernel=getattr(sim.workload, "kernel", None))
                    sim.plan.set_table_budget(int(per_step * self.table_steps))
                    sim.plan.prepare(sim.first_step, min(sim.last_step + 1, sim.first_step + self.table_steps))
                if sim.fill:
                    sim.fill(sim.plan)
            sim.slots = [Slot() for _ in range(self.n_slots)]
            sim.admitted_at = time.perf_counter()
            self.used += sim.bytes

    def _release(self, sim: Simulation):
        sim.stream.synchronize()
        sim.plan.close()
        sim.plan = None
        sim.slots = []
        self.used -= sim.bytes
        self._admit()

    def rewind(self):
        """Serve the same steps again: every retained simulation forgets its
        history, is refilled (untimed) and starts at its first step."""
        for sim in self.sims.values():
            if sim.plan is None:
                continue
            sim.stream.synchronize()
            sim.plan.reset()
            with self.torch.cuda.stream(sim.stream):
                if sim.fill:
                    sim.fill(sim.plan)
            sim.next_step = sim.first_step
            sim.remaining = sim.last_step - sim.first_step + 1
            sim.admitted_at = time.perf_counter()
        self.completed = []
        self.torch.cuda.synchronize()

    def close(self):
        for sim in self.sims.values():
            if sim.plan is not None:
                self._release(sim)

    # -------------------------------------------------------------- requests
    def submit(self, req: Request):
        if not req.arrival:
            req.arrival = time.perf_counter()
        sim = self.sims[req.sim]
        if req.step in sim.pending or req.step < sim.next_step:
            raise ValueError(f"{req.sim}: step {req.step} requested twice")
        sim.pending[req.step] = req  # launched once every earlier step has been

    def _stage(self, slot: Slot, n_src: int, pos, lum):
        """Copy a request's sources into the slot's page-locked buffers (grown
        to the next power of two when too small); returns views of n_src rows."""
        torch = self.torch
        if slot.lum is None or slot.lum.shape[0] < n_src:
            cap = 1024
            while cap < n_src:
                cap *= 2
            slot.pos = torch.empty((cap, 3), dtype=torch.float64).pin_memory()
            slot.lum = torch.empty((cap,), dtype=torch.float64).pin_memory()
        p, l_ = slot.pos[:n_src], slot.lum[:n_src]
        p.numpy()[...] = pos
        l_.numpy()[...] = lum
        return p, l_

    def _output(self, sim: Simulation, slot: Slot):
        torch = self.torch
        n = sim.workload.n
        if self.keep_outputs:
            if self.host_outputs:
                return torch.empty((n, n, n), dtype=torch.float32).pin_memory()
            return torch.empty((n, n, n), dtype=torch.float32, device="cuda")
        if slot.out is None:
            slot.out = (torch.empty((n, n, n), dtype=torch.float32).pin_memory() if self.host_outputs
                        else torch.empty((n, n, n), dtype=torch.float32, device="cuda"))
        return slot.out

    def _launch_ready(self):
        torch = self.torch
        for sim in self.sims.values():
            if sim.plan is None:
                continue
            while sim.next_step in sim.pending:
                free = [k for k, s in enumerate(sim.slots) if not s.busy]
                if not free:
                    break  # every slot in flight: launch once one completes
                req = sim.pending.pop(sim.next_step)
                slot = sim.slots[free[0]]
                slot.busy = True
                req.slot = free[0]
                req.admitted = max(req.arrival, sim.admitted_at)
                n_src = int(req.lum.shape[0])
                with torch.cuda.stream(sim.stream):
                    pos, lum = self._stage(slot, n_src, req.pos, req.lum)
                    sim.plan.push(req.step, pos, lum)  # page-locked host sources: an asynchronous copy
                    req.out = self._output(sim, slot)
                    if self.host_outputs:
                        req.ticket = sim.plan.field_async(req.step, req.out)
                    else:
                        sim.plan.field(req.step, req.out)
                    req.event = torch.cuda.Event()
                    req.event.record(sim.stream)
                req.launched = time.perf_counter()
                sim.next_step += 1
                sim.inflight.append(req)

    def _finished(self, sim: Simulation, req: Request) -> bool:
        if self.host_outputs:
            return sim.plan.poll(req.ticket)
        return req.event.query()

    def _poll(self) -> int:
        n_done = 0
        for sim in list(self.sims.values()):
            still = []
            for req in sim.inflight:
                if self._finished(sim, req):
                    req.done = time.perf_counter()
                    sim.slots[req.slot].busy = False
                    if not self.keep_outputs:
                        req.out = None
                    self.completed.append(req)
                    sim.remaining -= 1
                    n_done += 1
                else:
                    still.append(req)
            sim.inflight = still
            if sim.plan is not None and sim.remaining == 0 and not sim.inflight and not self.retain:
                self._release(sim)
        return n_done

    def pump(self) -> int:
        """One scheduler iteration: launch what is ready, collect what finished."""
        self._launch_ready()
        return self._poll()

    def busy(self) -> bool:
        return any(s.pending or s.inflight or (s.plan is not None and not self.retain)
                   for s in self.sims.values()) or bool(self.waiting)

    # -------------------------------------------------------------- driver
    def run_stream(self, requests: List[Request], arrivals: List[float], limit_s: float = 600.0) -> dict:
        """Feed requests at the given offsets (seconds from now) and serve them all
        (raises TimeoutError after `limit_s` seconds of wall clock).  The
        device time of the stream is taken between CUDA events: one recorded
        before the first request that every admitted simulation's stream
        waits on, one after every stream's last work."""
        torch = self.torch
        origin = torch.cuda.current_stream()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(origin)
        for sim in self.sims.values():
            if sim.stream is not None:
                sim.stream.wait_event(start)
        t0 = time.perf_counter()
        order = np.argsort(np.asarray(arrivals, dtype=np.float64), kind="stable")
        i = 0
        while i < len(order) or self.busy():
            now = time.perf_counter() - t0
            if now > limit_s:
                raise TimeoutError(f"serving did not finish within {limit_s} s")
            while i < len(order) and arrivals[order[i]] <= now:
                r = requests[order[i]]
                r.arrival = t0 + arrivals[order[i]]
                self.submit(r)
                i += 1
            self.pump()
            if i >= len(order) and not any(s.pending or s.inflight for s in self.sims.values()):
                break
        t_end = time.perf_counter()
        for sim in self.sims.values():
            if sim.stream is not None:
                ev = torch.cuda.Event()
                ev.record(sim.stream)
                origin.wait_event(ev)
        end.record(origin)
        end.synchronize()
        dev_s = start.elapsed_time(end) / 1e3
        return self.stats(t_end - t0, dev_s)

    def stats(self, host_s: float, device_s: float) -> dict:
        done = self.completed

        def pct(x, q):
            return float(np.percentile(x, q)) if len(x) else None

        lat = np.array([(r.done - r.arrival) * 1e3 for r in done])
        lat_adm = np.array([(r.done - r.admitted) * 1e3 for r in done])
        svc = np.array([(r.done - r.launched) * 1e3 for r in done])
        by_n: Dict[int, List[float]] = collections.defaultdict(list)
        for r, v in zip(done, lat):
            by_n[self.sims[r.sim].workload.n].append(v)
        return {"requests": len(done), "seconds": host_s, "device_seconds": device_s,
                "fields_per_s": len(done) / max(1e-9, device_s),
                "fields_per_s_host_clock": len(done) / max(1e-9, host_s),
                "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
                "p50_ms_without_admission_wait": pct(lat_adm, 50), "p99_ms_without_admission_wait": pct(lat_adm, 99),
                "service_p50_ms": pct(svc, 50), "service_p99_ms": pct(svc, 99),
                "by_grid": {int(n): {"requests": len(v), "p50_ms": pct(v, 50), "p99_ms": pct(v, 99)}
                            for n, v in sorted(by_n.items())},
                "peak_hbm_bytes_budgeted": self.budget}


__all__ = ["Server", "Request", "Simulation", "Slot"]
