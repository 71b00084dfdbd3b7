"""Continuous-batching server for retarded-field evaluations of many simulations.

Each admitted simulation owns a Plan: its Green's function tables and its
device-resident history ring stay on the GPU for as long as it is served.
Requests (simulation, step, sources) arrive over time; the loop

  * admits waiting simulations while the HBM budget allows (host estimate of
    the plan's bytes plus its prepared tables, `lc_plan_estimate`), and frees
    a simulation's memory when its last request completes;
  * launches every request whose step is the simulation's next one as soon
    as it arrives, each simulation on its own CUDA stream, so the work of
    requests that arrive while others are running overlaps on the device
    (requests of one simulation stay ordered by its stream);
  * records per-request latency = completion - arrival (host clock, the
    completion seen through a CUDA event), and the throughput in fields/s.

The arithmetic is entirely in liblc; this module only schedules.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Deque, Dict, List, Optional

import numpy as np

from . import HISTORY_BF16, Plan, estimate_bytes


@dataclasses.dataclass
class Request:
    sim: str
    step: int
    pos: object  # host numpy (n, 3) float64
    lum: object  # host numpy (n,) float64
    arrival: float = 0.0
    launched: float = 0.0
    done: float = 0.0
    out: Optional[object] = None  # device tensor with the field once launched
    event: Optional[object] = None


@dataclasses.dataclass
class Simulation:
    name: str
    workload: object
    first_step: int
    last_step: int
    plan: Optional[Plan] = None
    stream: Optional[object] = None
    next_step: int = 0
    bytes: int = 0
    pending: Dict[int, Request] = dataclasses.field(default_factory=dict)  # by step
    inflight: List[Request] = dataclasses.field(default_factory=list)
    remaining: int = 0


class Server:
    def __init__(self, hbm_budget_bytes: int, keep_outputs: bool = False):
        import torch

        self.torch = torch
        self.budget = int(hbm_budget_bytes)
        self.used = 0
        self.sims: Dict[str, Simulation] = {}
        self.waiting: Deque[str] = collections.deque()
        self.completed: List[Request] = []
        self.keep_outputs = keep_outputs

    # -------------------------------------------------------------- admission
    @staticmethod
    def plan_bytes(w, first_step: int, last_step: int) -> int:
        base, per_step = estimate_bytes(w.n, w.steps, w.omega_m, w.h, history=w.history,
                                        kernel=getattr(w, "kernel", None))
        return int(base + per_step * (last_step - first_step + 1))

    def add_simulation(self, name: str, workload, first_step: int, last_step: int, fill=None):
        """Register a simulation that will be served for steps [first_step, last_step].
        `fill(plan)` pushes the history before first_step (untimed)."""
        sim = Simulation(name, workload, first_step, last_step, next_step=first_step,
                         bytes=self.plan_bytes(workload, first_step, last_step),
                         remaining=last_step - first_step + 1)
        sim.fill = fill
        self.sims[name] = sim
        self.waiting.append(name)
        self._admit()

    def _admit(self):
        while self.waiting:
            sim = self.sims[self.waiting[0]]
            if self.used + sim.bytes > self.budget and self.used > 0:
                return  # wait for memory to free up
            self.waiting.popleft()
            sim.stream = self.torch.cuda.Stream()
            with self.torch.cuda.stream(sim.stream):
                sim.plan = Plan.from_workload(sim.workload, stream=sim.stream)
                sim.plan.prepare(sim.first_step, sim.last_step + 1)
                if sim.fill:
                    sim.fill(sim.plan)
            self.used += sim.bytes

    def _release(self, sim: Simulation):
        sim.stream.synchronize()
        sim.plan.close()
        sim.plan = None
        self.used -= sim.bytes
        self._admit()

    # -------------------------------------------------------------- requests
    def submit(self, req: Request):
        if not req.arrival:
            req.arrival = time.perf_counter()
        sim = self.sims[req.sim]
        if req.step in sim.pending or req.step < sim.next_step:
            raise ValueError(f"{req.sim}: step {req.step} requested twice")
        sim.pending[req.step] = req  # launched once every earlier step has been

    def _launch_ready(self):
        torch = self.torch
        for sim in self.sims.values():
            if sim.plan is None:
                continue
            while sim.next_step in sim.pending:
                req = sim.pending.pop(sim.next_step)
                n = sim.workload.n
                with torch.cuda.stream(sim.stream):
                    # stage the sources in pinned memory so that the copies are
                    # asynchronous (a copy from pageable memory waits for the
                    # stream, which would serialise the simulations)
                    pos = torch.from_numpy(req.pos).pin_memory().to("cuda", non_blocking=True)
                    lum = torch.from_numpy(req.lum).pin_memory().to("cuda", non_blocking=True)
                    req.out = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
                    sim.plan.push(req.step, pos, lum)
                    sim.plan.field(req.step, req.out)
                    req.event = torch.cuda.Event()
                    req.event.record(sim.stream)
                req.launched = time.perf_counter()
                sim.next_step += 1
                sim.inflight.append(req)

    def _poll(self) -> int:
        n_done = 0
        for sim in list(self.sims.values()):
            still = []
            for req in sim.inflight:
                if req.event.query():
                    req.done = time.perf_counter()
                    if not self.keep_outputs:
                        req.out = None
                    self.completed.append(req)
                    sim.remaining -= 1
                    n_done += 1
                else:
                    still.append(req)
            sim.inflight = still
            if sim.plan is not None and sim.remaining == 0 and not sim.inflight:
                self._release(sim)
        return n_done

    def pump(self) -> int:
        """One scheduler iteration: launch what is ready, collect what finished."""
        self._launch_ready()
        return self._poll()

    def busy(self) -> bool:
        return any(s.pending or s.inflight or s.plan is not None for s in self.sims.values()) or bool(self.waiting)

    # -------------------------------------------------------------- driver
    def run_stream(self, requests: List[Request], arrivals: List[float], limit_s: float = 600.0) -> dict:
        """Feed requests at the given offsets (seconds from now) and serve them all
        (raises TimeoutError after `limit_s` seconds of wall clock)."""
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
        lat = np.array([(r.done - r.arrival) * 1e3 for r in self.completed])
        return {"requests": len(self.completed), "seconds": t_end - t0,
                "fields_per_s": len(self.completed) / max(1e-9, t_end - t0),
                "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
                "peak_hbm_bytes_budgeted": self.budget}


__all__ = ["Server", "Request", "Simulation"]
