#!/usr/bin/env python
"""Benchmark: retarded (light-cone) Lyman-Werner field evaluations per second.

Workload (default): 128^3 periodic grid, 150 comoving Mpc box, flat LCDM
(Omega_m = 0.31, h = 0.68), 64 equal-cosmic-time steps z = 30 -> 10 (up to 7
active light-cone shells), 1e4 Gaussian-clustered sources with a M^-2 mass
function and 1-4 step lifetimes, FP32 FFT + shell multiply-accumulate.  A
"step" is one push of that step's sources (deposit + forward transform into
the history ring) plus one retarded-field evaluation (shell MAC + inverse
transform).  The 64-step run is cycled (history reset at the wrap).

Timing: W warm-up steps, then K steps timed one by one with CUDA events on the
plan's stream, L2 flushed (a 512 MB write) between timed steps, outside the
events.  Each step is one replay of a CUDA graph captured once per observed
step (the library's lc_graph_create); the per-phase events captured inside
the graphs give the shell-MAC kernel's own duration for the roofline.  Under torchrun each rank runs an independent simulation on its own
GPU (weak scaling, no data-path collective); the reported time is the max over
ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "retarded-field evals/s & cell·shell MAC/s vs plain FP32 path; HBM %; p50/p99"
UNIT = "fields/s"
WORKLOADS = {
    "c2": ("128^3 grid, 150 Mpc box, 64 equal-time steps z=30->10 (<=7 shells), 1e4 clustered sources "
           "(dN/dM~M^-2, 1-4 step lifetimes), FP32 FFT+MAC"),
    "c1": "32^3 grid, 100 Mpc box, 8 equal-time steps z=20->15 (<=2 shells), 200 uniform sources, FP32",
    "c3": ("256^3 grid, 200 Mpc box, 128 equal-conformal-time shells spanning the LW horizon at z=15, "
           "1e5 clustered sources, BF16 history with per-slot FP32 scale"),
    "c3s": ("256^3 grid, 200 Mpc box, 32 equal-conformal-time shells, 40 steps, 1e5 clustered sources, "
            "BF16 history (profiling size of the c3 path)"),
    "c4": ("16 uneven instances (grids 64..256 cycled, 32..128 shells, 1e3..1e5 clustered sources, 0.78 Mpc "
           "cells), FP32, all instances' step in one CUDA graph replay (parallel branches)"),
    "c5": ("serving: 8 simulations N = 128, 192, 256, 256, 384, 384, 512, 512 with 128, 112, 96, 128, 96, 64, "
           "96, 96 shells, BF16 history, 1e4-1e5 clustered sources, 16 requests each, continuous batching under an "
           "HBM budget; beside it the plain FP32 one-instance path on the same requests"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 2048 for c1/c2, 64 for c3, 32 for c3s/c4/c5, 16 for --impl reference)")
    ap.add_argument("--warmup", type=int, default=8)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--flush-mb", type=int, default=512)
    ap.add_argument("--kernel", default="lw", choices=["lw", "exp"],
                    help="radial kernel: Lyman-Werner (Eqs. 14-17) or exp(-r/30 Mpc) cut off at 80 Mpc")
    ap.add_argument("--near", default="ngp", choices=["ngp", "subcell"],
                    help="innermost slice's near field: cell-centred (NGP) or from the sources' own positions")
    ap.add_argument("--e2e-pipelined", action="store_true",
                    help="also time the host-I/O loop with Plan.field_async (each step's output copy overlaps the "
                         "next step; no L2 flush between steps, which would serialise that overlap)")
    ap.add_argument("--fdiff", action="store_true",
                    help="each step also builds the instantaneous field (Eq. 18) and the f_diff map")
    return ap.parse_args()


EXP_KERNEL = (1, 30.0, 80.0)  # exp(-r / 30 Mpc), cut off at r_max = 80 Mpc


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle
def oracle_field_rate(w, steps, cells_per_step=4096, seed=0):
    """Time the FP64 oracle on a bounded sample: for each step, its Green's
    functions plus `cells_per_step` sampled cells; extrapolate to a full field.
    Returns (fields/s, seconds spent, description)."""
    import oracle

    oracle.build()
    P = oracle.Problem.from_workload(w)
    spent = 0.0
    per_field = []
    for s in steps:
        grids = oracle.source_grids(P, w.cat, s)
        one = np.array([0], dtype=np.int64)
        t0 = time.perf_counter()
        P.field(s, grids, cells=one)  # Green's functions + one cell: the fixed cost
        t1 = time.perf_counter()
        cells = np.random.default_rng(seed + s).integers(0, w.n ** 3, size=cells_per_step).astype(np.int64)
        P.field(s, grids, cells=cells)
        t2 = time.perf_counter()
        fixed = t1 - t0
        per_cell = max(0.0, (t2 - t1) - fixed) / cells_per_step
        per_field.append(fixed + per_cell * w.n ** 3)
        spent += t2 - t0
    desc = (f"oracle FP64 on steps {list(steps)}: Green's functions + {cells_per_step} sampled cells per step, "
            f"full-field time extrapolated from the per-cell rate")
    return 1.0 / float(np.mean(per_field)), spent, desc


# ---------------------------------------------------------------- main
def active_shell_work(plan, w, s):
    """Shells the MAC reads at step s: active slices whose step had sources."""
    lo, hi, rh = plan.shells(s)
    return sum(1 for j in range(len(lo)) if w.cat.active(s - j)[1].shape[0] > 0), len(lo)


def run_batched(args, ClockSampler=ClockSampler):
    """16 uneven instances, one batch-graph replay per step."""
    import torch

    import paper_1502_02294_gb300 as lc
    import synth

    lc.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    ws = synth.batched_instances()
    window = 8
    plans, srcs, outs = [], [], []
    for w in ws:
        p = lc.Plan.from_workload(w, stream=stream)
        p.prepare(w.steps.n_shell, w.steps.n_shell + window)
        plans.append(p)
        srcs.append([(torch.from_numpy(w.cat.active(s)[0]).to(dev), torch.from_numpy(w.cat.active(s)[1]).to(dev))
                     for s in range(w.steps.n_steps)])
        outs.append(torch.empty((w.n,) * 3, dtype=torch.float32, device=dev))

    def refill():
        for p, w, sr in zip(plans, ws, srcs):
            p.reset()
            for s in range(w.steps.n_shell):
                p.push(s, *sr[s])

    graphs = [lc.BatchGraph(plans, [w.steps.n_shell + k for w in ws],
                            [sr[w.steps.n_shell + k] for w, sr in zip(ws, srcs)], outs) for k in range(window)]
    flush = torch.empty(args.flush_mb << 20, dtype=torch.uint8, device=dev)
    refill()
    for k in range(min(args.warmup, window)):
        graphs[k].launch(stream)
    torch.cuda.synchronize()
    refill()
    sampler = ClockSampler(0)
    sampler.start()
    launches0 = lc.kernel_launches()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        k = i % window
        if i and k == 0:
            refill()
        flush.zero_()
        evs[i][0].record(stream)
        graphs[k].launch(stream)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    launches = lc.kernel_launches() - launches0
    clocks = sampler.stop()
    per = np.array([a.elapsed_time(b) for a, b in evs])
    T = per.sum() / 1e3
    # MAC roofline: the same steps with per-instance timed graphs, one instance at a time
    mac_ms, mac_bytes = 0.0, 0.0
    refill()
    for p in plans:
        p.set_timing(True)
        p.timing(reset=True)
    tgs = [[p.graph(w.steps.n_shell + k, *sr[w.steps.n_shell + k], o) for k in range(window)]
           for p, w, sr, o in zip(plans, ws, srcs, outs)]
    for p in plans:
        p.set_timing(False)
    for k in range(window):
        for tg in tgs:
            tg[k].launch()
    torch.cuda.synchronize()
    for p, w in zip(plans, ws):
        ph = p.timing(reset=True)
        mac_ms += ph["mac_x"][0]
        nk = w.n * w.n * (w.n // 2 + 1)
        for k in range(window):
            s = w.steps.n_shell + k
            nsh, A = active_shell_work(p, w, s)
            mac_bytes += nk * (8 * nsh + 8) + p.wedge_size * 4 * A
    for tg in tgs:
        for g in tg:
            g.close()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    mac_gbs = mac_bytes / (mac_ms / 1e3) / 1e9 if mac_ms > 0 else None
    traffic, traffic_src = mac_traffic(args.workload)
    # e2e: host buffers through the plain batched call
    host_in = [[(np.ascontiguousarray(w.cat.active(s)[0]), np.ascontiguousarray(w.cat.active(s)[1]))
                for s in range(w.steps.n_steps)] for w in ws]
    refill()
    e2e_t, h2d = 0.0, 0
    for i in range(args.steps):
        k = i % window
        if i and k == 0:
            refill()
        torch.cuda.synchronize()
        tic = time.perf_counter()
        for p, w, hi in zip(plans, ws, host_in):
            s = w.steps.n_shell + k
            p.push(s, *hi[s])
        host_outs = []
        for p, w in zip(plans, ws):
            o = np.empty((w.n,) * 3, dtype=np.float32)
            p.field(w.steps.n_shell + k, o)
            host_outs.append(o)
        e2e_t += time.perf_counter() - tic
        h2d += sum(hi[w.steps.n_shell + k][0].nbytes + hi[w.steps.n_shell + k][1].nbytes for w, hi in zip(ws, host_in))
    for g in graphs:
        g.close()
    for p in plans:
        p.close()
    n_inst = len(ws)
    line = {
        "metric": METRIC, "value": n_inst * args.steps / T, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"c4: {WORKLOADS['c4']}", "instances": n_inst, "grids": [w.n for w in ws],
                   "shells": [w.steps.n_shell for w in ws], "timed_window_steps": window,
                   "l2": f"flushed between timed steps ({args.flush_mb} MB write outside the events)",
                   "inputs": "device-resident"},
        "latency_ms": {"p50": float(np.percentile(per, 50)), "p99": float(np.percentile(per, 99))},
        "roofline": {"bound": "hbm", "kernel": "shell MAC fused with the inverse x pass (all instances)",
                     "achieved": mac_gbs, "peak": hbm_peak, "unit": "GB/s",
                     "frac": (mac_gbs / hbm_peak) if mac_gbs else None, "traffic": None,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"},
        "clocks": clocks,
        "e2e": {"value": n_inst * args.steps / e2e_t, "unit": UNIT, "h2d_bytes_per_step": int(h2d // args.steps),
                "d2h_bytes_per_step": int(sum(4 * w.n ** 3 for w in ws))},
        "gpu_launches": int(launches), "cpu_baseline": None,
        "launch": "one batch CUDA graph per step: 16 parallel branches (one per instance)",
    }
    print(json.dumps(line))
    return 0


def run_serving(args, ClockSampler=ClockSampler):
    """Continuous batching of field requests from the 8 served simulations
    (128^3..512^3, BF16 history), beside the plain FP32 one-instance path on
    the same requests."""
    import dataclasses

    import torch

    import paper_1502_02294_gb300 as lc
    import synth
    from paper_1502_02294_gb300.serve import Request, Server

    lc.build()
    torch.cuda.set_device(0)
    ws = synth.served_simulations()
    per_sim = 16
    grids = [w.n for w in ws]
    shells = [w.steps.n_shell for w in ws]

    def fill(p, w):
        for s in range(w.steps.n_shell):
            p.push(s, *w.cat.active(s))

    def one_pass(rate):
        srv = Server(hbm_budget_bytes=int(0.6 * torch.cuda.get_device_properties(0).total_memory))
        reqs = []
        for w in ws:
            sh = w.steps.n_shell
            srv.add_simulation(w.name, w, sh, sh + per_sim - 1, fill=lambda p, w=w: fill(p, w))
            for s in range(sh, sh + per_sim):
                reqs.append(Request(w.name, s, *w.cat.active(s)))
        torch.cuda.synchronize()
        rng = np.random.default_rng(7)
        if rate is None:
            arr = [0.0] * len(reqs)
        else:
            # Poisson arrivals of the whole stream; each simulation's requests keep step order
            t = np.cumsum(rng.exponential(1.0 / rate, size=len(reqs)))
            order = rng.permutation(len(reqs))
            arr = [0.0] * len(reqs)
            for slot, i in enumerate(order):
                arr[i] = float(t[slot])
            for w in ws:
                idx = [i for i, r in enumerate(reqs) if r.sim == w.name]
                ts = sorted(arr[i] for i in idx)
                for i, tt in zip(idx, ts):
                    arr[i] = tt
        return srv.run_stream(reqs, arr, limit_s=300.0)

    def plain_fp32():
        """The same requests, one simulation at a time in FP32 history: eager
        push + field per request on the default stream, no graph, no overlap;
        tables and history filled before the clock starts."""
        total, n = 0.0, 0
        for w in ws:
            wf = dataclasses.replace(w, history=synth.HISTORY_FP32)
            sh = w.steps.n_shell
            plan = lc.Plan.from_workload(wf)
            plan.prepare(sh, sh + per_sim)
            fill(plan, wf)
            reqs = [wf.cat.active(s) for s in range(sh, sh + per_sim)]
            out = torch.empty((w.n,) * 3, dtype=torch.float32, device="cuda")
            torch.cuda.synchronize()
            tic = time.perf_counter()
            for k, (pos, lum) in enumerate(reqs):
                plan.push(sh + k, torch.from_numpy(pos).to("cuda"), torch.from_numpy(lum).to("cuda"))
                plan.field(sh + k, out)
            torch.cuda.synchronize()
            total += time.perf_counter() - tic
            n += len(reqs)
            plan.close()
            del out
            torch.cuda.empty_cache()
        return n / total, total

    one_pass(None)  # warm-up: touches every code path and tunes the kernels
    sampler = ClockSampler(0)
    sampler.start()
    sat = one_pass(None)
    clocks = sampler.stop()
    pois = one_pass(0.8 * sat["fields_per_s"])
    plain_rate, plain_s = plain_fp32()
    line = {
        "metric": METRIC, "value": sat["fields_per_s"], "unit": UNIT, "n_gpus": 1, "steps": sat["requests"],
        "warmup": len(ws) * per_sim, "ms_per_step": 1e3 / sat["fields_per_s"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32", "data": "synthetic",
        "config": {"workload": f"c5: {WORKLOADS['c5']}", "grids": grids, "shells": shells,
                   "requests_per_sim": per_sim, "poisson_rate_fields_per_s": 0.8 * sat["fields_per_s"]},
        "latency_ms": {"saturation_p50": sat["p50_ms"], "saturation_p99": sat["p99_ms"],
                       "poisson_p50": pois["p50_ms"], "poisson_p99": pois["p99_ms"]},
        "poisson_fields_per_s": pois["fields_per_s"],
        "plain_fp32_one_instance": {"fields_per_s": plain_rate, "seconds": plain_s,
                                    "served_over_plain": sat["fields_per_s"] / plain_rate,
                                    "path": "FP32 history, one plan at a time, eager push + field per request, "
                                            "no graph, no overlap (tables and history prepared untimed)"},
        "clocks": clocks,
        "e2e": {"value": sat["fields_per_s"], "unit": UNIT,
                "h2d_bytes_per_step": int(np.mean([w.cat.active(w.steps.n_shell)[1].nbytes * 4 for w in ws])),
                "d2h_bytes_per_step": 0, "note": "requests carry host sources; fields stay on the device"},
        "roofline": None, "cpu_baseline": None,
        "launch": "per-simulation streams, requests launched as they arrive (continuous batching)",
    }
    print(json.dumps(line))
    return 0


# DRAM traffic (ncu dram__bytes_read.sum + dram__bytes_write.sum) of the
# shell-MAC phase per step, from the captures summarised in profiles/, valid
# only for the MAC kernel sources they were taken with (hash below: the
# warp-specialised and bulk kernels, the gather pass and its slot list); c3 is
# the c3s capture (32 slices) with its reads scaled to 128 slices.
MAC_TRAFFIC = {
    "c2": {"sources": "575a4b4d64a0d777", "bytes": 38.472e6,
           "from": "profiles/c2_dram_traffic.md (64-step window, all MAC-phase launches)"},
    "c3": {"sources": "575a4b4d64a0d777", "bytes": 4 * 1.192879e9 + 73.619e6,
           "from": "profiles/k_mac_ws_256_bf16_pair.md (c3s, reads x 128/32)"},
}


def max_over_ranks(x, device):
    """The largest of every rank's x (the job's time is its slowest rank's);
    x itself when no process group is running."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _function_text(src, head):
    """The text of the function whose definition line contains `head`, from
    the start of that line to the closing brace at the start of a line."""
    i = src.rfind("\n", 0, src.index(head)) + 1
    return src[i:src.index("\n}\n", i) + 3]


def mac_sources_hash():
    import hashlib

    d = os.path.join(ROOT, "paper_1502_02294_gb300", "csrc")
    h = hashlib.sha256()
    with open(os.path.join(d, "lc_mac.cuh"), "rb") as fh:
        h.update(fh.read())
    with open(os.path.join(d, "lc_kernels.cuh")) as fh:
        k = fh.read()
    h.update(_function_text(k, "__device__ __forceinline__ void mac_slot_list(").encode())
    h.update(_function_text(k, " k_cols(ColArgs a) {").encode())
    return h.hexdigest()[:16]


def mac_traffic(workload):
    t = MAC_TRAFFIC.get(workload)
    if t is None or t["sources"] != mac_sources_hash():
        return None, None
    return t["bytes"], t["from"]


DEFAULT_STEPS = {"c1": 2048, "c2": 2048, "c3": 64, "c3s": 32, "c4": 32, "c5": 32}


def main():
    args = parse()
    if args.steps is None:
        args.steps = 16 if args.impl == "reference" else DEFAULT_STEPS.get(args.workload, 64)
    if args.workload == "c4" and args.impl == "ours":
        return run_batched(args)
    if args.workload == "c5" and args.impl == "ours":
        return run_serving(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import synth

    w = synth.config(args.workload)
    variant = {}
    if args.kernel == "exp":
        w = dataclasses.replace(w, kernel=EXP_KERNEL)
        variant["radial_kernel"] = "exp(-r/30 Mpc), cut off at 80 Mpc"
    if args.near == "subcell":
        w = dataclasses.replace(w, near_mode=1)
        variant["near_field"] = "sub-cell (s^3 sub-samples around each source's own position)"
    if args.fdiff:
        variant["step_adds"] = "instantaneous field (Eq. 18) + f_diff map, inside the timed step"

    if args.impl == "reference":
        if rank != 0:
            return 0
        import oracle

        threads = oracle.threads()
        steps_pool = list(range(max(1, w.steps.n_steps // 2), w.steps.n_steps))
        for i in range(args.warmup):
            oracle_field_rate(w, [steps_pool[i % len(steps_pool)]], cells_per_step=256)
        # each step: one observing step's Green's functions plus a cell sample
        # sized so that the K steps take about two minutes in all
        cells = 1024
        rates, spent = [], 0.0
        for i in range(args.steps):
            r, sp, desc = oracle_field_rate(w, [steps_pool[i % len(steps_pool)]], cells_per_step=cells, seed=i)
            rates.append(r)
            spent += sp
            if i == 0:
                cells = int(min(65536, w.n ** 3, max(64, cells * (120.0 / args.steps) / max(sp, 1e-3))))
        value = float(np.mean(rates))
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}", "grid": w.n,
                           "steps_in_run": w.steps.n_steps, **variant},
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                                 "sample": f"each step: one observing step's Green's functions + {cells} sampled "
                                           "cells (1024 on the first), full-field time extrapolated from the per-cell "
                                           "rate" + ("; the retarded field alone (cell-centred near field, no "
                                                     "f_diff map)" if args.near != "ngp" or args.fdiff else "")},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "cpu_seconds": spent}
        print(json.dumps(line))
        return 0

    import torch

    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    import paper_1502_02294_gb300 as lc

    lc.build()
    stream = torch.cuda.current_stream()
    plan = lc.Plan.from_workload(w, stream=stream)
    T = w.steps.n_steps
    t_first = 0 if w.steps.kind != synth.STEPS_EQUAL_TAU else w.steps.n_shell
    plan.prepare(t_first, T)  # the observed steps' Green's function tables (plan time)
    # device-resident inputs of every step
    src_dev = []
    for s in range(T):
        pos, lum = w.cat.active(s)
        src_dev.append((torch.from_numpy(pos).to(dev), torch.from_numpy(lum).to(dev)))
    out = torch.empty((w.n,) * 3, dtype=torch.float32, device=dev)
    out_inst = torch.empty_like(out) if args.fdiff else None
    out_fdiff = torch.empty_like(out) if args.fdiff else None
    flush = torch.empty(args.flush_mb << 20, dtype=torch.uint8, device=dev)

    def fdiff_after(s):
        # the instantaneous field of step s and f_diff = (J_inst - J) / J per cell
        plan.instant_field(s, out_inst)
        lc.fdiff_map(out, out_inst, out_fdiff, stream=stream)
    # timed window: every step for the equal-time runs; for the equal-conformal-time
    # run the last n_shell/4 steps, after n_shell untimed fill steps (history only)
    t0 = 0 if w.steps.kind != synth.STEPS_EQUAL_TAU else w.steps.n_shell
    work = {s: active_shell_work(plan, w, s) for s in range(t0, T)}
    nk = w.n * w.n * (w.n // 2 + 1)

    def refill():
        plan.reset()
        for s in range(t0):
            plan.push(s, *src_dev[s])

    # one CUDA graph per observed step (push + field on device buffers).  The
    # headline pass replays graphs without instrumentation; a second pass
    # replays graphs captured with the per-phase events inside, which time the
    # shell-MAC kernel on its own for the roofline.
    window = T - t0
    graphs = {s: plan.graph(s, *src_dev[s], out) for s in range(t0, T)}
    plan.set_timing(True)
    graphs_timed = {s: plan.graph(s, *src_dev[s], out) for s in range(t0, T)}
    plan.set_timing(False)
    # which shell-MAC kernel the autotuner picked for each active-slice count
    tag = f"/N{w.n}/{'bf16' if w.history else 'fp32'}/"
    mac_choice = {k.rsplit("/", 1)[1]: v for k, v in lc.autotune_report().items() if tag in k}

    def run_pass(gs, evs=None, nvtx=False):
        refill()
        steps_done = []
        for i in range(args.steps):
            s = t0 + i % window
            if i and s == t0:
                refill()  # history restarts (untimed: outside the events)
            flush.zero_()  # L2 flush between timed steps, outside the events
            if evs:
                evs[i][0].record(stream)
            if nvtx:
                torch.cuda.nvtx.range_push("step")  # lets a profiler select the timed replays
            gs[s].launch()
            if args.fdiff:
                fdiff_after(s)
            if nvtx:
                torch.cuda.nvtx.range_pop()
            if evs:
                evs[i][1].record(stream)
            steps_done.append(s)
        return steps_done

    refill()
    for i in range(max(3, args.warmup)):
        s = t0 + i % window
        if i and s == t0:
            refill()
        graphs[s].launch()
        if args.fdiff:
            fdiff_after(s)
    torch.cuda.synchronize()
    sampler = ClockSampler(dev.index)
    sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = lc.kernel_launches()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    done_steps = run_pass(graphs, evs, nvtx=True)
    torch.cuda.synchronize()
    launches = lc.kernel_launches() - launches0
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    # profiling pass (same steps, graphs with in-graph phase events)
    plan.timing(reset=True)
    mac_steps = run_pass(graphs_timed)
    torch.cuda.synchronize()
    phases = plan.timing(reset=True)
    for g in list(graphs.values()) + list(graphs_timed.values()):
        g.close()
    fdiff_stats = None
    if args.fdiff:
        # the profiling pass ended on the same step as the timed one: its maps are in place
        f = out_fdiff.double()
        lit = out > 0
        fa = f[lit].abs()
        fdiff_stats = {"step": done_steps[-1], "cells_with_flux": int(lit.sum()),
                       "mean_abs": float(fa.mean()) if fa.numel() else None,
                       "p50_abs": float(fa.kthvalue(max(1, fa.numel() // 2))[0]) if fa.numel() else None,
                       "p99_abs": float(fa.kthvalue(max(1, int(0.99 * fa.numel())))[0]) if fa.numel() else None,
                       "frac_over_10pct": float((fa > 0.1).double().mean()) if fa.numel() else None}
    per_step_ms = np.array([a.elapsed_time(b) for a, b in evs])
    t_total = float(per_step_ms.sum()) / 1e3
    t_max = max_over_ranks(t_total, dev)
    value = world * args.steps / t_max
    mac_cells = sum(nk * work[s][0] for s in done_steps)

    # roofline of the dominant kernel (shell MAC fused with the inverse x pass):
    # algorithmic bytes = ring reads (8 B per k per non-empty shell) + the
    # complex write (8 B per k) + one read of the step's Ghat wedge table
    mac_ms, mac_launches = phases["mac_x"]
    W = plan.wedge_size
    hb = 4 if w.history else 8
    mac_bytes = sum(nk * (hb * work[s][0] + 8) + W * 4 * work[s][1] for s in mac_steps)
    import json as _json

    peaks = {}
    try:
        peaks = _json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    mac_gbs = mac_bytes / (mac_ms / 1e3) / 1e9 if mac_ms > 0 else None
    # the captured DRAM traffic is for the Lyman-Werner kernel's shell count
    traffic, traffic_src = mac_traffic(args.workload) if args.kernel == "lw" else (None, None)
    phase_share = {k: round(v[0] / max(1e-12, sum(x[0] for x in phases.values())), 4) for k, v in phases.items()}

    # end to end through the public API: pinned host inputs, host output
    pinned = []
    for s in range(T):
        pos, lum = w.cat.active(s)
        pinned.append((torch.from_numpy(pos).pin_memory(), torch.from_numpy(lum).pin_memory()))
    host_out = torch.empty((w.n,) * 3, dtype=torch.float32).pin_memory()
    host_fdiff = torch.empty((w.n,) * 3, dtype=torch.float32).pin_memory() if args.fdiff else None

    def e2e_field(s):
        if not args.fdiff:
            plan.field(s, host_out)  # synchronises and copies to the host
            return
        plan.field(s, out)
        fdiff_after(s)
        host_out.copy_(out, non_blocking=True)
        host_fdiff.copy_(out_fdiff, non_blocking=True)
        stream.synchronize()

    refill()
    e_cursor = t0
    for _ in range(max(3, args.warmup)):
        plan.push(e_cursor, *pinned[e_cursor])
        e2e_field(e_cursor)
        e_cursor += 1
        if e_cursor == T:
            refill()
            e_cursor = t0
    e2e_t = 0.0
    h2d = 0
    for i in range(args.steps):
        s = e_cursor
        if s == t0:
            refill()
        flush.zero_()
        torch.cuda.synchronize()
        tic = time.perf_counter()
        plan.push(s, *pinned[s])
        e2e_field(s)
        e2e_t += time.perf_counter() - tic
        h2d += pinned[s][0].numel() * 8 + pinned[s][1].numel() * 8
        e_cursor = t0 + (s + 1 - t0) % (T - t0)
    e2e_t = max_over_ranks(e2e_t, dev)
    e2e = {"value": world * args.steps / e2e_t, "unit": UNIT, "h2d_bytes_per_step": int(h2d // args.steps),
           "d2h_bytes_per_step": int(w.n ** 3 * 4 * (2 if args.fdiff else 1))}
    e2e_pipe = None
    if args.e2e_pipelined and not args.fdiff:
        # the same steps and copies through field_async: step i's output copy
        # drains while step i+1 computes; refills (history restarts) untimed
        outs = [torch.empty((w.n,) * 3, dtype=torch.float32).pin_memory() for _ in range(2)]
        refill()
        torch.cuda.synchronize()
        p_t, prev, cur = 0.0, 0, t0
        tic = time.perf_counter()
        for i in range(args.steps):
            if i and cur == t0:
                if prev:
                    plan.wait(prev)
                p_t += time.perf_counter() - tic
                refill()
                torch.cuda.synchronize()
                prev = 0
                tic = time.perf_counter()
            plan.push(cur, *pinned[cur])
            tk = plan.field_async(cur, outs[i % 2])
            if prev:
                plan.wait(prev)
            prev = tk
            cur = t0 + (cur + 1 - t0) % (T - t0)
        plan.wait(prev)
        p_t += time.perf_counter() - tic
        p_t = max_over_ranks(p_t, dev)
        e2e_pipe = {"value": world * args.steps / p_t, "unit": UNIT, "h2d_bytes_per_step": e2e["h2d_bytes_per_step"],
                    "d2h_bytes_per_step": e2e["d2h_bytes_per_step"], "api": "Plan.push + Plan.field_async/wait",
                    "l2": "not flushed between steps"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        if args.workload == "c2":
            rate, spent, desc = oracle_field_rate(w, [10, 20, 30, 41, 50, 63], cells_per_step=131072)
        else:
            rate, spent, desc = oracle_field_rate(w, [w.steps.n_steps - 1], cells_per_step=2048)
        if args.near != "ngp" or args.fdiff:
            desc += "; the sample times the retarded field alone (cell-centred near field, no f_diff map)"
        cpu = {"value": rate, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle", "sample": desc,
               "seconds": round(spent, 2)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32" if w.history else "f32", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}", "grid": w.n,
                       "box_mpc": w.box, "steps_in_run": T, "timed_window": [t0, T], "ring_slots": plan.n_ring,
                       "history": "bf16" if w.history else "fp32",
                       "mac_kernel": dict(sorted(mac_choice.items(), key=lambda kv: int(kv[0][1:]))),
                       "l2": f"flushed between timed steps "
                       f"({args.flush_mb} MB write outside the events)", "inputs": "device-resident", **variant},
            "cell_shell_mac_per_s": world * mac_cells / t_max,
            "latency_ms": {"p50": float(np.percentile(per_step_ms, 50)), "p99": float(np.percentile(per_step_ms, 99))},
            "roofline": {"bound": "hbm", "kernel": "shell-MAC phase: k_cols<N,+1,MAC> (gather) or k_mac_tma + "
                         "Nyquist k_cols (bulk), fused with the inverse x pass",
                         "achieved": mac_gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": (mac_gbs / hbm_peak) if mac_gbs else None,
                         "traffic": traffic, "traffic_source": traffic_src,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)",
                         "bytes_per_launch": mac_bytes / max(1, len(mac_steps)),
                         "ms_per_launch": mac_ms / max(1, len(mac_steps))},
            "phase_ms_per_step": {k: v[0] / max(1, len(mac_steps)) for k, v in phases.items()},
            "launch": "one CUDA graph replay per step (push + field captured once per observed step); "
                      "phase times from a second pass of graphs with in-graph events",
            "phase_share": phase_share,
            "clocks": clocks,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "cpu_baseline": cpu,
        }
        if fdiff_stats is not None:
            line["fdiff"] = fdiff_stats
        if e2e_pipe is not None:
            line["e2e_pipelined"] = e2e_pipe
        print(json.dumps(line))
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
