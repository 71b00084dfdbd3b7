"""Batched uneven instances (one CUDA graph) and the continuous-batching
server: every result equals the same instance computed alone, and every
served field matches the FP64 oracle."""
import numpy as np
import pytest

import oracle
import paper_1502_02294_gb300 as lc
import synth
from test_gpu_parity import BF16_L2, FP32_L2, FP32_MAX, errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    lc.build()
    oracle.build()


def ulp32(x):
    a = np.abs(np.asarray(x, dtype=np.float64))
    return np.exp2(np.floor(np.log2(np.maximum(a, np.finfo(np.float32).tiny))) - 23)


def instances():
    out = []
    for k, (n, box, hist) in enumerate([(32, 60.0, synth.HISTORY_FP32), (64, 90.0, synth.HISTORY_BF16),
                                        (96, 110.0, synth.HISTORY_FP32)]):
        w = synth.small(n=n, box=box, n_steps=6, n_src=150 + 50 * k, seed=500 + k, clustered=True, history=hist)
        out.append(w)
    return out


def test_batch_graph_equals_instances_alone():
    ws = instances()
    steps = [3, 4, 5]
    # alone: each plan stepped with the plain API
    alone = []
    for w, last in zip(ws, steps):
        p = lc.Plan.from_workload(w)
        for s in range(last + 1):
            pos, lum = w.cat.active(s)
            p.push(s, torch.from_numpy(pos).cuda(), torch.from_numpy(lum).cuda())
        alone.append(p.field(last).cpu().numpy())
        p.close()
    # batched: history pushed alone up to last-1, then the last step of all
    # three instances as one graph replay
    plans, srcs, outs = [], [], []
    for w, last in zip(ws, steps):
        p = lc.Plan.from_workload(w)
        for s in range(last):
            pos, lum = w.cat.active(s)
            p.push(s, torch.from_numpy(pos).cuda(), torch.from_numpy(lum).cuda())
        pos, lum = w.cat.active(last)
        srcs.append((torch.from_numpy(pos).cuda(), torch.from_numpy(lum).cuda()))
        outs.append(torch.full((w.n,) * 3, float("nan"), device="cuda"))
        plans.append(p)
    g = lc.BatchGraph(plans, steps, srcs, outs)
    g.launch()
    torch.cuda.synchronize()
    for a, o, w in zip(alone, outs, ws):
        b = o.cpu().numpy()
        d = np.abs(a.astype(np.float64) - b)
        # the near-field fold adds FP64 atomics in any order: at most an ulp apart
        assert (d <= 2 * ulp32(a) + 1e-30).all()
    with pytest.raises(lc.LCError):
        g.launch()  # the same steps again: out of order
    g.close()
    for p in plans:
        p.close()


def test_server_results_alone_equal_mixed():
    from paper_1502_02294_gb300.serve import Request, Server

    ws = instances()

    def serve(names, arrival_spread):
        srv = Server(hbm_budget_bytes=40 << 30, keep_outputs=True)
        reqs, arr = [], []
        rng = np.random.default_rng(1)
        for k, w in enumerate(ws):
            name = f"s{k}"
            if name not in names:
                continue
            srv.add_simulation(name, w, 2, 5, fill=lambda p, w=w: [p.push(s, *w.cat.active(s)) for s in range(2)])
            for s in range(2, 6):
                pos, lum = w.cat.active(s)
                reqs.append(Request(name, s, pos, lum))
                arr.append(rng.uniform(0, arrival_spread))
        # requests of one simulation must arrive in step order
        for name in names:
            idx = [i for i, r in enumerate(reqs) if r.sim == name]
            ts = sorted(arr[i] for i in idx)
            for i, t in zip(idx, ts):
                arr[i] = t
        stats = srv.run_stream(reqs, arr)
        torch.cuda.synchronize()
        return {(r.sim, r.step): r.out.cpu().numpy() for r in srv.completed}, stats

    mixed, st = serve({"s0", "s1", "s2"}, 0.01)
    assert st["requests"] == 12 and st["p99_ms"] >= st["p50_ms"] > 0
    # every served field against the FP64 oracle (Eq. 11), full grid
    for k, w in enumerate(ws):
        P = oracle.Problem.from_workload(w)
        for s in range(2, 6):
            rel, mx, raw = errors(mixed[(f"s{k}", s)], oracle.field_for(P, w.cat, s))
            if w.history == synth.HISTORY_BF16:
                assert rel <= BF16_L2, (k, s, rel)
            else:
                assert rel <= FP32_L2 and mx <= FP32_MAX, (k, s, rel, mx, raw)
    for k, w in enumerate(ws):
        alone, _ = serve({f"s{k}"}, 0.0)
        for key, a in alone.items():
            b = mixed[key]
            assert (np.abs(a.astype(np.float64) - b) <= 2 * ulp32(a) + 1e-30).all(), key


def test_server_admits_by_hbm_budget():
    from paper_1502_02294_gb300.serve import Request, Server

    ws = instances()[:2]
    need = [Server.plan_bytes(w, 2, 5) for w in ws]
    srv = Server(hbm_budget_bytes=max(need) + 1)  # room for one simulation at a time
    for k, w in enumerate(ws):
        srv.add_simulation(f"s{k}", w, 2, 5, fill=lambda p, w=w: [p.push(s, *w.cat.active(s)) for s in range(2)])
    admitted = [n for n, s in srv.sims.items() if s.plan is not None]
    assert len(admitted) == 1 and len(srv.waiting) == 1
    reqs = [Request(f"s{k}", s, *w.cat.active(s)) for k, w in enumerate(ws) for s in range(2, 6)]
    st = srv.run_stream(reqs, [0.0] * len(reqs))
    assert st["requests"] == 8 and srv.used == 0
