"""Step graphs with the gather MAC: the push leaves its x pass into the
history ring to the field's MAC kernel, which forward-transforms the newest
slice's tile, stores it to its ring slot and uses it as lookback 0.  Graph
replays over many steps (each step reading ring slots the fused kernel
wrote) equal the eager push + field bit for bit, FP32 and BF16 history, and
the fields match the FP64 oracle."""
import dataclasses

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


def ulp32(x):
    a = np.abs(np.asarray(x, dtype=np.float64))
    return np.exp2(np.floor(np.log2(np.maximum(a, np.finfo(np.float32).tiny))) - 23)


@pytest.mark.parametrize("n,hist,dep", [(32, synth.HISTORY_FP32, lc.DEPOSIT_NGP), (64, synth.HISTORY_BF16, lc.DEPOSIT_NGP),
                                        (128, synth.HISTORY_FP32, lc.DEPOSIT_NGP), (96, synth.HISTORY_BF16, lc.DEPOSIT_NGP),
                                        (64, synth.HISTORY_FP32, lc.DEPOSIT_CIC)])
@pytest.mark.parametrize("near", [lc.NEAR_NONE, lc.NEAR_NGP])
def test_graph_with_fused_x_pass_equals_eager(monkeypatch, n, hist, dep, near):
    monkeypatch.setenv("LC_MAC_VARIANT", "gather")
    steps = 8
    w = synth.small(n=n, box=0.78125 * n, n_steps=steps, n_src=200, seed=4100 + n, clustered=True, history=hist)
    w = dataclasses.replace(w, deposit=dep)
    eager = lc.Plan.from_workload(w, near_mode=near)
    graph = lc.Plan.from_workload(w, near_mode=near)
    graph.prepare(0, steps)
    outs = [torch.full((n,) * 3, float("nan"), device="cuda") for _ in range(steps)]
    srcs = [(torch.from_numpy(w.cat.active(s)[0]).cuda(), torch.from_numpy(w.cat.active(s)[1]).cuda())
            for s in range(steps)]
    graphs = [graph.graph(s, *srcs[s], outs[s]) for s in range(steps)]
    for s in range(steps):
        eager.push(s, *srcs[s])
        a = eager.field(s).cpu().numpy()
        graphs[s].launch()
        b = outs[s].cpu().numpy()
        assert np.isfinite(b).all(), s
        if near == lc.NEAR_NONE:
            assert np.array_equal(a.view(np.uint32), b.view(np.uint32)), s
        else:  # the near fold adds FP64 atomics in any order
            assert (np.abs(a.astype(np.float64) - b) <= 2 * ulp32(a) + 1e-30).all(), s
    # the last field against the FP64 oracle (with the near split, as every
    # default field; without it the innermost shell's largest values pass
    # through the history's precision)
    if near != lc.NEAR_NGP:
        return
    P = oracle.Problem.from_workload(w)
    cells = synth.sample_cells(4200 + n, n, 1500)
    ref = oracle.field_for(P, w.cat, steps - 1, cells=cells)
    got = outs[-1].cpu().numpy().reshape(-1)[cells].astype(np.float64)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= (1e-5 if hist == synth.HISTORY_FP32 else 5e-3), rel
