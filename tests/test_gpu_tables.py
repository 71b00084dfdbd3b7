"""The Green's-function table budget: tables of other observing steps are
freed to stay under it, rebuilt identically when needed again, and tables
held by a graph are never freed."""
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


def _w():
    return synth.small(n=32, box=60.0, n_steps=8, n_src=120, seed=77, clustered=True, z_start=16.0, z_end=15.0)


def _sizes(w):
    sizes = []
    for s in range(8):
        p = lc.Plan.from_workload(w)
        p.prepare(s, s + 1)
        sizes.append(p.table_bytes)
        p.close()
    return sizes


def test_budget_evicts_and_rebuilds_identically():
    w = _w()
    sizes = _sizes(w)
    assert min(sizes) > 0 and max(sizes) > min(sizes)  # the slice count grows with the step
    ref = lc.Plan.from_workload(w)
    tight = lc.Plan.from_workload(w)
    tight.set_table_budget(max(sizes))  # room for one table
    for s in range(8):
        pos, lum = w.cat.active(s)
        for p in (ref, tight):
            p.push(s, torch.from_numpy(pos).cuda(), torch.from_numpy(lum).cuda())
        a = ref.field(s).cpu().numpy()
        b = tight.field(s).cpu().numpy()
        assert np.array_equal(a, b), s
        assert tight.table_bytes == sizes[s]  # only the current step's table is left
    assert ref.table_bytes == sum(sizes)
    # tables evicted earlier are rebuilt bit for bit
    g_ref, g0_ref = ref.green_wedge(2, 1)
    g, g0 = tight.green_wedge(2, 1)
    assert np.array_equal(g, g_ref) and g0 == g0_ref
    ref.close()
    tight.close()


def test_graph_pins_its_table():
    w = _w()
    sizes = _sizes(w)
    p = lc.Plan.from_workload(w)
    p.set_table_budget(1)  # no room at all: only pinned tables and the newest survive
    pos, lum = w.cat.active(0)
    dpos, dlum = torch.from_numpy(pos).cuda(), torch.from_numpy(lum).cuda()
    out = torch.empty((w.n,) * 3, dtype=torch.float32, device="cuda")
    g = p.graph(0, dpos, dlum, out)
    p.prepare(1, 8)
    assert p.table_bytes == sizes[0] + sizes[7]
    g.close()
    p.prepare(3, 4)  # rebuild step 3: steps 0 and 7 go
    assert p.table_bytes == sizes[3]
    p.set_table_budget(0)
    p.prepare(0, 8)
    assert p.table_bytes == sum(sizes)
    p.close()


def test_graph_keeps_its_near_lists_when_they_grow():
    # the second graph's step has more sources than the near-field lists the
    # first graph was captured with: the lists grow, and the first graph must
    # still replay on the lists it holds
    w = _w()
    rng = np.random.default_rng(5)
    src = []
    for n in (40, 3000):
        src.append((rng.uniform(0.0, w.box, (n, 3)), rng.uniform(0.5, 2.0, n)))
    ref = lc.Plan.from_workload(w)
    want = []
    for s, (pos, lum) in enumerate(src):
        ref.push(s, torch.from_numpy(pos).cuda(), torch.from_numpy(lum).cuda())
        want.append(ref.field(s).cpu().numpy())
    ref.close()
    p = lc.Plan.from_workload(w)
    dev = [(torch.from_numpy(pos).cuda(), torch.from_numpy(lum).cuda()) for pos, lum in src]
    outs = [torch.empty((w.n,) * 3, dtype=torch.float32, device="cuda") for _ in src]
    graphs = [p.graph(s, *dev[s], outs[s]) for s in range(2)]
    for _ in range(2):
        p.reset()
        for g in graphs:
            g.launch()
        torch.cuda.synchronize()
        for s in range(2):
            got = outs[s].cpu().numpy()
            assert np.allclose(got, want[s], rtol=1e-6, atol=1e-6 * np.abs(want[s]).max()), s
    for g in graphs:
        g.close()
    p.close()
