"""Launch overlap (programmatic dependent launch of the per-step kernels)
changes scheduling only: the field of a step computed with it on equals the
field computed with it off, eager and captured in a step graph, for the
register FFT passes (N <= 192) and the tiled passes with the warp-specialised
MAC (N = 256, BF16 history)."""
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
    prev = lc.launch_overlap(-1)
    yield
    lc.launch_overlap(int(prev))


def ulp32(x):
    a = np.abs(np.asarray(x, dtype=np.float64))
    return np.exp2(np.floor(np.log2(np.maximum(a, np.finfo(np.float32).tiny))) - 23)


def field_at(w, last, overlap, near_mode, graph):
    lc.launch_overlap(int(overlap))
    p = lc.Plan.from_workload(w, near_mode=near_mode)
    for s in range(last):
        pos, lum = w.cat.active(s)
        p.push(s, torch.from_numpy(pos).cuda(), torch.from_numpy(lum).cuda())
    pos, lum = w.cat.active(last)
    pos, lum = torch.from_numpy(pos).cuda(), torch.from_numpy(lum).cuda()
    if graph:
        out = torch.full((w.n,) * 3, float("nan"), device="cuda")
        g = p.graph(last, pos, lum, out)
        g.launch()
        torch.cuda.synchronize()
        r = out.cpu().numpy()
        g.close()
    else:
        p.push(last, pos, lum)
        r = p.field(last).cpu().numpy()
    p.close()
    return r


CASES = [
    (64, 90.0, synth.HISTORY_FP32, 6),
    (128, 150.0, synth.HISTORY_FP32, 6),
    (256, 200.0, synth.HISTORY_BF16, 4),
]


@pytest.mark.parametrize("n,box,hist,steps", CASES)
@pytest.mark.parametrize("graph", [False, True])
def test_overlap_bit_identical_without_near_split(n, box, hist, steps, graph):
    w = synth.small(n=n, box=box, n_steps=steps, n_src=300, seed=900 + n, clustered=True, history=hist)
    last = steps - 1
    a = field_at(w, last, 0, lc.NEAR_NONE, graph)
    b = field_at(w, last, 1, lc.NEAR_NONE, graph)
    assert np.isfinite(a).all()
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.parametrize("n,box,hist,steps", CASES)
def test_overlap_with_near_split(n, box, hist, steps):
    w = synth.small(n=n, box=box, n_steps=steps, n_src=300, seed=950 + n, clustered=True, history=hist)
    last = steps - 1
    a = field_at(w, last, 0, lc.NEAR_NGP, True)
    b = field_at(w, last, 1, lc.NEAR_NGP, True)
    c = field_at(w, last, 1, lc.NEAR_NGP, False)
    # the near fold adds FP64 atomics in any order: at most an ulp or two apart
    for x in (b, c):
        assert (np.abs(a.astype(np.float64) - x) <= 2 * ulp32(a) + 1e-30).all()
