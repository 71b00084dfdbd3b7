"""The particle-mesh hybrid near the sources (Discussion): with near_mode =
NEAR_SUBCELL the innermost slice's near cube of every source comes from the
source's own position.  The CUDA path against the FP64 oracle's definition
(full fields), the centred limit, the kernel plug-in, checkpoints and errors."""
import numpy as np
import pytest

import oracle
import paper_1502_02294_gb300 as lc
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_L2, FP32_MAX = 1e-5, 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    lc.build()
    oracle.build()


def _errors(J, ref):
    J = np.asarray(J, dtype=np.float64)
    a = np.abs(ref)
    ulp = np.exp2(np.floor(np.log2(np.maximum(a, np.finfo(np.float32).tiny))) - 23)
    rel = np.linalg.norm(J - ref) / np.linalg.norm(ref)
    mx = np.maximum(np.abs(J - ref) - 2.0 * ulp, 0.0).max() / a.mean()
    return rel, mx


def _fields(w, steps, check, near_mode):
    plan = lc.Plan.from_workload(w, near_mode=near_mode)
    out = {}
    for s in steps:
        pos, lum = w.cat.active(s)
        plan.push(s, torch.from_numpy(pos).cuda(), torch.from_numpy(lum).cuda())
        if s in check:
            out[s] = plan.field(s).cpu().numpy()
    plan.close()
    return out


@pytest.mark.parametrize("kernel", [None, (lc.KERNEL_EXP, 25.0, 60.0)])
def test_subcell_near_field_against_oracle(kernel):
    w = synth.small(n=32, box=60.0, n_steps=8, n_src=150, subsamples=4, seed=3301, z_start=16.0, z_end=15.0)
    w.kernel = kernel
    P = oracle.Problem.from_workload(w)
    out = _fields(w, range(8), {3, 7}, lc.NEAR_SUBCELL)
    for s, J in out.items():
        ref = oracle.hybrid_field_for(P, w.cat, s)
        rel, mx = _errors(J, ref)
        assert rel <= FP32_L2 and mx <= FP32_MAX, (s, rel, mx)
        # the hybrid differs from the NGP field near the sources
        assert np.linalg.norm(ref - oracle.field_for(P, w.cat, s)) > 1e-3 * np.linalg.norm(ref)


def test_sources_on_cell_centres_give_the_ngp_field():
    w = synth.small(n=32, box=60.0, n_steps=6, n_src=120, subsamples=4, seed=3302)
    l = w.box / w.n
    w.cat.pos = np.round(w.cat.pos / l) * l % w.box
    a = _fields(w, range(6), {5}, lc.NEAR_NGP)[5]
    b = _fields(w, range(6), {5}, lc.NEAR_SUBCELL)[5]
    rel, mx = _errors(b, a.astype(np.float64))
    assert rel <= FP32_L2 and mx <= FP32_MAX, (rel, mx)


def test_subcell_checkpoint():
    w = synth.small(n=32, box=60.0, n_steps=6, n_src=100, subsamples=4, seed=3303)
    a = lc.Plan.from_workload(w, near_mode=lc.NEAR_SUBCELL)
    for s in range(4):
        pos, lum = w.cat.active(s)
        a.push(s, torch.from_numpy(pos).cuda(), torch.from_numpy(lum).cuda())
    buf = a.save()
    b = lc.Plan.from_workload(w, near_mode=lc.NEAR_SUBCELL)
    b.load(buf)
    ja, jb = a.field(3).cpu().numpy(), b.field(3).cpu().numpy()
    rel, mx = _errors(jb, ja.astype(np.float64))
    assert rel <= 1e-7 and mx <= 1e-6
    # a checkpoint of the NGP mode does not load into a sub-cell plan
    c = lc.Plan.from_workload(w)
    with pytest.raises(lc.LCError):
        c.load(buf)
    for p in (a, b, c):
        p.close()


def test_subcell_near_field_bf16_history():
    # the sub-cell near cube is summed in FP64 from the sources' positions
    # whatever the history format: with the BF16 history the field meets the
    # BF16 bound against the FP64 oracle, and stays close to the FP32-history
    # field of the same mode
    w = synth.small(n=32, box=60.0, n_steps=8, n_src=150, subsamples=4, seed=3304, z_start=16.0, z_end=15.0,
                    history=synth.HISTORY_BF16)
    P = oracle.Problem.from_workload(w)
    got = _fields(w, range(8), {3, 7}, lc.NEAR_SUBCELL)
    w32 = synth.small(n=32, box=60.0, n_steps=8, n_src=150, subsamples=4, seed=3304, z_start=16.0, z_end=15.0)
    f32 = _fields(w32, range(8), {3, 7}, lc.NEAR_SUBCELL)
    for s, J in got.items():
        ref = oracle.hybrid_field_for(P, w.cat, s)
        rel = np.linalg.norm(J.astype(np.float64) - ref) / np.linalg.norm(ref)
        assert rel <= 5e-3, (s, rel)
        d = np.linalg.norm(J.astype(np.float64) - f32[s]) / np.linalg.norm(f32[s])
        assert d <= 5e-3, (s, d)
