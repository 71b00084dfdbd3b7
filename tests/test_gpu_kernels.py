"""The CUDA path with the second radial kernel (exponential attenuation with a
cut-off, the generic dilution factor of Eq. 7) against the FP64 oracle: full
fields for equal-time and equal-conformal-time steps, FP32 and BF16 history."""
import numpy as np
import pytest

import oracle
import paper_1502_02294_gb300 as lc
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_L2, FP32_MAX, BF16_L2 = 1e-5, 1e-4, 5e-3
KERN = (lc.KERNEL_EXP, 25.0, 60.0)  # exp(-r / 25 Mpc), cut off at 60 Mpc


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


def _run(w, steps, check):
    plan = lc.Plan.from_workload(w)
    out = {}
    for s in steps:
        pos, lum = w.cat.active(s)
        plan.push(s, torch.from_numpy(pos).cuda(), torch.from_numpy(lum).cuda())
        if s in check:
            out[s] = plan.field(s).cpu().numpy()
    plan.close()
    return out


@pytest.mark.parametrize("history", [synth.HISTORY_FP32, synth.HISTORY_BF16])
def test_exp_kernel_equal_time_full_grid(history):
    w = synth.small(n=32, box=75.0, n_steps=8, n_src=150, subsamples=2, clustered=True, seed=2601,
                    z_start=16.0, z_end=15.0, history=history)
    w.kernel = KERN
    P = oracle.Problem.from_workload(w)
    assert P.active_shells(7) >= 3
    out = _run(w, range(8), {4, 7})
    for s, J in out.items():
        ref = oracle.field_for(P, w.cat, s)
        rel, mx = _errors(J, ref)
        if history == synth.HISTORY_FP32:
            assert rel <= FP32_L2 and mx <= FP32_MAX, (s, rel, mx)
        else:
            assert rel <= BF16_L2, (s, rel)


def test_exp_kernel_equal_tau_steps_ring_full():
    # equal conformal-time steps of width r_max / 6: six shells up to the cut-off
    st = synth.StepSpec(synth.STEPS_EQUAL_TAU, 10, z_end=15.0, n_shell=6)
    cat = synth.make_catalogue(synth.SEED_BASE + 2602, 200, 64.0, 10, clustered=True, n_centres=8, sigma=3.0)
    w = synth.Workload("exp64", 64, 64.0, 0.31, 0.68, st, 2, synth.HISTORY_FP32, cat, kernel=KERN)
    P = oracle.Problem.from_workload(w)
    assert P.active_shells(9) == 6
    plan = lc.Plan.from_workload(w)
    lo, hi, rh = plan.shells(9)
    olo, ohi, orh = P.shells(9)
    assert rh == KERN[2] and orh == KERN[2]
    assert np.allclose(lo, olo, rtol=1e-12, atol=1e-12) and np.allclose(hi, ohi, rtol=1e-12)
    plan.close()
    out = _run(w, range(10), {9})
    ref = oracle.field_for(P, w.cat, 9)
    rel, mx = _errors(out[9], ref)
    assert rel <= FP32_L2 and mx <= FP32_MAX, (rel, mx)


def test_exp_kernel_invalid_parameters_refused():
    w = synth.small(n=16, box=40.0, n_steps=4)
    for bad in [(lc.KERNEL_EXP, 0.0, 50.0), (lc.KERNEL_EXP, 20.0, -1.0), (7, 1.0, 1.0)]:
        with pytest.raises(lc.LCError):
            lc.Plan.from_workload(w, kernel=bad)
