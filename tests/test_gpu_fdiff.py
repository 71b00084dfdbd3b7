"""The light-cone vs instantaneous fractional difference of Section 3 (after
Eq. 18), f_diff = (J_instant - J) / J, from the CUDA path against the FP64
oracle's two fields."""
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


def test_fdiff_map_against_oracle():
    # sources live 1-3 steps, so the source field evolves fast and f_diff is large
    w = synth.small(n=32, box=75.0, n_steps=8, n_src=200, seed=1812, clustered=True, life=(1, 3))
    P = oracle.Problem.from_workload(w)
    plan = lc.Plan.from_workload(w)
    for s in range(8):
        pos, lum = w.cat.active(s)
        plan.push(s, torch.from_numpy(pos).cuda(), torch.from_numpy(lum).cuda())
    s = 7
    J = plan.field(s)
    Ji = plan.instant_field(s)
    f = lc.fdiff_map(J, Ji)
    torch.cuda.synchronize()
    got = f.cpu().numpy()
    # the kernel's own arithmetic: FP64 difference and quotient of its inputs, rounded once
    a, b = J.cpu().numpy().astype(np.float64), Ji.cpu().numpy().astype(np.float64)
    own = np.where((a == 0) & (b == 0), 0.0, (b - a) / np.where(a == 0, 1.0, a)).astype(np.float32)
    assert np.array_equal(got, own)
    # against the oracle.  f = Ji/J - 1 carries the relative errors of both
    # fields, each within 1e-4 of the mean field (the FP32 max criterion), so
    # |df| <= 2e-4 (1 + |f|) mean(J) / J, checked where J > 1e-2 mean(J)
    ref = oracle.field_for(P, w.cat, s)
    ref_i = oracle.instant_field_for(P, w.cat, s)
    fo = (ref_i - ref) / ref
    m = ref > 1e-2 * ref.mean()
    assert np.abs(fo[m]).mean() > 1e-2  # the light-cone effect is visible
    tol = 2e-4 * (1.0 + np.abs(fo[m])) * ref.mean() / ref[m]
    assert np.all(np.abs(got[m] - fo[m]) <= tol)
    plan.close()


def test_fdiff_zero_cells_and_argument_errors():
    z = torch.zeros(64, device="cuda")
    one = torch.ones(64, device="cuda")
    assert torch.equal(lc.fdiff_map(z, z), z)
    assert torch.isinf(lc.fdiff_map(z, one)).all()
    assert torch.equal(lc.fdiff_map(one, one), z)
    with pytest.raises(lc.LCError):
        lc._check(lc._lib().lc_fdiff_map(4, None, None, None, None), "lc_fdiff_map")
    host = np.zeros(4, dtype=np.float32)
    with pytest.raises(lc.LCError):
        lc._check(lc._lib().lc_fdiff_map(4, host.ctypes.data, host.ctypes.data, host.ctypes.data, None), "lc_fdiff_map")


@pytest.mark.parametrize("hist,tol", [(synth.HISTORY_FP32, 1e-5), (synth.HISTORY_BF16, 5e-3)])
def test_instant_field_many_shells(hist, tol):
    # Eq. 18 through ten shells: every shell sees the observing step's sources
    st = synth.StepSpec(synth.STEPS_EQUAL_TAU, 14, z_end=15.0, n_shell=10)
    cat = synth.make_catalogue(4242, 150, 60.0, 14, clustered=True, n_centres=5, sigma=3.0, lum_kind="lognormal",
                               life=(1, 3))
    w = synth.Workload("ten-shells", 32, 60.0, 0.31, 0.68, st, 4, hist, cat)
    P = oracle.Problem.from_workload(w)
    plan = lc.Plan.from_workload(w)
    for s in range(14):
        pos, lum = w.cat.active(s)
        plan.push(s, torch.from_numpy(pos).cuda(), torch.from_numpy(lum).cuda())
        if s in (9, 13):
            assert len(plan.shells(s)[0]) == 10
            Ji = plan.instant_field(s).cpu().numpy()
            ref_i = oracle.instant_field_for(P, w.cat, s)
            rel = np.linalg.norm(Ji - ref_i) / np.linalg.norm(ref_i)
            assert rel <= tol, (s, rel)
            # a second call reuses the step's summed table: the same field
            assert np.array_equal(plan.instant_field(s).cpu().numpy(), Ji)
            # and the retarded field of the step is unchanged by it
            J = plan.field(s).cpu().numpy()
            ref = oracle.field_for(P, w.cat, s)
            assert np.linalg.norm(J - ref) / np.linalg.norm(ref) <= tol
    plan.close()
