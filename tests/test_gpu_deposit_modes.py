"""The plan options of the boundary's step description, on the GPU against
the FP64 oracle: cloud-in-cell deposit (bit-exact int64 grid, then fields),
the Lyman-Werner kernel cut at Section 1's rough horizon 100[21/(1+z_s)]^0.5,
and the cap on lookback slices per step.

Tolerances as in test_gpu_parity: FP32 history relative L2 <= 1e-5 and the
max criterion beyond two FP32 ulps <= 1e-4 of the mean field; BF16 history
relative L2 <= 5e-3; deposits bit-exact.
"""
import dataclasses

import numpy as np
import pytest

import oracle
import paper_1502_02294_gb300 as lc
import synth
from test_gpu_parity import BF16_L2, FP32_L2, FP32_MAX, errors, run_steps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    lc.build()
    oracle.build()


CIC = lc.DEPOSIT_CIC


# ------------------------------------------------------------------ CIC deposit
def test_cic_deposit_bit_exact_against_oracle():
    w = synth.config("c2")
    for s in (0, 17, 40):
        pos, lum = w.cat.active(s)
        g, S, tot = lc.deposit_grid(w.n, w.box, pos, lum, deposit=CIC)
        go, So, to = oracle.deposit_cic_fixed(w.n, w.box, pos, lum)
        assert S == So and tot == to and np.array_equal(g, go)
        gd = torch.zeros((w.n,) * 3, dtype=torch.int64, device="cuda")
        _, S2, t2 = lc.deposit_grid(w.n, w.box, torch.from_numpy(pos).cuda(), torch.from_numpy(lum).cuda(), out=gd,
                                    deposit=CIC)
        assert S2 == So and t2 == to and np.array_equal(gd.cpu().numpy(), go)


def test_cic_deposit_edge_positions_and_order():
    N, box = 16, 32.0
    l = box / N
    rng = np.random.default_rng(15)
    pos = np.concatenate([
        rng.uniform(-3 * box, 4 * box, size=(400, 3)),
        rng.integers(-40, 60, size=(50, 3)) * l,                        # cell centres
        rng.integers(-40, 60, size=(50, 3)) * l + 0.5 * l,              # midpoints
        np.array([[0.0, 0.0, 0.0], [box, box, box], [-1e-300, 0.5 * l, 1.5 * l], [(N - 1e-9) * l, 1e-12, 7.5 * l],
                  [1e6 + 0.3, -1e6 - 0.7, 12345.678]]),
    ])
    lum = 10.0 ** rng.normal(0, 2, size=pos.shape[0])
    lum[7] = 0.0
    g, S, t = lc.deposit_grid(N, box, pos, lum, deposit=CIC)
    go, So, to = oracle.deposit_cic_fixed(N, box, pos, lum)
    assert np.array_equal(g, go) and S == So and t == to and g.sum() == t
    perm = rng.permutation(pos.shape[0])
    g2, S2, t2 = lc.deposit_grid(N, box, pos[perm], lum[perm], deposit=CIC)
    assert np.array_equal(g2, go) and t2 == to
    ge, Se, te = lc.deposit_grid(N, box, np.zeros((0, 3)), np.zeros(0), deposit=CIC)
    assert te == 0 and not ge.any()


# ------------------------------------------------------------------ CIC fields
def test_cic_field_c1_every_step_full_grid():
    w = dataclasses.replace(synth.config("c1"), deposit=CIC)
    P = oracle.Problem.from_workload(w)
    plan = lc.Plan.from_workload(w)
    out = run_steps(plan, w.cat, range(8), set(range(8)))
    for s, J in out.items():
        ref = oracle.field_for(P, w.cat, s)
        rel, mx, raw = errors(J, ref)
        assert rel <= FP32_L2 and mx <= FP32_MAX, (s, rel, mx, raw)
    # the assignment matters: the NGP field differs
    ngp = oracle.field_for(oracle.Problem.from_workload(synth.config("c1")), w.cat, 7)
    assert np.linalg.norm(ngp - out[7]) > 1e-3 * np.linalg.norm(ngp)
    plan.close()


@pytest.mark.parametrize("n,box,hist", [(96, 120.0, synth.HISTORY_FP32), (64, 80.0, synth.HISTORY_BF16)])
def test_cic_field_clustered_full_grid(n, box, hist):
    w = dataclasses.replace(synth.small(n=n, box=box, n_steps=6, n_src=150, subsamples=2, clustered=True,
                                        seed=500 + n, history=hist), deposit=CIC)
    P = oracle.Problem.from_workload(w)
    plan = lc.Plan.from_workload(w)
    out = run_steps(plan, w.cat, range(6), {3, 5})
    for s, J in out.items():
        rel, mx, raw = errors(J, oracle.field_for(P, w.cat, s))
        if hist == synth.HISTORY_FP32:
            assert rel <= FP32_L2 and mx <= FP32_MAX, (n, s, rel, mx, raw)
        else:
            assert rel <= BF16_L2, (n, s, rel)
    plan.close()


def test_cic_step_graph_equals_eager_path():
    w = dataclasses.replace(synth.config("c1"), deposit=CIC)
    a, b = lc.Plan.from_workload(w), lc.Plan.from_workload(w)
    srcs = [(torch.from_numpy(w.cat.active(s)[0]).cuda(), torch.from_numpy(w.cat.active(s)[1]).cuda())
            for s in range(8)]
    for s in range(5):
        a.push(s, *srcs[s])
        b.push(s, *srcs[s])
    out = torch.empty((w.n,) * 3, dtype=torch.float32, device="cuda")
    graphs = [a.graph(s, *srcs[s], out) for s in (5, 6, 7)]
    for k, s in enumerate((5, 6, 7)):
        graphs[k].launch()
        ja = out.clone()
        b.push(s, *srcs[s])
        jb = b.field(s)
        torch.cuda.synchronize()
        assert torch.equal(ja, jb), s
    for g in graphs:
        g.close()
    a.close()
    b.close()


# ------------------------------------------------------------------ rough horizon
def test_rough_horizon_c1_every_step_full_grid():
    w = dataclasses.replace(synth.config("c1"), horizon_mode=lc.HORIZON_ROUGH)
    P = oracle.Problem.from_workload(w)
    plan = lc.Plan.from_workload(w)
    for s in range(8):
        lo, hi, rh = plan.shells(s)
        plo, phi, prh = P.shells(s)
        assert rh == pytest.approx(prh, rel=1e-12) and len(lo) == len(plo)
        assert np.allclose(lo, plo, rtol=1e-12) and np.allclose(hi, phi, rtol=1e-12)
    assert rh == pytest.approx(oracle.rough_horizon_radius(w.omega_m, w.h, P.z_edges[-1]), rel=1e-12)
    out = run_steps(plan, w.cat, range(8), set(range(8)))
    for s, J in out.items():
        ref = oracle.field_for(P, w.cat, s)
        rel, mx, raw = errors(J, ref)
        assert rel <= FP32_L2 and mx <= FP32_MAX, (s, rel, mx, raw)
    plan.close()


def test_rough_horizon_equal_tau_bf16():
    # shells spanning the rough horizon, BF16 history: 24 shells, 30 steps at 32^3
    st = synth.StepSpec(synth.STEPS_EQUAL_TAU, 30, z_end=15.0, n_shell=24)
    cat = synth.make_catalogue(synth.SEED_BASE + 611, 400, 50.0, 30, clustered=True, n_centres=8, sigma=2.0)
    w = synth.Workload("rough_tau", 32, 50.0, 0.31, 0.68, st, 2, synth.HISTORY_BF16, cat,
                       horizon_mode=lc.HORIZON_ROUGH)
    P = oracle.Problem.from_workload(w)
    plan = lc.Plan.from_workload(w)
    assert np.allclose(plan.z_edges, P.z_edges, rtol=1e-12)
    out = run_steps(plan, w.cat, range(30), {29})
    rel, mx, raw = errors(out[29], oracle.field_for(P, w.cat, 29))
    assert rel <= BF16_L2, rel
    plan.close()


# ------------------------------------------------------------------ slice cap
@pytest.mark.parametrize("cap,hist", [(1, synth.HISTORY_FP32), (3, synth.HISTORY_FP32), (3, synth.HISTORY_BF16)])
def test_n_shell_max_against_oracle(cap, hist):
    w = dataclasses.replace(synth.small(n=32, box=60.0, n_steps=10, n_src=120, seed=77, z_start=20.0, z_end=18.0,
                                        life=(2, 4), history=hist), n_shell_max=cap)
    P = oracle.Problem.from_workload(w)
    plan = lc.Plan.from_workload(w)
    assert plan.n_ring == cap
    out = run_steps(plan, w.cat, range(10), {6, 9})
    for s, J in out.items():
        assert len(plan.shells(s)[0]) == P.active_shells(s) == cap
        rel, mx, raw = errors(J, oracle.field_for(P, w.cat, s))
        if hist == synth.HISTORY_FP32:
            assert rel <= FP32_L2 and mx <= FP32_MAX, (cap, s, rel, mx, raw)
        else:
            assert rel <= BF16_L2, (cap, s, rel)
    plan.close()


# ------------------------------------------------------------------ launch shapes and special values
@pytest.mark.parametrize("n_src", [1, 31, 33, 300, 5000, 70000])
@pytest.mark.parametrize("dep", [lc.DEPOSIT_NGP, CIC])
def test_deposit_launch_shapes_and_special_values(n_src, dep):
    """Sources spread over CTAs of 32 to 256 threads; a -0 luminosity (valid,
    no effect on the fixed-point unit), coordinates far outside the box
    (cell wrap beyond 2^53 cells), negative coordinates; bit-exact grid, unit
    and total against the oracle."""
    N, box = 32, 64.0
    rng = np.random.default_rng(n_src + 7 * dep)
    pos = rng.uniform(-2 * box, 3 * box, size=(n_src, 3))
    lum = 10.0 ** rng.normal(0, 1.5, size=n_src)
    lum[0] = -0.0
    if n_src > 3:
        pos[1] = [1e17 + 0.25, -3e18, 5.5]
        pos[2] = [-1e-320, 2.0 * box, -0.5 * box / N]
        lum[3] = 0.0
    f = oracle.deposit_cic_fixed if dep == CIC else oracle.deposit_fixed
    go, So, to = f(N, box, pos, lum)
    g, S, t = lc.deposit_grid(N, box, pos, lum, deposit=dep)
    assert S == So and t == to and np.array_equal(g, go)
