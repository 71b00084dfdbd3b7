"""Pins of the oracle's cloud-in-cell deposit, its literal-horizon LW kernel
(Section 1's rough horizon), and its cap on the lookback slices per step.

The cloud-in-cell grid is pinned by properties that a wrong neighbour, a
flipped weight, a swapped axis or a lost charge would break: exact charge
conservation, the first moment (trilinear weights reproduce a source's
position as the charge-weighted mean of the cell centres), equal halves at a
midpoint, equality with the nearest grid point for sources at cell centres,
integer-cell translation covariance and independence of source order.  The
rough-horizon kernel is pinned by the closed form of its horizon in a
matter-only universe and by agreement with the Eq. 15 kernel inside 97.39
alpha.  The slice cap is pinned by linearity: capped fields equal uncapped
ones with the dropped slices' sources removed.
"""
import math

import numpy as np
import pytest

import synth

C = 299792.458


# ---------------------------------------------------------------- CIC deposit
def test_cic_conserves_charge_and_reproduces_position(oracle_lib):
    # dyadic cell size (l = 2) so that x / l is exact
    N, box = 16, 32.0
    l = box / N
    rng = np.random.default_rng(3)
    for _ in range(20):
        # one source away from the periodic seam: its 8 cells are contiguous
        x = rng.uniform(3 * l, (N - 3) * l, size=3)
        L = float(10.0 ** rng.uniform(-2, 3))
        g = oracle_lib.deposit_cic(N, box, x[None, :], np.array([L]))
        assert g.sum() == pytest.approx(L, rel=1e-15)
        assert np.count_nonzero(g) <= 8 and g.min() >= 0.0
        idx = np.indices(g.shape).reshape(3, -1).astype(np.float64) * l
        com = (idx * g.reshape(-1)).sum(axis=1) / g.sum()
        assert np.allclose(com, x, rtol=0, atol=1e-12 * box)
        gi, S, tot = oracle_lib.deposit_cic_fixed(N, box, x[None, :], np.array([L]))
        assert gi.sum() == tot and gi.min() >= 0
        # fixed point: each cell within the rounding of the split (three
        # products of a charge below 2^62 with a weight, 2^-53 relative each)
        # of the FP64 share
        assert np.abs(gi * S - g).max() <= 4 * 2.0 ** -52 * L + 2 * S


def test_cic_midpoint_halves_and_cell_centre_equals_ngp(oracle_lib):
    N, box = 8, 16.0
    l = box / N
    # midway between cells 2 and 3 along x, at centres along y and z
    g = oracle_lib.deposit_cic(N, box, np.array([[2.5 * l, 4 * l, 7 * l]]), np.array([6.0]))
    assert g[2, 4, 7] == 3.0 and g[3, 4, 7] == 3.0 and g.sum() == 6.0
    gi, S, tot = oracle_lib.deposit_cic_fixed(N, box, np.array([[2.5 * l, 4 * l, 7 * l]]), np.array([6.0]))
    assert abs(gi[2, 4, 7] - gi[3, 4, 7]) <= 1 and gi[2, 4, 7] + gi[3, 4, 7] == tot
    # sources exactly at cell centres: CIC is NGP, bit for bit in fixed point
    rng = np.random.default_rng(4)
    cells = rng.integers(-20, 30, size=(50, 3))
    pos = cells * l
    lum = 10.0 ** rng.normal(0, 1, size=50)
    a, Sa, ta = oracle_lib.deposit_cic_fixed(N, box, pos, lum)
    b, Sb, tb = oracle_lib.deposit_fixed(N, box, pos, lum)
    assert Sa == Sb and ta == tb and np.array_equal(a, b)
    assert np.allclose(oracle_lib.deposit_cic(N, box, pos, lum), oracle_lib.deposit_ngp(N, box, pos, lum),
                       rtol=1e-15, atol=0)


def test_cic_wraps_periodically_and_is_translation_covariant(oracle_lib):
    N, box = 16, 32.0
    l = box / N
    rng = np.random.default_rng(5)
    # positions on a 1/64-cell lattice: every x / l, shifted or not, is exact
    pos = rng.integers(-64 * N, 2 * 64 * N, size=(200, 3)) * (l / 64)
    lum = 10.0 ** rng.normal(0, 1.5, size=200)
    a, S, t = oracle_lib.deposit_cic_fixed(N, box, pos, lum)
    assert a.sum() == t and a.min() >= 0
    for shift in ([3, 0, 0], [0, -5, 17], [N, 2 * N, -N]):
        b, S2, t2 = oracle_lib.deposit_cic_fixed(N, box, pos + np.array(shift) * l, lum)
        assert S2 == S and t2 == t
        assert np.array_equal(b, np.roll(a, shift, axis=(0, 1, 2)))
    # a source at the top edge of the box shares with cell 0
    g = oracle_lib.deposit_cic(N, box, np.array([[(N - 0.25) * l, 0.0, 0.0]]), np.array([4.0]))
    assert g[N - 1, 0, 0] == 1.0 and g[0, 0, 0] == 3.0


def test_cic_fixed_point_matches_fp64_and_is_order_independent(oracle_lib):
    w = synth.config("c2")
    pos, lum = w.cat.active(30)
    gi, S, tot = oracle_lib.deposit_cic_fixed(w.n, w.box, pos, lum)
    assert gi.sum() == tot and tot < 2 ** 62 + len(lum)
    assert S == 2.0 ** (math.frexp(len(lum) * lum.max())[1] - 62)
    f = oracle_lib.deposit_cic(w.n, w.box, pos, lum)
    # every cell within the split's rounding (2^-53 relative per product) of its FP64 value
    assert np.abs(gi * S - f).max() <= 4 * 2.0 ** -52 * lum.sum() + 8 * S
    assert np.abs(gi * S - f).max() <= 1e-6 * f.max()
    assert gi.sum() * S == pytest.approx(lum.sum(), rel=1e-15)
    perm = np.random.default_rng(0).permutation(len(lum))
    g2, S2, t2 = oracle_lib.deposit_cic_fixed(w.n, w.box, pos[perm], lum[perm])
    assert S2 == S and t2 == tot and np.array_equal(g2, gi)
    with pytest.raises(ValueError):
        oracle_lib.deposit_cic(8, 16.0, np.array([[np.inf, 0, 0]]), np.array([1.0]))


def test_cic_field_uniform_source_and_point_limit(oracle_lib):
    # a uniform lattice of equal sources deposits a uniform grid with CIC too,
    # so the field takes the uniform closed form J = U rho sum_j I_j
    st = synth.StepSpec(synth.STEPS_EQUAL_TIME, 6, z_start=20.0, z_end=15.0)
    P = oracle_lib.Problem(12, 60.0, 0.31, 0.68, st, deposit=oracle_lib.DEPOSIT_CIC)
    l = P.box / P.n
    s = 4
    _, _, I = P.shell_table(s)
    g = np.arange(12) * l + 0.3 * l
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    lum = np.full(pos.shape[0], 0.37 * l ** 3)
    grid = oracle_lib.deposit(P, pos, lum)
    assert np.allclose(grid, 0.37 * l ** 3, rtol=1e-13)
    J = P.field(s, [grid] * len(I))
    assert np.allclose(J, 0.37 * I.sum(), rtol=1e-12)


# ---------------------------------------------------------------- rough horizon
def test_rough_horizon_matter_only_closed_form(oracle_lib):
    # Omega_m = 1: chi(z_o, z_s) = K (a_o - b), b = (1 + z_s)^-1/2, K = 2c/H0.
    # r = 100 sqrt(21) b and r = K (a_o - b) give r = 100 sqrt(21) K a_o / (K + 100 sqrt(21)).
    h = 0.7
    K = 2 * C / (100 * h)
    for zo in (10.0, 15.0, 20.0, 27.9):
        ao = 1 / math.sqrt(1 + zo)
        want = 100 * math.sqrt(21) * K * ao / (K + 100 * math.sqrt(21))
        assert oracle_lib.rough_horizon_radius(1.0, h, zo) == pytest.approx(want, rel=1e-12)
        assert oracle_lib.rough_horizon(20.0) == pytest.approx(100.0, rel=1e-15)


def test_rough_horizon_kernel_agrees_with_eq15_inside_and_clamps_outside(oracle_lib):
    om, h, zo = 0.31, 0.68, 15.0
    rough = (oracle_lib.KERNEL_LW_ROUGH, 0.0, 0.0)
    rh = oracle_lib.horizon(om, h, zo)
    rz = oracle_lib.fmod_zero_radius(om, h, zo)
    rr = oracle_lib.rough_horizon_radius(om, h, zo)
    assert rh < rz < rr  # Eq. 15's cut, the zero of f_mod, the rough horizon (this cosmology)
    assert oracle_lib.horizon_kernel(rough, om, h, zo) == pytest.approx(rr, rel=1e-14)
    for r in np.linspace(0.5, rh * 0.999, 25):
        assert oracle_lib.g_kernel(rough, om, h, zo, r) == pytest.approx(oracle_lib.g(om, h, zo, r), rel=1e-15)
    # between Eq. 15's cut and the zero crossing the clamped f_mod is small and positive,
    for r in np.linspace(rh * 1.0001, rz * 0.9999, 5):
        v = oracle_lib.g_kernel(rough, om, h, zo, r)
        assert 0.0 < v and oracle_lib.g(om, h, zo, r) == 0.0
    # and beyond it zero
    for r in np.linspace(rz * 1.0001, rr * 1.5, 7):
        assert oracle_lib.g_kernel(rough, om, h, zo, r) == 0.0
    # shell integrals: equal inside Eq. 15's horizon, the extra sliver beyond it small
    I0 = oracle_lib.shell_integral(om, h, zo, 10.0, rh)
    I2 = oracle_lib.shell_integral_kernel(rough, om, h, zo, 10.0, rh)
    assert I2 == pytest.approx(I0, rel=1e-12)
    extra = oracle_lib.shell_integral_kernel(rough, om, h, zo, rh, rr)
    assert 0.0 < extra < 1e-4 * I0


def test_rough_horizon_sliver_integral_vs_scipy(oracle_lib):
    from scipy import integrate

    h, zo = 0.7, 18.0
    rough = (oracle_lib.KERNEL_LW_ROUGH, 0.0, 0.0)

    def integrand(r):
        zs = (1 / math.sqrt(1 + zo) - r * 100 * h / (2 * C)) ** -2 - 1
        al = (1.0 / 0.27) ** -0.5 * ((1 + zs) / 21) ** -0.5
        if r > 100 * math.sqrt(21 / (1 + zs)):
            return 0.0
        f = 1.7 * math.exp(-((r / (116.29 * al)) ** 0.68)) - 0.7
        return (1 + zo) ** 3 * max(f, 0.0) / (4 * math.pi * (1 + zs))

    rr = oracle_lib.rough_horizon_radius(1.0, h, zo)
    rz = oracle_lib.fmod_zero_radius(1.0, h, zo)
    for lo, hi in [(0.0, 5.0), (40.0, rr + 3.0), (rz - 2.0, rr)]:
        want, _ = integrate.quad(integrand, lo, min(hi, rr), points=[rz], epsabs=0, epsrel=1e-12, limit=500)
        assert oracle_lib.shell_integral_kernel(rough, 1.0, h, zo, lo, hi) == pytest.approx(want, rel=1e-9)


# ---------------------------------------------------------------- slice cap
def test_n_shell_max_is_the_uncapped_field_without_older_slices(oracle_lib):
    w = synth.small(n=12, box=60.0, n_steps=10, n_src=60, seed=321, z_start=20.0, z_end=18.0, life=(2, 4))
    full = oracle_lib.Problem.from_workload(w)
    s = 9
    A = full.active_shells(s)
    assert A >= 3
    grids = oracle_lib.source_grids(full, w.cat, s)
    J_full = full.field(s, grids)
    for m in (1, 2):
        cap = oracle_lib.Problem.from_workload(w, n_shell_max=m)
        assert cap.active_shells(s) == m
        lo, hi, _ = cap.shells(s)
        lo0, hi0, _ = full.shells(s)
        assert np.array_equal(lo, lo0[:m]) and np.array_equal(hi, hi0[:m])
        J = oracle_lib.field_for(cap, w.cat, s)
        want = full.field(s, grids[:m] + [None] * (A - m))
        assert np.allclose(J, want, rtol=1e-14, atol=0)
        assert not np.allclose(J, J_full)
