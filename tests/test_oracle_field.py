"""Pins of the oracle's shell Green's functions (Eq. 10), deposit (Eq. 11/17)
and direct-convolution field (Eqs. 9, 11), and of its brute-force DFT (Eq. 12).

Checks are against brute force without symmetry, convergence of the lattice
sum to the shell integral, the far-field limit g(r), closed forms (uniform
source), invariances (linearity, translation, rotation), causality, and numpy's
FFT on tiny grids (a library special case of the convolution theorem, Eq. 13).
"""
import math

import numpy as np
import pytest

import synth


def tiny_problem(oracle_lib, n=16, box=40.0, n_steps=6, subsamples=4, normalise=1, z_start=20.0, z_end=15.0):
    st = synth.StepSpec(synth.STEPS_EQUAL_TIME, n_steps, z_start=z_start, z_end=z_end)
    return oracle_lib.Problem(n, box, 0.31, 0.68, st, subsamples=subsamples, normalise=normalise)


def test_rgf_octant_matches_direct_sum_without_symmetry(oracle_lib):
    P = tiny_problem(oracle_lib, n=12, box=60.0, normalise=0)
    s = 3
    A = P.active_shells(s)
    assert A >= 2
    rng = np.random.default_rng(1)
    N = P.n
    for j in range(A):
        full = P.rgf_full(s, j)
        for _ in range(6):
            d = rng.integers(0, N, size=3)
            assert full[tuple(d)] == pytest.approx(P.rgf_direct(s, j, d), rel=1e-12, abs=1e-300)


def test_rgf_shell_support_and_normalisation(oracle_lib):
    P = tiny_problem(oracle_lib, n=16, box=100.0)
    s = 4
    lo, hi, rh = P.shells(s)
    l = P.box / P.n
    N = P.n
    idx = np.arange(N)
    for j in range(len(lo)):
        G, I, sm = P.rgf_octant(s, j)
        full = P.rgf_full(s, j)
        assert l ** 3 * full.sum() == pytest.approx(I, rel=1e-12)
        # a cell contributes only if some periodic image of it lies in the shell
        X, Y, Z = np.meshgrid(idx, idx, idx, indexing="ij")
        dmin = np.full(X.shape, np.inf)
        dmax = np.zeros(X.shape)
        for u in range(-3, 4):
            for v in range(-3, 4):
                for w in range(-3, 4):
                    r = l * np.sqrt((X + u * N) ** 2 + (Y + v * N) ** 2 + (Z + w * N) ** 2)
                    inside = (r + 0.87 * l >= lo[j]) & (r - 0.87 * l < min(hi[j], rh))
                    dmin = np.where(inside, 0.0, dmin)
        assert np.all(full[np.isinf(dmin)] == 0.0)
        assert np.count_nonzero(full) > 0


def test_lattice_sum_converges_to_shell_integral(oracle_lib):
    # the un-normalised sub-sampled sum is a Riemann sum of int 4 pi r^2 g dr
    errs = []
    for s_sub in (2, 4, 8):
        P = tiny_problem(oracle_lib, n=16, box=100.0, subsamples=s_sub, normalise=0)
        _, I, sm = P.rgf_octant(4, 1)
        l = P.box / P.n
        errs.append(abs(l ** 3 * sm / I - 1.0))
    assert errs[2] < errs[0]
    assert errs[2] < 2e-3


def test_rgf_far_field_equals_image_sum_of_kernel(oracle_lib):
    # Eq. 10: G_j(d) = sum over periodic images u inside the shell of g(|d + u L|).
    # For cells whose images all sit at least a cell away from the shell edges,
    # the s^3-sample cell average of g -> g(r) up to O((l/r)^2).
    P = tiny_problem(oracle_lib, n=32, box=100.0, normalise=0)
    s = 4
    lo, hi, rh = P.shells(s)
    l = P.box / P.n
    zo = P.z_edges[s + 1]
    N = P.n
    checked = 0
    for j in range(len(lo)):
        top = min(hi[j], rh)
        full = P.rgf_full(s, j)
        for d in [(10, 3, 2), (5, 11, 7), (12, 12, 1), (9, 9, 9), (3, 2, 1), (6, 0, 0), (16, 16, 16), (0, 16, 5)]:
            rs = [l * math.sqrt((d[0] + u * N) ** 2 + (d[1] + v * N) ** 2 + (d[2] + w * N) ** 2)
                  for u in range(-3, 4) for v in range(-3, 4) for w in range(-3, 4)]
            if any(abs(r - lo[j]) < l or abs(r - top) < l for r in rs):
                continue  # a partially covered cell
            inside = [r for r in rs if lo[j] <= r < top]
            want = sum(oracle_lib.g(P.om, P.h, zo, r) for r in inside)
            if not inside:
                assert full[d] == 0.0
                continue
            assert full[d] == pytest.approx(want, rel=3 * (l / min(inside)) ** 2)
            checked += 1
    assert checked >= 4


def test_deposit_ngp_cells_and_wrap(oracle_lib):
    N, box = 8, 16.0  # l = 2
    pos = np.array([[0.99, 0.0, 0.0],     # x/l + 1/2 = 0.995 -> cell 0
                    [1.0, 0.0, 0.0],      # exactly 1.0 -> cell 1 (ties round up)
                    [-0.5, 15.2, 33.0],   # -0.25+.5 -> 0 ; 8.1 -> 8 -> 0 ; 17 -> 1
                    [3.1, 2.9, 1e6 + 1.0]])
    lum = np.array([1.0, 2.0, 4.0, 8.0])
    g = oracle_lib.deposit_ngp(N, box, pos, lum)
    assert g[0, 0, 0] == 1.0 and g[1, 0, 0] == 2.0 and g[0, 0, 1] == 4.0
    k = int(math.floor((1e6 + 1.0) / 2 + 0.5)) % 8
    assert g[2, 1, k] == 8.0
    assert g.sum() == 15.0
    with pytest.raises(ValueError):
        oracle_lib.deposit_ngp(N, box, pos, np.array([1.0, -1.0, 0.0, 0.0]))
    with pytest.raises(ValueError):
        oracle_lib.deposit_ngp(N, box, np.array([[np.nan, 0, 0]]), np.array([1.0]))


def test_deposit_fixed_point_exact_and_order_independent(oracle_lib):
    w = synth.config("c2")
    pos, lum = w.cat.active(30)
    grid, S, tot = oracle_lib.deposit_fixed(w.n, w.box, pos, lum)
    assert grid.sum() == tot and tot < 2 ** 62 + len(lum)
    assert S == 2.0 ** (math.frexp(len(lum) * lum.max())[1] - 62)
    f = oracle_lib.deposit_ngp(w.n, w.box, pos, lum)
    assert np.allclose(grid * S, f, rtol=1e-14, atol=0)
    perm = np.random.default_rng(0).permutation(len(lum))
    g2, S2, t2 = oracle_lib.deposit_fixed(w.n, w.box, pos[perm], lum[perm])
    assert S2 == S and t2 == tot and np.array_equal(g2, grid)
    e, Se, te = oracle_lib.deposit_fixed(w.n, w.box, np.zeros((0, 3)), np.zeros(0))
    assert te == 0 and not e.any()


def test_uniform_source_closed_form(oracle_lib):
    # every cell holds rho l^3  =>  J = U rho sum_j I_j  (exact with normalisation)
    P = tiny_problem(oracle_lib, n=12, box=60.0)
    s = 4
    rho = 0.37
    l = P.box / P.n
    _, _, I = P.shell_table(s)
    grids = [np.full((P.n,) * 3, rho * l ** 3) for _ in range(len(I))]
    J = P.field(s, grids)
    assert np.allclose(J, rho * I.sum(), rtol=1e-12)


def test_point_source_is_sum_of_green_functions(oracle_lib):
    P = tiny_problem(oracle_lib, n=12, box=60.0)
    s = 4
    A = P.active_shells(s)
    c = (3, 7, 10)
    L = 2.5
    grids = []
    for j in range(A):
        g = np.zeros((P.n,) * 3)
        g[c] = L
        grids.append(g)
    J = P.field(s, grids)
    want = sum(np.roll(P.rgf_full(s, j), c, axis=(0, 1, 2)) for j in range(A)) * L
    assert np.allclose(J, want, rtol=1e-13, atol=0)


def test_linearity_translation_rotation_and_dc(oracle_lib):
    w = synth.small(n=12, box=50.0, n_src=40, n_steps=5)
    P = oracle_lib.Problem.from_workload(w)
    s = 4
    rng = np.random.default_rng(3)
    A = P.active_shells(s)
    f1 = [rng.random((P.n,) * 3) * (rng.random((P.n,) * 3) < 0.05) for _ in range(A)]
    f2 = [rng.random((P.n,) * 3) * (rng.random((P.n,) * 3) < 0.05) for _ in range(A)]
    J1, J2 = P.field(s, f1), P.field(s, f2)
    J12 = P.field(s, [2.0 * a - 0.5 * b for a, b in zip(f1, f2)])
    assert np.allclose(J12, 2.0 * J1 - 0.5 * J2, rtol=1e-11, atol=1e-12 * np.abs(J1).max())
    sh = (2, -3, 5)
    Jt = P.field(s, [np.roll(a, sh, axis=(0, 1, 2)) for a in f1])
    assert np.allclose(Jt, np.roll(J1, sh, axis=(0, 1, 2)), rtol=1e-12)
    Jr = P.field(s, [np.transpose(a, (2, 0, 1)) for a in f1])
    assert np.allclose(Jr, np.transpose(J1, (2, 0, 1)), rtol=1e-12)
    Jf = P.field(s, [a[::-1, :, :] for a in f1])
    assert np.allclose(Jf, J1[::-1, :, :], rtol=1e-12)  # G is even: reflection commutes
    # DC identity: mean J = U N^-3 sum_j (I_j / l^3) sum f_j
    _, _, I = P.shell_table(s)
    l = P.box / P.n
    dc = sum(I[j] / l ** 3 * f1[j].sum() for j in range(A))
    assert J1.mean() == pytest.approx(dc / P.n ** 3, rel=1e-12)


def test_causality_flash_and_horizon(oracle_lib):
    # a source that shone during one slice only affects cells in that slice's shell
    P = tiny_problem(oracle_lib, n=16, box=100.0)
    s = 5
    lo, hi, rh = P.shells(s)
    A = len(lo)
    j = 1
    grids = [None] * A
    g = np.zeros((P.n,) * 3)
    g[0, 0, 0] = 1.0
    grids[j] = g
    J = P.field(s, grids)
    assert np.array_equal(J, P.rgf_full(s, j))
    # every lookback beyond the active set is outside the horizon
    assert P.shells(s)[0].shape[0] == A and A <= s + 1
    lo_all = [oracle_lib.chi(P.om, P.h, P.z_edges[s + 1], P.z_edges[n + 1]) for n in range(s + 1)]
    for jj in range(A, s + 1):
        assert lo_all[s - jj] >= rh * (1 - 1e-9)


def test_brute_dft_against_numpy_and_parseval(oracle_lib):
    rng = np.random.default_rng(7)
    x = rng.standard_normal((8, 8, 8)) + 1j * rng.standard_normal((8, 8, 8))
    X = oracle_lib.dft3(x, -1)
    assert np.allclose(X, np.fft.fftn(x), rtol=1e-12, atol=1e-11)
    back = oracle_lib.dft3(X, +1) / 8 ** 3  # Eq. 12: inverse with +i and 1/N^3
    assert np.allclose(back, x, atol=1e-12)
    assert np.sum(np.abs(X) ** 2) / 8 ** 3 == pytest.approx(np.sum(np.abs(x) ** 2), rel=1e-12)


def test_direct_convolution_equals_convolution_theorem(oracle_lib):
    # Eq. 11 by direct sum equals Eq. 13 evaluated with numpy's FFT (8^3 case)
    P = tiny_problem(oracle_lib, n=8, box=30.0)
    s = 3
    A = P.active_shells(s)
    rng = np.random.default_rng(11)
    f = [rng.random((8, 8, 8)) for _ in range(A)]
    J = P.field(s, f)
    Jhat = sum(np.fft.fftn(P.rgf_full(s, j)) * np.fft.fftn(f[j]) for j in range(A))
    assert np.allclose(J, np.fft.ifftn(Jhat).real, rtol=1e-11)
    # and the Green's function transforms are real (G even)
    for j in range(A):
        assert np.abs(np.fft.fftn(P.rgf_full(s, j)).imag).max() < 1e-12 * np.abs(P.rgf_full(s, j)).sum()


def test_instant_field_equals_retarded_for_steady_sources(oracle_lib):
    # Eq. 18 freezes the sources at the observing redshift; if the sources never
    # change, the instantaneous and the light-cone fields coincide, and a source
    # that switched on at the observing step is seen too early by Eq. 18.
    w = synth.small(n=12, box=50.0, n_src=30, n_steps=5, life=(5, 5))
    w.cat.birth[:] = 0
    P = oracle_lib.Problem.from_workload(w)
    s = 4
    J = oracle_lib.field_for(P, w.cat, s)
    Ji = oracle_lib.instant_field_for(P, w.cat, s)
    assert np.allclose(Ji, J, rtol=1e-13)
    w.cat.birth[:] = s  # all switched on at the observing step
    Ji2 = oracle_lib.instant_field_for(P, w.cat, s)
    J2 = oracle_lib.field_for(P, w.cat, s)
    assert (Ji2 >= J2 - 1e-12 * np.abs(J2).max()).all() and Ji2.sum() > J2.sum()


def test_field_from_occupied_cells_equals_dense_grids(oracle_lib):
    # field_for hands the oracle each slice's occupied cells instead of dense
    # grids; the sum is the same, in the same order, so the bits agree
    w = synth.small(n=16, box=40.0, n_steps=6, n_src=60, seed=1234, clustered=True)
    P = oracle_lib.Problem.from_workload(w)
    for s in (3, 5):
        dense = P.field(s, oracle_lib.source_grids(P, w.cat, s))
        assert np.array_equal(oracle_lib.field_for(P, w.cat, s), dense)
        cells = synth.sample_cells(s, w.n, 50)
        assert np.array_equal(oracle_lib.field_for(P, w.cat, s, cells=cells), dense.reshape(-1)[cells])
