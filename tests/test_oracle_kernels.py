"""Pins of the oracle's second radial kernel: the dilution and redshift
factors of Eq. 14 with a distance-only attenuation exp(-r / lambda) in place
of f_mod and a cut-off r_max as its horizon (the generic dilution factor of
Eq. 7 needs only to depend on distance).

In a matter-only universe the light-cone redshift is exact,
(1 + z_s)^(-1/2) = (1 + z_obs)^(-1/2) - r H0 / (2c), so g(r) and the shell
integral int 4 pi r^2 g dr have closed forms; the lattice Green's functions,
the far-field limit and the uniform-source field are then checked against
those closed forms, never against the oracle's own quadrature.
"""
import math

import numpy as np
import pytest

import synth

C = 299792.458
KERN = (1, 30.0, 80.0)  # exp(-r / 30 Mpc), cut off at 80 Mpc


def _ab(h, zo):
    return 1.0 / math.sqrt(1.0 + zo), 100.0 * h / (2.0 * C)


def g_closed(h, zo, r, lam=KERN[1], rmax=KERN[2]):
    if r >= rmax:
        return 0.0
    a, b = _ab(h, zo)
    return (1 + zo) ** 3 * (a - b * r) ** 2 * math.exp(-r / lam) / ((4 * math.pi) ** 2 * r * r)


def shell_closed(h, zo, r_lo, r_hi, lam=KERN[1], rmax=KERN[2]):
    # int_{r_lo}^{min(r_hi, rmax)} (1+zo)^3/(4 pi) (a - b r)^2 exp(-r/lam) dr:
    # the antiderivative of P(r) e^{-r/lam} is -lam e^{-r/lam} (P + lam P' + lam^2 P'')
    a, b = _ab(h, zo)
    top = min(r_hi, rmax)
    if not r_lo < top:
        return 0.0

    def F(r):
        u = a - b * r
        return -lam * math.exp(-r / lam) * (u * u - 2 * lam * b * u + 2 * lam * lam * b * b)

    return (1 + zo) ** 3 / (4 * math.pi) * (F(top) - F(r_lo))


def test_g_exp_matter_only_closed_form(oracle_lib):
    h, zo = 0.7, 12.0
    for r in [0.3, 5.0, 29.0, 79.9]:
        assert oracle_lib.g_kernel(KERN, 1.0, h, zo, r) == pytest.approx(g_closed(h, zo, r), rel=1e-11)
    for r in [80.0, 81.0, 200.0]:
        assert oracle_lib.g_kernel(KERN, 1.0, h, zo, r) == 0.0
    # the LW kernel stays the default
    assert oracle_lib.g_kernel(None, 0.31, 0.68, zo, 7.0) == oracle_lib.g(0.31, 0.68, zo, 7.0)


def test_shell_integral_exp_closed_form(oracle_lib):
    h, zo = 0.7, 12.0
    for lo, hi in [(0.0, 4.0), (4.0, 11.0), (20.0, 55.0), (60.0, 95.0), (85.0, 90.0)]:
        want = shell_closed(h, zo, lo, hi)
        got = oracle_lib.shell_integral_kernel(KERN, 1.0, h, zo, lo, hi)
        if want == 0.0:
            assert got == 0.0
        else:
            assert got == pytest.approx(want, rel=1e-10)


def test_horizon_and_equal_tau_edges(oracle_lib):
    assert oracle_lib.horizon_kernel(KERN, 0.31, 0.68, 15.0) == KERN[2]
    st = synth.StepSpec(synth.STEPS_EQUAL_TAU, 12, z_end=15.0, n_shell=8)
    z = oracle_lib.step_edges(0.31, 0.68, st, KERN)
    widths = [oracle_lib.chi(0.31, 0.68, z[k + 1], z[k]) for k in range(12)]
    assert np.allclose(widths, KERN[2] / 8, rtol=1e-9)


def _matter_problem(oracle_lib, n, box, normalise, subsamples=4, n_steps=6):
    st = synth.StepSpec(synth.STEPS_EQUAL_TAU, n_steps, z_end=12.0, n_shell=4)
    return oracle_lib.Problem(n, box, 1.0, 0.7, st, subsamples=subsamples, normalise=normalise, kernel=KERN)


def test_shells_follow_the_cut_off(oracle_lib):
    P = _matter_problem(oracle_lib, 16, 100.0, 1)
    lo, hi, rh = P.shells(5)
    assert rh == KERN[2] and len(lo) == 4  # 4 shells of 20 Mpc reach the cut-off
    assert np.allclose(np.diff(np.concatenate([[0.0], hi])), 20.0, rtol=1e-9)
    _, _, I = P.shell_table(5)
    zo = P.z_edges[6]
    want = [shell_closed(0.7, zo, a, b) for a, b in zip(lo, hi)]
    assert np.allclose(I, want, rtol=1e-10)


def test_lattice_sum_converges_to_closed_form(oracle_lib):
    # the un-normalised s^3-sample lattice sum of g tends to the closed-form shell integral
    errs = []
    for s_sub in (2, 4, 8):
        P = _matter_problem(oracle_lib, 16, 100.0, 0, subsamples=s_sub)
        lo, hi, _ = P.shells(5)
        _, _, sm = P.rgf_octant(5, 1)
        l = P.box / P.n
        errs.append(abs(l ** 3 * sm / shell_closed(0.7, P.z_edges[6], lo[1], hi[1]) - 1.0))
    assert errs[2] < errs[0] and errs[2] < 3e-3


def test_far_field_equals_image_sum_of_closed_form(oracle_lib):
    P = _matter_problem(oracle_lib, 32, 100.0, 0)
    s = 5
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
                continue
            inside = [r for r in rs if lo[j] <= r < top]
            if not inside:
                assert full[d] == 0.0
                continue
            want = sum(g_closed(0.7, zo, r) for r in inside)
            assert full[d] == pytest.approx(want, rel=3 * (l / min(inside)) ** 2)
            checked += 1
    assert checked >= 4


def test_uniform_source_field_closed_form(oracle_lib):
    # every cell holds rho l^3 => J = U rho sum_j I_j, with I_j in closed form
    P = _matter_problem(oracle_lib, 12, 60.0, 1)
    s = 5
    lo, hi, _ = P.shells(s)
    rho = 0.41
    l = P.box / P.n
    grids = [np.full((P.n,) * 3, rho * l ** 3) for _ in range(len(lo))]
    J = P.field(s, grids)
    want = rho * sum(shell_closed(0.7, P.z_edges[s + 1], a, b) for a, b in zip(lo, hi))
    assert np.allclose(J, want, rtol=1e-9)
