"""Pins of the oracle's cosmology, LW kernel constants and step edges.

Each check compares the oracle against something other than itself: a closed
form (matter-only universe), an independent library quadrature (scipy), or a
number printed in the paper (tests/golden/paper_constants.json).
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
C = 299792.458


def test_chi_matter_only_closed_form(oracle_lib):
    # Omega_m = 1: chi = 2c/H0 (1/sqrt(1+z1) - 1/sqrt(1+z2))  (Eq. 6 with a ~ t^(2/3))
    h = 0.7
    for z1, z2 in [(0.0, 1.0), (10.0, 30.0), (15.0, 15.3), (27.9, 29.78)]:
        want = 2 * C / (100 * h) * (1 / math.sqrt(1 + z1) - 1 / math.sqrt(1 + z2))
        got = oracle_lib.chi(1.0, h, z1, z2)
        assert got == pytest.approx(want, rel=1e-13)
    assert oracle_lib.chi(1.0, h, 3.0, 2.0) == pytest.approx(-oracle_lib.chi(1.0, h, 2.0, 3.0), rel=1e-15)


def test_chi_lcdm_within_lambda_bound(oracle_lib):
    # c/H <= c/(H0 sqrt(Om (1+z)^3)): LCDM distance is below the matter-only one
    # by at most a fraction OL / (2 Om (1+z1)^3).
    om, h, z1, z2 = 0.31, 0.68, 15.0, 20.0
    md = 2 * C / (100 * h * math.sqrt(om)) * (1 / math.sqrt(1 + z1) - 1 / math.sqrt(1 + z2))
    got = oracle_lib.chi(om, h, z1, z2)
    assert 0.0 < md - got <= md * (1 - om) / (2 * om * (1 + z1) ** 3)
    assert got == pytest.approx(503.2250717, rel=1e-9)


def test_cosmic_time_closed_form_vs_scipy(oracle_lib):
    om, h = 0.31, 0.68
    tH = 3.0856775814913673e19 / (100 * h) / 3.15576e13
    for z in [10.0, 15.0, 27.9]:
        num, _ = integrate.quad(lambda zz: 1.0 / ((1 + zz) * math.sqrt(om * (1 + zz) ** 3 + 1 - om)), z, np.inf,
                                epsabs=0, epsrel=1e-13, limit=200)
        assert oracle_lib.time_myr(om, h, z) == pytest.approx(num * tH, rel=1e-9)
        assert oracle_lib.z_of_time(om, h, oracle_lib.time_myr(om, h, z)) == pytest.approx(z, rel=1e-12)


def test_zs_of_r_matter_only_closed_form(oracle_lib):
    h = 0.7
    for zo, r in [(15.0, 1.0), (15.0, 80.0), (27.9, 50.0), (10.0, 120.0)]:
        x = 1 / math.sqrt(1 + zo) - r * 100 * h / (2 * C)
        want = x ** -2 - 1
        assert oracle_lib.zs_of_r(1.0, h, zo, r) == pytest.approx(want, rel=1e-13)
        assert oracle_lib.chi(1.0, h, zo, oracle_lib.zs_of_r(1.0, h, zo, r)) == pytest.approx(r, rel=1e-13)


def test_paper_constants_alpha_and_fmod(oracle_lib):
    a = GOLD["alpha_fiducial"]
    assert oracle_lib.alpha(a["omega_m"], a["h"], a["z_s"]) == pytest.approx(a["value"], rel=1e-15)
    # Eq. 15 at r = 0: 1.7 - 0.7 = 1
    assert oracle_lib.fmod(0.0, 1.0) == pytest.approx(GOLD["fmod_amplitude"]["value"] - GOLD["fmod_offset"]["value"])
    hz = GOLD["horizon_over_alpha"]["value"]
    for al in [0.8, 1.0, 1.3]:
        # nearly continuous cut: the modulation has almost reached zero at the horizon
        edge = oracle_lib.fmod(hz * al * (1 - 1e-12), al)
        assert 0.0 < edge < 1e-3
        assert oracle_lib.fmod(hz * al * (1 + 1e-12), al) == 0.0
    assert oracle_lib.fmod(50.0, 1.0) < oracle_lib.fmod(10.0, 1.0) < 1.0


def test_g_matter_only_closed_form(oracle_lib):
    # Eq. 14/17 with an exactly known z_s(r) (matter only) and Eq. 15/16.
    h = 0.7
    zo = 20.0
    for r in [0.5, 10.0, 40.0]:  # all inside the horizon (alpha ~ 0.52 here)
        zs = (1 / math.sqrt(1 + zo) - r * 100 * h / (2 * C)) ** -2 - 1
        al = (h / 0.7) ** -1 * (1.0 / 0.27) ** -0.5 * ((1 + zs) / 21) ** -0.5
        fm = 1.7 * math.exp(-((r / (116.29 * al)) ** 0.68)) - 0.7
        want = (1 + zo) ** 3 * fm / ((4 * math.pi) ** 2 * (1 + zs) * r * r)
        assert oracle_lib.g(1.0, h, zo, r) == pytest.approx(want, rel=1e-12)


def test_horizon_definition_and_rough_form(oracle_lib):
    om, h = 0.27, 0.7
    hz = GOLD["horizon_over_alpha"]["value"]
    rough = GOLD["rlw_rough_form"]
    for zo in [10.0, 15.0, 20.0, 27.9]:
        rh = oracle_lib.horizon(om, h, zo)
        zs = oracle_lib.zs_of_r(om, h, zo, rh)
        assert rh / oracle_lib.alpha(om, h, zs) == pytest.approx(hz, rel=1e-12)
        # Section 1's rough form, with z the emission redshift, agrees to ~3 %
        approx = rough["coefficient_mpc"] * (rough["z_pivot_plus_one"] / (1 + zs)) ** rough["power"]
        assert rh == pytest.approx(approx, rel=0.03)


def test_rlw_inside_ten_myr_lookback(oracle_lib):
    g = GOLD["rlw_inside_lookback"]
    om, h, zo = g["omega_m"], g["h"], g["z_obs"]
    t_obs = oracle_lib.time_myr(om, h, zo)
    z_back = oracle_lib.z_of_time(om, h, t_obs - g["lookback_myr"])
    reach = oracle_lib.chi(om, h, zo, z_back)
    assert oracle_lib.horizon(om, h, zo) < reach
    # but not inside the first 2-Myr slice: the 2nd-5th slices contribute (Section 3)
    z2 = oracle_lib.z_of_time(om, h, t_obs - 2.0)
    assert oracle_lib.horizon(om, h, zo) > oracle_lib.chi(om, h, zo, z2)
    # the same holds with the workload cosmology
    om, h = 0.31, 0.68
    t_obs = oracle_lib.time_myr(om, h, zo)
    assert oracle_lib.horizon(om, h, zo) < oracle_lib.chi(om, h, zo, oracle_lib.z_of_time(om, h, t_obs - 10.0))


def test_step_edges_equal_time_and_equal_tau(oracle_lib):
    om, h = 0.31, 0.68
    w = synth.config("c1")
    z = oracle_lib.step_edges(om, h, w.steps)
    assert z[0] == 20.0 and z[-1] == 15.0 and np.all(np.diff(z) < 0)
    t = np.array([oracle_lib.time_myr(om, h, zz) for zz in z])
    assert np.allclose(np.diff(t), (t[-1] - t[0]) / 8, rtol=1e-10)
    assert np.diff(t)[0] == pytest.approx(11.26, abs=0.01)  # 8 equal steps z=20->15 of 11.26 Myr
    spec = synth.StepSpec(synth.STEPS_EQUAL_TAU, 20, z_end=15.0, n_shell=16)
    z = oracle_lib.step_edges(om, h, spec)
    d = np.array([oracle_lib.chi(om, h, 15.0, zz) for zz in z])
    dtau = oracle_lib.horizon(om, h, 15.0) / 16
    assert np.allclose(-np.diff(d), dtau, rtol=1e-11)
    ex = synth.StepSpec(synth.STEPS_EXPLICIT, 2, z_edges=(9.0, 8.0, 7.5))
    assert list(oracle_lib.step_edges(om, h, ex)) == [9.0, 8.0, 7.5]


def test_shell_integral_matter_only_vs_scipy(oracle_lib):
    # I = int 4 pi r^2 g dr with z_s(r) closed form (Omega_m = 1) and scipy's quad
    h, zo = 0.7, 18.0

    def integrand(r):
        zs = (1 / math.sqrt(1 + zo) - r * 100 * h / (2 * C)) ** -2 - 1
        al = (1.0 / 0.27) ** -0.5 * ((1 + zs) / 21) ** -0.5
        if r / al > 97.39:
            return 0.0
        return (1 + zo) ** 3 * (1.7 * math.exp(-((r / (116.29 * al)) ** 0.68)) - 0.7) / (4 * math.pi * (1 + zs))

    rh = oracle_lib.horizon(1.0, h, zo)
    for lo, hi in [(0.0, 5.0), (5.0, 40.0), (40.0, rh + 10.0)]:
        want, _ = integrate.quad(integrand, lo, min(hi, rh), epsabs=0, epsrel=1e-12, limit=500)
        assert oracle_lib.shell_integral(1.0, h, zo, lo, hi) == pytest.approx(want, rel=1e-9)
    assert oracle_lib.shell_integral(1.0, h, zo, rh + 1, rh + 5) == 0.0
