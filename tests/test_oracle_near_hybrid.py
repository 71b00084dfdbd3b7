"""Pins of the oracle's particle-mesh hybrid near the sources (Discussion):
the innermost slice's near cube around each source from the source's own
position.  Checked against the oracle's independent octant builder (a source
at its cell centre must give back G_0, Eq. 10), exact translation and mirror
symmetries, and the ordering that a decreasing kernel imposes."""
import numpy as np
import pytest

import synth

R = 2


def _problem(oracle_lib, n=16, box=40.0):
    st = synth.StepSpec(synth.STEPS_EQUAL_TIME, 6, z_start=16.0, z_end=15.0)
    return oracle_lib.Problem(n, box, 0.31, 0.68, st, subsamples=4)


def _cube(J, c, n):
    idx = [(np.arange(c[d] - R, c[d] + R + 1) % n) for d in range(3)]
    return J[np.ix_(*idx)]


def test_centred_source_gives_back_g0(oracle_lib):
    P = _problem(oracle_lib)
    s, n, l = 4, P.n, P.box / P.n
    G0 = P.rgf_full(s, 0)  # octant builder: integer shell classification, image sum
    c = (5, 9, 2)
    pos = np.array([[c[0] * l + 0.3 * l, c[1] * l - 0.2 * l, c[2] * l + 0.1 * l]])
    lum = np.array([2.5])
    J = oracle_lib.near_cube(P, s, pos, lum, centred=True)
    want = np.zeros_like(J)
    for dx in range(-R, R + 1):
        for dy in range(-R, R + 1):
            for dz in range(-R, R + 1):
                want[(c[0] + dx) % n, (c[1] + dy) % n, (c[2] + dz) % n] = 2.5 * G0[dx % n, dy % n, dz % n]
    assert np.allclose(J, want, rtol=1e-12, atol=0)
    assert (J != 0).sum() == (2 * R + 1) ** 3


def test_exact_position_translation_mirror_and_order(oracle_lib):
    P = _problem(oracle_lib)
    s, n, l = 4, P.n, P.box / P.n
    lum = np.array([1.0])
    base = np.array([4.0 * l + 0.3 * l, 7.0 * l, 11.0 * l])
    A = oracle_lib.near_cube(P, s, base[None], lum, centred=False)
    # one cell over in x: the same cube, one cell over
    B = oracle_lib.near_cube(P, s, (base + [l, 0, 0])[None], lum, centred=False)
    assert np.allclose(np.roll(A, 1, axis=0), B, rtol=1e-12)
    # the mirror image of the offset in x mirrors the cube about the source cell
    M = oracle_lib.near_cube(P, s, np.array([[4.0 * l - 0.3 * l, 7.0 * l, 11.0 * l]]), lum, centred=False)
    ca, cm = _cube(A, (4, 7, 11), n), _cube(M, (4, 7, 11), n)
    assert np.allclose(ca, cm[::-1, :, :], rtol=1e-12)
    # the source sits towards +x: the +x neighbour gets more than the -x one,
    # and both differ from the centred values
    C = _cube(oracle_lib.near_cube(P, s, base[None], lum, centred=True), (4, 7, 11), n)
    assert ca[R + 1, R, R] > C[R + 1, R, R] > ca[R - 1, R, R]
    assert ca[R + 2, R, R] > ca[R - 2, R, R]


def test_hybrid_is_linear_and_equals_ngp_for_centred_sources(oracle_lib):
    P = _problem(oracle_lib)
    s, l = 4, P.box / P.n
    pos = np.array([[3.4 * l, 8.1 * l, 1.7 * l], [12.6 * l, 2.5001 * l, 9.2 * l]])
    lum = np.array([1.5, 0.7])
    one = oracle_lib.near_cube(P, s, pos[:1], lum[:1], centred=False)
    two = oracle_lib.near_cube(P, s, pos[1:], lum[1:], centred=False)
    both = oracle_lib.near_cube(P, s, pos, lum, centred=False)
    assert np.allclose(both, one + two, rtol=1e-12)
    # sources exactly on cell centres: the hybrid changes nothing
    cpos = np.round(pos / l) * l
    ex = oracle_lib.near_cube(P, s, cpos, lum, centred=False)
    ce = oracle_lib.near_cube(P, s, cpos, lum, centred=True)
    assert np.allclose(ex, ce, rtol=1e-12)
