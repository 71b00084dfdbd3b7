"""Seeded synthetic workloads for the light-cone retarded-field path.

This module is shared by the CUDA path's tests/benchmark and by the CPU
oracle's tests.  It holds only workload *descriptions* (grid, box, cosmology,
step specification, source catalogues) and random draws.  It contains none of
the method's arithmetic: no cosmology, no Green's function, no deposit, no
transform.  Step edges are handed to both implementations as a specification
(equal cosmic time between two redshifts, or equal conformal time ending at a
redshift), and each side derives the edges with its own cosmology code.

The paper's own application data (the source catalogue of a 114/h Mpc,
256^3 reionization simulation, Section 3) is not available; these seeded
catalogues stand in for it.  Their structure follows the workload list:

* ``c1``  32^3 grid, 100 Mpc box, 8 equal-cosmic-time steps z = 20 -> 15,
  200 sources, uniform positions, log10 L ~ N(0, 1) (sigma = 1 dex),
  every source lives 2 steps.
* ``c2``  128^3 grid, 150 Mpc box, 64 equal-cosmic-time steps z = 30 -> 10,
  1e4 sources, halo mass from dN/dM ~ M^-2 on [1e8, 1e11] Msun, L = M / 1e8,
  lifetimes uniform in {1..4} steps, positions Gaussian-clustered (sigma = 2
  Mpc) around 100 uniform centres, wrapped into the box.
* ``c3``  256^3 grid, 200 Mpc box, 128 equal-conformal-time shells spanning
  the Lyman-Werner horizon at z_obs = 15, 160 steps, 1e5 clustered sources
  (1000 centres), history stored in BF16.
* ``c3s`` the same 256^3 BF16 path with 32 shells and 40 steps (a profiling size).
* ``c5s`` the 512^3 BF16 path of the serving set with 16 shells and 24 steps (a profiling size).
* ``c4``  16 uneven instances (grids 64..256, 32..128 shells, 1e3..1e5
  sources, 0.78 Mpc cells).
* ``c5``  8 served simulations at 128^3..512^3.

Random stream: config k draws from ``numpy.random.Generator(PCG64(20150210 + k))``
in this order: cluster centres (if clustered), positions, luminosities (or
masses), birth steps, lifetimes.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Tuple

import numpy as np

SEED_BASE = 20150210

# Step specification kinds (mirrors the C-ABI enum values).
STEPS_EXPLICIT = 0
STEPS_EQUAL_TIME = 1
STEPS_EQUAL_TAU = 2

HISTORY_FP32 = 0
HISTORY_BF16 = 1


@dataclasses.dataclass
class StepSpec:
    """How the time axis is cut into steps (slices).

    kind = STEPS_EQUAL_TIME: n_steps slices of equal cosmic time between
    z_start and z_end (z_start > z_end).
    kind = STEPS_EQUAL_TAU: n_steps slices of equal conformal time, the last
    edge at z_end, with width r_h(z_end) / n_shell (r_h the Lyman-Werner
    horizon of an observer at z_end).
    kind = STEPS_EXPLICIT: the n_steps + 1 decreasing redshifts in z_edges.
    """

    kind: int
    n_steps: int
    z_start: float = 0.0
    z_end: float = 0.0
    n_shell: int = 0
    z_edges: Optional[Tuple[float, ...]] = None


@dataclasses.dataclass
class Catalogue:
    """Point sources over the whole run; a source is active at step s when
    birth <= s < birth + life."""

    pos: np.ndarray  # (n, 3) float64, comoving Mpc, in [0, box)
    lum: np.ndarray  # (n,) float64, luminosity units
    birth: np.ndarray  # (n,) int64
    life: np.ndarray  # (n,) int64

    def active(self, step: int) -> Tuple[np.ndarray, np.ndarray]:
        m = (self.birth <= step) & (step < self.birth + self.life)
        return (np.ascontiguousarray(self.pos[m]), np.ascontiguousarray(self.lum[m]))

    @property
    def n(self) -> int:
        return int(self.lum.shape[0])


@dataclasses.dataclass
class Workload:
    name: str
    n: int  # grid side
    box: float  # comoving Mpc
    omega_m: float
    h: float
    steps: StepSpec
    subsamples: int
    history: int
    cat: Catalogue
    out_unit: float = 1.0
    normalise: int = 1
    # radial kernel: None for the Lyman-Werner one, or (kind, length, rmax)
    # with kind 1 = exponential attenuation (length, cut-off in comoving Mpc)
    kernel: Optional[Tuple[int, float, float]] = None
    # near field of the innermost slice: 0 from NGP cells, 1 from the sources'
    # own positions (sub-cell)
    near_mode: int = 0
    # source assignment: 0 nearest grid point, 1 cloud in cell
    deposit: int = 0
    # Lyman-Werner horizon: 0 the cut of Eq. 15, 1 the rough horizon of Section 1
    horizon_mode: int = 0
    # > 0: at most this many lookback slices per observing step
    n_shell_max: int = 0


def _uniform_positions(rng, n, box):
    return rng.uniform(0.0, box, size=(n, 3))


def _clustered_positions(rng, centres, n, box, sigma):
    idx = rng.integers(0, centres.shape[0], size=n)
    p = centres[idx] + rng.normal(0.0, sigma, size=(n, 3))
    return np.mod(p, box)


def _power_law_masses(rng, n, m1, m2):
    # dN/dM ~ M^-2 on [m1, m2]: inverse CDF M = 1 / (1/m1 - u (1/m1 - 1/m2))
    u = rng.uniform(0.0, 1.0, size=n)
    return 1.0 / (1.0 / m1 - u * (1.0 / m1 - 1.0 / m2))


def make_catalogue(seed: int, n_src: int, box: float, n_steps: int, *,
                   clustered: bool, n_centres: int = 100, sigma: float = 2.0,
                   lum_kind: str = "powerlaw", life: Tuple[int, int] = (1, 4)) -> Catalogue:
    rng = np.random.Generator(np.random.PCG64(seed))
    if clustered:
        centres = rng.uniform(0.0, box, size=(n_centres, 3))
        pos = _clustered_positions(rng, centres, n_src, box, sigma)
    else:
        pos = _uniform_positions(rng, n_src, box)
    if lum_kind == "lognormal":
        lum = 10.0 ** rng.normal(0.0, 1.0, size=n_src)
    else:
        lum = _power_law_masses(rng, n_src, 1e8, 1e11) / 1e8
    birth = rng.integers(0, n_steps, size=n_src).astype(np.int64)
    lo, hi = life
    lifetime = rng.integers(lo, hi + 1, size=n_src).astype(np.int64)
    return Catalogue(pos=np.ascontiguousarray(pos), lum=lum, birth=birth, life=lifetime)


def config(name: str) -> Workload:
    """The seeded workloads c1..c3 (single instances)."""
    if name == "c1":
        st = StepSpec(STEPS_EQUAL_TIME, 8, z_start=20.0, z_end=15.0)
        cat = make_catalogue(SEED_BASE + 0, 200, 100.0, 8, clustered=False,
                             lum_kind="lognormal", life=(2, 2))
        return Workload("c1", 32, 100.0, 0.31, 0.68, st, 4, HISTORY_FP32, cat)
    if name == "c2":
        st = StepSpec(STEPS_EQUAL_TIME, 64, z_start=30.0, z_end=10.0)
        cat = make_catalogue(SEED_BASE + 1, 10_000, 150.0, 64, clustered=True,
                             n_centres=100, sigma=2.0)
        return Workload("c2", 128, 150.0, 0.31, 0.68, st, 4, HISTORY_FP32, cat)
    if name == "c3":
        st = StepSpec(STEPS_EQUAL_TAU, 160, z_end=15.0, n_shell=128)
        cat = make_catalogue(SEED_BASE + 2, 100_000, 200.0, 160, clustered=True,
                             n_centres=1000, sigma=2.0)
        return Workload("c3", 256, 200.0, 0.31, 0.68, st, 4, HISTORY_BF16, cat)
    if name == "c3s":
        # the 256^3 BF16 path at a profiling size: 32 equal-conformal-time
        # shells (ring ~1.1 GB), 40 steps, 1e5 clustered sources
        st = StepSpec(STEPS_EQUAL_TAU, 40, z_end=15.0, n_shell=32)
        cat = make_catalogue(SEED_BASE + 77, 100_000, 200.0, 40, clustered=True,
                             n_centres=1000, sigma=2.0)
        return Workload("c3s", 256, 200.0, 0.31, 0.68, st, 4, HISTORY_BF16, cat)
    if name == "c5s":
        # the 512^3 BF16 path of the serving set at a profiling size: 16
        # equal-conformal-time shells (ring ~4.3 GB), 24 steps, 4e4 clustered sources
        st = StepSpec(STEPS_EQUAL_TAU, 24, z_end=15.0, n_shell=16)
        cat = make_catalogue(SEED_BASE + 78, 40_000, 400.0, 24, clustered=True,
                             n_centres=400, sigma=2.0)
        return Workload("c5s", 512, 400.0, 0.31, 0.68, st, 4, HISTORY_BF16, cat)
    if name == "c5m":
        # the 384^3 BF16 path of the serving set at a profiling size: 16
        # equal-conformal-time shells (ring ~1.8 GB), 24 steps, 3e4 clustered sources
        st = StepSpec(STEPS_EQUAL_TAU, 24, z_end=15.0, n_shell=16)
        cat = make_catalogue(SEED_BASE + 79, 30_000, 300.0, 24, clustered=True,
                             n_centres=300, sigma=2.0)
        return Workload("c5m", 384, 300.0, 0.31, 0.68, st, 4, HISTORY_BF16, cat)
    raise KeyError(name)


def small(name: str = "tiny", n: int = 16, box: float = 40.0, n_steps: int = 6,
          n_src: int = 50, seed: int = SEED_BASE + 100, z_start: float = 20.0,
          z_end: float = 15.0, subsamples: int = 4, history: int = HISTORY_FP32,
          clustered: bool = False, life: Tuple[int, int] = (1, 3)) -> Workload:
    """Small cases for parity tests: a few tiles, ragged edges, seconds on the CPU."""
    st = StepSpec(STEPS_EQUAL_TIME, n_steps, z_start=z_start, z_end=z_end)
    cat = make_catalogue(seed, n_src, box, n_steps, clustered=clustered, n_centres=5,
                         sigma=box / 20, lum_kind="lognormal", life=life)
    return Workload(name, n, box, 0.31, 0.68, st, subsamples, history, cat)


def batched_instances() -> List[Workload]:
    """16 uneven instances: grids {64, 96, 128, 192, 256} cycled, shells
    32 + round(96 i / 15), sources log-uniform in [1e3, 1e5], boxes with
    0.78 Mpc cells, equal conformal-time steps ending at z = 15."""
    out = []
    grids = [64, 96, 128, 192, 256]
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 3))
    n_srcs = np.round(10.0 ** rng.uniform(3.0, 5.0, size=16)).astype(int)
    for i in range(16):
        n = grids[i % 5]
        shells = 32 + int(round(96 * i / 15))
        box = 0.78125 * n
        steps = shells + 8
        st = StepSpec(STEPS_EQUAL_TAU, steps, z_end=15.0, n_shell=shells)
        cat = make_catalogue(SEED_BASE + 1000 + i, int(n_srcs[i]), box, steps,
                             clustered=True, n_centres=max(10, int(n_srcs[i]) // 100),
                             sigma=2.0)
        out.append(Workload(f"c4_{i}", n, box, 0.31, 0.68, st, 4, HISTORY_FP32, cat))
    return out


def served_simulations(served_steps: int = 32) -> List[Workload]:
    """8 simulations for the serving loop: N in {128,192,256,256,384,384,512,512},
    64..128 shells (96 at 512^3), BF16 history, 0.78 Mpc cells; each runs
    its shell count of history-filling steps and then `served_steps` steps
    that requests ask for."""
    grids = [128, 192, 256, 256, 384, 384, 512, 512]
    shells = [128, 112, 96, 128, 96, 64, 96, 96]
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 4))
    n_srcs = np.round(10.0 ** rng.uniform(4.0, 5.0, size=8)).astype(int)
    out = []
    for i, (n, sh) in enumerate(zip(grids, shells)):
        box = 0.78125 * n
        steps = sh + served_steps
        st = StepSpec(STEPS_EQUAL_TAU, steps, z_end=15.0, n_shell=sh)
        cat = make_catalogue(SEED_BASE + 2000 + i, int(n_srcs[i]), box, steps,
                             clustered=True, n_centres=max(10, int(n_srcs[i]) // 100),
                             sigma=2.0)
        out.append(Workload(f"c5_{i}", n, box, 0.31, 0.68, st, 4, HISTORY_BF16, cat))
    return out


def sample_cells(seed: int, n: int, count: int, dense_line_through: Optional[np.ndarray] = None) -> np.ndarray:
    """Flat C-order cell indices to evaluate: `count` uniform draws plus,
    optionally, the x-line through a given cell (the densest-cluster line)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cells = rng.integers(0, n ** 3, size=count).astype(np.int64)
    if dense_line_through is not None:
        i, j, k = (int(v) for v in dense_line_through)
        line = np.array([((x * n + j) * n + k) for x in range(n)], dtype=np.int64)
        cells = np.concatenate([cells, line])
    return np.unique(cells)


__all__ = [
    "StepSpec", "Catalogue", "Workload", "config", "small", "batched_instances",
    "served_simulations", "sample_cells", "make_catalogue", "SEED_BASE",
    "STEPS_EXPLICIT", "STEPS_EQUAL_TIME", "STEPS_EQUAL_TAU", "HISTORY_FP32", "HISTORY_BF16",
]
