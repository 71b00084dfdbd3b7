"""FP64 CPU oracle for the light-cone retarded field (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product path (``paper_1502_02294_gb300``)
never does, and the two share no code: this package wraps ``lc_oracle.c``, a
plain double-precision implementation of the paper's definitions (Eqs. 6,
9-11, 14-17), built with gcc + OpenMP.

Pinned against: closed forms of the cosmology (matter-only conformal distance
and time), the paper's printed numbers (f_mod(0) = 1, the horizon constants,
alpha = 1 at the fiducial cosmology, r_LW inside 10 Myr of lookback at
z = 27.90), brute-force symmetry checks, the uniform-source closed form,
linearity, translation and rotation covariance, causality, and a brute-force
DFT checked against numpy on 8^3 grids; the cloud-in-cell deposit by charge
conservation, its first moment, midpoint halves, equality with the nearest
grid point at cell centres and translation covariance; the rough horizon by
its matter-only closed form (see tests/test_oracle_*.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lc_oracle.c")
_LIB = os.path.join(_HERE, "liblc_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2 -fopenmp, no architecture-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("box", ctypes.c_double), ("om", ctypes.c_double),
                ("h", ctypes.c_double), ("n_steps", ctypes.c_int),
                ("z_edges", ctypes.POINTER(ctypes.c_double)), ("subsamples", ctypes.c_int),
                ("normalise", ctypes.c_int), ("out_unit", ctypes.c_double),
                ("kernel", ctypes.c_int), ("k_length", ctypes.c_double), ("k_rmax", ctypes.c_double),
                ("n_shell_max", ctypes.c_int)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        d, i, i64 = ctypes.c_double, ctypes.c_int, ctypes.c_int64
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        pp = ctypes.POINTER(_Problem)
        for name, res, args in [
            ("lco_hubble", d, [d, d, d]), ("lco_chi", d, [d, d, d, d]),
            ("lco_time_myr", d, [d, d, d]), ("lco_z_of_time", d, [d, d, d]),
            ("lco_zs_of_r", d, [d, d, d, d]), ("lco_alpha", d, [d, d, d]),
            ("lco_fmod", d, [d, d]), ("lco_g", d, [d, d, d, d]), ("lco_horizon", d, [d, d, d]),
            ("lco_shell_integral", d, [d, d, d, d, d]),
            ("lco_step_edges", i, [d, d, i, i, d, d, i, dp, dp]),
            ("lco_fk", d, [i, d, d, d, d, d, d]), ("lco_gk", d, [i, d, d, d, d, d, d]),
            ("lco_horizonk", d, [i, d, d, d, d, d]), ("lco_shell_integralk", d, [i, d, d, d, d, d, d, d]),
            ("lco_step_edgesk", i, [i, d, d, d, d, i, i, d, d, i, dp, dp]),
            ("lco_shells", i, [pp, i, dp, dp, dp]), ("lco_active_shells", i, [pp, i]),
            ("lco_rgf_octant", i, [pp, i, i, dp, dp, dp]),
            ("lco_rgf_direct", d, [pp, i, i, i, i, i]),
            ("lco_deposit_ngp", i, [i, d, i64, dp, dp, dp]),
            ("lco_deposit_fixed", i, [i, d, i64, dp, dp, i64p, dp, i64p]),
            ("lco_deposit_cic", i, [i, d, i64, dp, dp, dp]),
            ("lco_deposit_cic_fixed", i, [i, d, i64, dp, dp, i64p, dp, i64p]),
            ("lco_rough_horizon", d, [d]), ("lco_rough_horizon_r", d, [d, d, d]), ("lco_fzero_r", d, [d, d, d]),
            ("lco_field", i, [pp, i, i, ctypes.POINTER(dp), i64, i64p, dp]),
            ("lco_field_sparse", i, [pp, i, i, i64p, i64p, dp, i64, i64p, dp]),
            ("lco_shell_table", i, [pp, i, dp, dp, dp]),
            ("lco_near_cube", i, [pp, i, i64, dp, dp, i, d, i, dp]),
            ("lco_dft3", i, [i, dp, dp, i, dp, dp]), ("lco_threads", i, []),
        ]:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i64p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


# ---------------------------------------------------------------- cosmology
def hubble(om, h, z):
    return lib().lco_hubble(om, h, z)


def chi(om, h, z1, z2):
    return lib().lco_chi(om, h, z1, z2)


def time_myr(om, h, z):
    return lib().lco_time_myr(om, h, z)


def z_of_time(om, h, t):
    return lib().lco_z_of_time(om, h, t)


def zs_of_r(om, h, z_obs, r):
    return lib().lco_zs_of_r(om, h, z_obs, r)


def alpha(om, h, zs):
    return lib().lco_alpha(om, h, zs)


def fmod(r, a):
    return lib().lco_fmod(r, a)


def g(om, h, z_obs, r):
    return lib().lco_g(om, h, z_obs, r)


def horizon(om, h, z_obs):
    return lib().lco_horizon(om, h, z_obs)


def shell_integral(om, h, z_obs, r_lo, r_hi):
    return lib().lco_shell_integral(om, h, z_obs, r_lo, r_hi)


# radial kernels other than the LW one: kernel = (kind, length, rmax), kind 1 =
# exp(-r / length) attenuation with a cut-off at rmax, kind 2 = the LW kernel
# with the rough horizon of Section 1 (see lco_fk)
KERNEL_LW, KERNEL_EXP, KERNEL_LW_ROUGH = 0, 1, 2
DEPOSIT_NGP, DEPOSIT_CIC = 0, 1


def _k(kernel, horizon_mode=0):
    k = (0, 0.0, 0.0) if kernel is None else (int(kernel[0]), float(kernel[1]), float(kernel[2]))
    if horizon_mode and k[0] == KERNEL_LW:
        k = (KERNEL_LW_ROUGH, 0.0, 0.0)
    return k


def rough_horizon(zs):
    """100 [21 / (1 + z_s)]^0.5 comoving Mpc (Section 1)."""
    return lib().lco_rough_horizon(zs)


def rough_horizon_radius(om, h, z_obs):
    """The radius r with r = 100 [21 / (1 + z_s(r))]^0.5 seen from z_obs."""
    return lib().lco_rough_horizon_r(om, h, z_obs)


def fmod_zero_radius(om, h, z_obs):
    """The radius where the unclamped f_mod of Eq. 15 reaches 0, seen from z_obs."""
    return lib().lco_fzero_r(om, h, z_obs)


def g_kernel(kernel, om, h, z_obs, r):
    return lib().lco_gk(*_k(kernel), om, h, z_obs, r)


def horizon_kernel(kernel, om, h, z_obs):
    return lib().lco_horizonk(*_k(kernel), om, h, z_obs)


def shell_integral_kernel(kernel, om, h, z_obs, r_lo, r_hi):
    return lib().lco_shell_integralk(*_k(kernel), om, h, z_obs, r_lo, r_hi)


def step_edges(om, h, spec, kernel=None) -> np.ndarray:
    out = np.zeros(spec.n_steps + 1)
    zx = np.ascontiguousarray(np.asarray(spec.z_edges if spec.z_edges is not None else [0.0], dtype=np.float64))
    rc = lib().lco_step_edgesk(*_k(kernel), om, h, spec.kind, spec.n_steps, spec.z_start, spec.z_end, spec.n_shell,
                               _dp(zx), _dp(out))
    if rc:
        raise ValueError("bad step specification")
    return out


# ---------------------------------------------------------------- problem
class Problem:
    """A workload as the oracle sees it (edges derived here, from the spec)."""

    def __init__(self, n, box, om, h, steps, subsamples=4, normalise=1, out_unit=1.0, kernel=None,
                 horizon_mode=0, n_shell_max=0, deposit=DEPOSIT_NGP):
        self.n, self.box, self.om, self.h = int(n), float(box), float(om), float(h)
        self.steps = steps
        self.kernel = _k(kernel, horizon_mode)
        self.z_edges = step_edges(om, h, steps, self.kernel)
        self.subsamples, self.normalise, self.out_unit = int(subsamples), int(normalise), float(out_unit)
        self.n_shell_max = int(n_shell_max)
        self.deposit = int(deposit)
        self._c = _Problem(self.n, self.box, self.om, self.h, int(steps.n_steps), _dp(self.z_edges),
                           self.subsamples, self.normalise, self.out_unit, *self.kernel, self.n_shell_max)

    @classmethod
    def from_workload(cls, w, **kw):
        args = dict(n=w.n, box=w.box, om=w.omega_m, h=w.h, steps=w.steps, subsamples=w.subsamples,
                    normalise=w.normalise, out_unit=w.out_unit, kernel=getattr(w, "kernel", None),
                    horizon_mode=getattr(w, "horizon_mode", 0), n_shell_max=getattr(w, "n_shell_max", 0),
                    deposit=getattr(w, "deposit", DEPOSIT_NGP))
        args.update(kw)
        return cls(**args)

    @property
    def ref(self):
        return ctypes.byref(self._c)

    def shells(self, s):
        lo = np.zeros(s + 1)
        hi = np.zeros(s + 1)
        rh = ctypes.c_double()
        A = lib().lco_shells(self.ref, s, _dp(lo), _dp(hi), ctypes.byref(rh))
        return lo[:A].copy(), hi[:A].copy(), rh.value

    def active_shells(self, s) -> int:
        return lib().lco_active_shells(self.ref, s)

    def shell_table(self, s):
        lo = np.zeros(s + 1)
        hi = np.zeros(s + 1)
        I = np.zeros(s + 1)
        A = lib().lco_shell_table(self.ref, s, _dp(lo), _dp(hi), _dp(I))
        return lo[:A].copy(), hi[:A].copy(), I[:A].copy()

    def rgf_octant(self, s, j):
        M = self.n // 2
        out = np.zeros((M + 1) ** 3)
        I = ctypes.c_double()
        sm = ctypes.c_double()
        rc = lib().lco_rgf_octant(self.ref, s, j, _dp(out), ctypes.byref(I), ctypes.byref(sm))
        if rc:
            raise ValueError("inactive shell")
        return out.reshape(M + 1, M + 1, M + 1), I.value, sm.value

    def rgf_full(self, s, j) -> np.ndarray:
        """G_j expanded from the octant to the full N^3 grid of displacements."""
        octv, _, _ = self.rgf_octant(s, j)
        N = self.n
        f = np.minimum(np.arange(N), N - np.arange(N))
        return octv[np.ix_(f, f, f)]

    def rgf_direct(self, s, j, d):
        return lib().lco_rgf_direct(self.ref, s, j, int(d[0]), int(d[1]), int(d[2]))

    def field(self, s, src_grids: Sequence[Optional[np.ndarray]], cells: Optional[np.ndarray] = None) -> np.ndarray:
        grids = [None if gr is None else np.ascontiguousarray(gr, dtype=np.float64).ravel() for gr in src_grids]
        arr = (ctypes.POINTER(ctypes.c_double) * max(1, len(grids)))()
        for j, gr in enumerate(grids):
            arr[j] = _dp(gr) if gr is not None else ctypes.POINTER(ctypes.c_double)()
        if cells is None:
            out = np.zeros(self.n ** 3)
            rc = lib().lco_field(self.ref, s, len(grids), arr, 0, ctypes.POINTER(ctypes.c_int64)(), _dp(out))
            out = out.reshape(self.n, self.n, self.n)
        else:
            cells = np.ascontiguousarray(cells, dtype=np.int64)
            out = np.zeros(cells.shape[0])
            rc = lib().lco_field(self.ref, s, len(grids), arr, cells.shape[0], _i64p(cells), _dp(out))
        if rc:
            raise RuntimeError("oracle field failed")
        return out

    def field_sparse(self, s, slices, cells: Optional[np.ndarray] = None) -> np.ndarray:
        """As field(), from each slice's occupied cells: slices[j] = (flat
        C-order indices, FP64 values) of lookback j, or None for no sources."""
        counts = np.array([0 if sl is None else len(sl[0]) for sl in slices] or [0], dtype=np.int64)
        flat = np.ascontiguousarray(np.concatenate([sl[0] for sl in slices if sl is not None] or [np.zeros(0)]),
                                    dtype=np.int64)
        val = np.ascontiguousarray(np.concatenate([sl[1] for sl in slices if sl is not None] or [np.zeros(0)]),
                                   dtype=np.float64)
        n_slices = len(slices)
        if cells is None:
            out = np.zeros(self.n ** 3)
            rc = lib().lco_field_sparse(self.ref, s, n_slices, _i64p(counts), _i64p(flat), _dp(val), 0,
                                        ctypes.POINTER(ctypes.c_int64)(), _dp(out))
            out = out.reshape(self.n, self.n, self.n)
        else:
            cells = np.ascontiguousarray(cells, dtype=np.int64)
            out = np.zeros(cells.shape[0])
            rc = lib().lco_field_sparse(self.ref, s, n_slices, _i64p(counts), _i64p(flat), _dp(val), cells.shape[0],
                                        _i64p(cells), _dp(out))
        if rc:
            raise RuntimeError("oracle field failed")
        return out


# ---------------------------------------------------------------- deposit
def deposit_ngp(n, box, pos, lum) -> np.ndarray:
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    lum = np.ascontiguousarray(lum, dtype=np.float64)
    out = np.zeros(n ** 3)
    rc = lib().lco_deposit_ngp(n, box, lum.shape[0], _dp(pos), _dp(lum), _dp(out))
    if rc:
        raise ValueError("invalid sources")
    return out.reshape(n, n, n)


def deposit_fixed(n, box, pos, lum):
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    lum = np.ascontiguousarray(lum, dtype=np.float64)
    out = np.zeros(n ** 3, dtype=np.int64)
    S = ctypes.c_double()
    tot = ctypes.c_int64()
    rc = lib().lco_deposit_fixed(n, box, lum.shape[0], _dp(pos), _dp(lum), _i64p(out), ctypes.byref(S),
                                 ctypes.byref(tot))
    if rc:
        raise ValueError("invalid sources")
    return out.reshape(n, n, n), S.value, tot.value


def deposit_cic(n, box, pos, lum) -> np.ndarray:
    """FP64 cloud-in-cell luminosity per cell (see lco_deposit_cic)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    lum = np.ascontiguousarray(lum, dtype=np.float64)
    out = np.zeros(n ** 3)
    rc = lib().lco_deposit_cic(n, box, lum.shape[0], _dp(pos), _dp(lum), _dp(out))
    if rc:
        raise ValueError("invalid sources")
    return out.reshape(n, n, n)


def deposit_cic_fixed(n, box, pos, lum):
    """Integer fixed-point cloud-in-cell grid, unit and total (see lco_deposit_cic_fixed)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    lum = np.ascontiguousarray(lum, dtype=np.float64)
    out = np.zeros(n ** 3, dtype=np.int64)
    S = ctypes.c_double()
    tot = ctypes.c_int64()
    rc = lib().lco_deposit_cic_fixed(n, box, lum.shape[0], _dp(pos), _dp(lum), _i64p(out), ctypes.byref(S),
                                     ctypes.byref(tot))
    if rc:
        raise ValueError("invalid sources")
    return out.reshape(n, n, n), S.value, tot.value


def deposit(prob: "Problem", pos, lum) -> np.ndarray:
    """The FP64 source grid of one slice with the problem's assignment (NGP or CIC)."""
    f = deposit_cic if prob.deposit == DEPOSIT_CIC else deposit_ngp
    return f(prob.n, prob.box, pos, lum)


def source_grids(prob: Problem, cat, s: int) -> List[Optional[np.ndarray]]:
    """FP64 source grids of the active slices of step s (index j = lookback)."""
    A = prob.active_shells(s)
    out = []
    for j in range(A):
        pos, lum = cat.active(s - j)
        out.append(deposit(prob, pos, lum) if lum.shape[0] else None)
    return out


def source_lists(prob: Problem, cat, s: int):
    """The occupied cells (flat index, FP64 value) of each active slice of
    step s, one dense grid alive at a time."""
    out = []
    for j in range(prob.active_shells(s)):
        pos, lum = cat.active(s - j)
        if not lum.shape[0]:
            out.append(None)
            continue
        g = deposit(prob, pos, lum).reshape(-1)
        flat = np.flatnonzero(g)
        out.append((flat.astype(np.int64), g[flat].copy()))
        del g
    return out


def field_for(prob: Problem, cat, s: int, cells: Optional[np.ndarray] = None) -> np.ndarray:
    return prob.field_sparse(s, source_lists(prob, cat, s), cells)


NEAR_R = 2  # near cube of the innermost slice: |d| <= NEAR_R cells per axis


def near_cube(prob: Problem, s: int, pos, lum, centred: bool, R: int = NEAR_R) -> np.ndarray:
    """The innermost slice's near cube around each source (see lco_near_cube):
    from the sources' own positions, or (centred) from their NGP cells."""
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    lum = np.ascontiguousarray(lum, dtype=np.float64)
    out = np.zeros(prob.n ** 3)
    if prob.active_shells(s) == 0 or lum.shape[0] == 0:
        return out.reshape((prob.n,) * 3)
    _, I0, sm0 = prob.rgf_octant(s, 0)
    l = prob.box / prob.n
    f0 = I0 / (l ** 3 * sm0) if (prob.normalise and sm0 > 0) else 1.0
    rc = lib().lco_near_cube(prob.ref, s, lum.shape[0], _dp(pos), _dp(lum), int(R), float(f0), int(centred), _dp(out))
    if rc:
        raise ValueError("bad step")
    return out.reshape((prob.n,) * 3)


def hybrid_field_for(prob: Problem, cat, s: int) -> np.ndarray:
    """The field with the particle-mesh hybrid near the sources (Discussion):
    the innermost slice's near cube of every source taken from its position
    instead of its NGP cell; everything else as field_for."""
    J = field_for(prob, cat, s)
    pos, lum = cat.active(s)
    return J - near_cube(prob, s, pos, lum, centred=True) + near_cube(prob, s, pos, lum, centred=False)


def instant_field_for(prob: Problem, cat, s: int, cells: Optional[np.ndarray] = None) -> np.ndarray:
    """Eq. 18: the same shells and kernel, every shell applied to the sources
    of the observing step s (source term frozen at the observing redshift)."""
    A = prob.active_shells(s)
    pos, lum = cat.active(s)
    g = deposit(prob, pos, lum) if lum.shape[0] else None
    return prob.field(s, [g] * A, cells)


def dft3(x: np.ndarray, sign: int = -1) -> np.ndarray:
    n = x.shape[0]
    re = np.ascontiguousarray(x.real, dtype=np.float64).ravel()
    im = np.ascontiguousarray(x.imag, dtype=np.float64).ravel() if np.iscomplexobj(x) else np.zeros(n ** 3)
    ore = np.zeros(n ** 3)
    oim = np.zeros(n ** 3)
    lib().lco_dft3(n, _dp(re), _dp(im), sign, _dp(ore), _dp(oim))
    return (ore + 1j * oim).reshape(n, n, n)


def threads() -> int:
    return lib().lco_threads()
