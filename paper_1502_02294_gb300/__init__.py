"""GB300-native light-cone (retarded) radiation field of Ahn 2015 (arXiv:1502.02294).

A thin ctypes binding over ``liblc.so`` (C ABI declared in ``include/lc.h``).
It only marshals arguments: the deposit, the FFTs, the Green's function
builder and the shell multiply-accumulate all run in the library's CUDA
kernels.  There is no CPU fallback: if the library is missing or no CUDA
device is present the calls raise.

PyTorch provides device memory and streams.  Host inputs may be numpy arrays;
device inputs are torch CUDA tensors (float64 positions/luminosities, float32
output).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblc.so")

LC_OK, LC_ERR_INVALID_ARG, LC_ERR_UNSUPPORTED_SIZE, LC_ERR_STEP_ORDER = 0, 1, 2, 3
LC_ERR_OOM, LC_ERR_CUDA, LC_ERR_TIMEOUT, LC_ERR_DEVICE_CHECK = 4, 5, 6, 7
STEPS_EXPLICIT, STEPS_EQUAL_TIME, STEPS_EQUAL_TAU = 0, 1, 2
HISTORY_FP32, HISTORY_BF16 = 0, 1
KERNEL_LW, KERNEL_EXP = 0, 1  # radial kernels (lc_steps.kernel)
NEAR_NGP, NEAR_SUBCELL, NEAR_NONE = 0, 1, 2  # near field of the innermost slice (lc_steps.near_mode)
DEPOSIT_NGP, DEPOSIT_CIC = 0, 1  # source assignment (lc_steps.deposit)
HORIZON_EQ15, HORIZON_ROUGH = 0, 1  # Lyman-Werner horizon (lc_steps.horizon_mode)
SUPPORTED_N = (8, 16, 32, 64, 96, 128, 192, 256, 384, 512)
PHASES = ("deposit", "r2c_z", "fwd_y", "fwd_x_ring", "mac_x", "inv_y", "c2r_z", "near")


def autotune_report() -> dict:
    """The autotuner's current kernel choices: {key: variant}."""
    n = _lib().lc_autotune_report(None, 0)
    buf = ctypes.create_string_buffer(n + 1)
    _lib().lc_autotune_report(buf, n + 1)
    out = {}
    for line in buf.value.decode().splitlines():
        k, v = line.split()
        out[k] = v
    return out


FFT_STAGES, FFT_LANES, FFT_LANES3, FFT_TMA, FFT_TMA4, FFT_PLANE4 = 0, 1, 2, 3, 4, 5  # FFT pass forms


def fft_set_variant(n: int, variant: int):
    """Force the FFT pass form for grid size n (one of FFT_STAGES ... FFT_PLANE4)."""
    _check(_lib().lc_fft_set_variant(int(n), int(variant)), "lc_fft_set_variant")


def fft_variant(n: int) -> int:
    """The FFT pass form in use for grid size n (-1: n not supported)."""
    return int(_lib().lc_fft_variant(int(n)))


def kernel_launches() -> int:
    """Kernels liblc has launched in this process."""
    return int(_lib().lc_kernel_launches())


class LCError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {_lib().lc_status_string(status).decode()} (status {status})")


class _Cosmology(ctypes.Structure):
    _fields_ = [("omega_m", ctypes.c_double), ("h", ctypes.c_double)]


class _Steps(ctypes.Structure):
    _fields_ = [("n_steps", ctypes.c_int), ("spacing", ctypes.c_int),
                ("z_edges", ctypes.POINTER(ctypes.c_double)), ("z_start", ctypes.c_double),
                ("z_end", ctypes.c_double), ("n_shell", ctypes.c_int), ("subsamples", ctypes.c_int),
                ("history", ctypes.c_int), ("normalise", ctypes.c_int), ("out_unit", ctypes.c_double),
                ("kernel", ctypes.c_int), ("kernel_length", ctypes.c_double), ("kernel_rmax", ctypes.c_double),
                ("near_mode", ctypes.c_int), ("deposit", ctypes.c_int), ("horizon_mode", ctypes.c_int),
                ("n_shell_max", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("n_steps", ctypes.c_int), ("n_ring", ctypes.c_int),
                ("history", ctypes.c_int), ("wedge_size", ctypes.c_int), ("spectrum_row", ctypes.c_int),
                ("box_mpc", ctypes.c_double), ("z_edges", ctypes.POINTER(ctypes.c_double))]


# (name, restype, argtypes) of every entry point declared in include/lc.h
_P, _D, _I, _I64, _VP = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
SIGNATURES = [
    ("lc_plan_create", _I, [_I, _D, ctypes.POINTER(_Cosmology), ctypes.POINTER(_Steps), _VP, ctypes.POINTER(_P)]),
    ("lc_plan_prepare", _I, [_P, _I, _I]),
    ("lc_push_sources", _I, [_P, _I, _I64, _VP, _VP]),
    ("lc_retarded_field", _I, [_P, _I, _VP]),
    ("lc_instant_field", _I, [_P, _I, _VP]),
    ("lc_retarded_field_async", _I, [_P, _I, _VP, ctypes.POINTER(ctypes.c_uint64)]),
    ("lc_plan_wait", _I, [_P, ctypes.c_uint64]),
    ("lc_plan_poll", _I, [_P, ctypes.c_uint64, ctypes.POINTER(_I)]),
    ("lc_plan_reset", _I, [_P]),
    ("lc_plan_check", _I, [_P]),
    ("lc_plan_set_stream", _I, [_P, _VP]),
    ("lc_plan_destroy", _I, [_P]),
    ("lc_status_string", ctypes.c_char_p, [_I]),
    ("lc_plan_device_bytes", ctypes.c_size_t, [_P]),
    ("lc_plan_estimate", _I, [_I, ctypes.POINTER(_Steps), ctypes.POINTER(_Cosmology),
                              ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
    ("lc_step_shells", _I, [_P, _I, ctypes.POINTER(_I), _DP, _DP, _DP, _DP]),
    ("lc_plan_info", _I, [_P, ctypes.POINTER(_Info)]),
    ("lc_plan_green_wedge", _I, [_P, _I, _I, _VP, _DP]),
    ("lc_batch_step", _I, [ctypes.POINTER(_P), _I, ctypes.POINTER(_I), ctypes.POINTER(_I64),
                           ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP)]),
    ("lc_graph_create", _I, [_P, _I, _I64, _VP, _VP, _VP, ctypes.POINTER(_P)]),
    ("lc_graph_launch", _I, [_P]),
    ("lc_graph_destroy", _I, [_P]),
    ("lc_batch_graph_create", _I, [ctypes.POINTER(_P), _I, ctypes.POINTER(_I), ctypes.POINTER(_I64),
                                   ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_P)]),
    ("lc_batch_graph_launch", _I, [_P, _VP]),
    ("lc_batch_graph_destroy", _I, [_P]),
    ("lc_plan_set_timing", _I, [_P, _I]),
    ("lc_plan_timing", _I, [_P, _DP, ctypes.POINTER(_I64), _I]),
    ("lc_kernel_launches", ctypes.c_uint64, []),
    ("lc_deposit_grid", _I, [_I, _D, _I, _I64, _VP, _VP, _VP, _DP, ctypes.POINTER(_I64), _VP]),
    ("lc_fft_r2c", _I, [_I, _VP, _VP, _VP]),
    ("lc_fft_c2r", _I, [_I, _VP, _VP, ctypes.c_float, _VP]),
    ("lc_fft_r2c_static", _I, [_I, _VP, _VP, _VP]),
    ("lc_autotune_report", _I, [ctypes.c_char_p, _I]),
    ("lc_fft_set_variant", _I, [_I, _I]),
    ("lc_fft_variant", _I, [_I]),
    ("lc_fdiff_map", _I, [_I64, _VP, _VP, _VP, _VP]),
    ("lc_plan_set_table_budget", _I, [_P, ctypes.c_size_t]),
    ("lc_plan_table_bytes", ctypes.c_size_t, [_P]),
    ("lc_plan_checkpoint_bytes", ctypes.c_size_t, [_P]),
    ("lc_plan_save", _I, [_P, _VP, ctypes.c_size_t]),
    ("lc_plan_load", _I, [_P, _VP, ctypes.c_size_t]),
]

_L = None


def _lib():
    global _L
    if _L is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"liblc.so is not built ({LIB_PATH}); run paper_1502_02294_gb300._build.build() "
                               "-- there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _L = L
    return _L


def build(force: bool = False) -> str:
    from . import _build

    return _build.build(force=force)


def _check(st: int, what: str):
    if st != LC_OK:
        raise LCError(st, what)


def _torch():
    import torch

    return torch


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        torch = _torch()
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
        return None
    return stream if isinstance(stream, int) else stream.cuda_stream


def _ptr(x, dtype) -> Tuple[int, object]:
    """Pointer to a contiguous buffer of `dtype` (host numpy or torch tensor); returns (ptr, keepalive)."""
    if x is None:
        return 0, None
    if hasattr(x, "data_ptr"):  # torch tensor
        torch = _torch()
        want = {np.float64: torch.float64, np.float32: torch.float32, np.int64: torch.int64}[dtype]
        if x.dtype != want or not x.is_contiguous():
            x = x.to(want).contiguous()
        return x.data_ptr(), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, a


def _steps_struct(spec, subsamples=4, history=HISTORY_FP32, normalise=1, out_unit=1.0, kernel=None, near_mode=0,
                  deposit=DEPOSIT_NGP, horizon_mode=HORIZON_EQ15, n_shell_max=0):
    z = None
    zp = ctypes.POINTER(ctypes.c_double)()
    if getattr(spec, "z_edges", None) is not None:
        z = np.ascontiguousarray(spec.z_edges, dtype=np.float64)
        zp = z.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = _Steps(int(spec.n_steps), int(spec.kind), zp, float(getattr(spec, "z_start", 0.0)),
                float(getattr(spec, "z_end", 0.0)), int(getattr(spec, "n_shell", 0)), int(subsamples), int(history),
                int(normalise), float(out_unit), *_kernel_fields(kernel), int(near_mode), int(deposit),
                int(horizon_mode), int(n_shell_max))
    return st, z


def _kernel_fields(kernel):
    """(kind, length, rmax) from None (the LW kernel) or a (kind, length, rmax) tuple."""
    if kernel is None:
        return KERNEL_LW, 0.0, 0.0
    kind, length, rmax = kernel
    return int(kind), float(length), float(rmax)


class Plan:
    """One simulation's light-cone field: Green's function tables, a device
    ring of past source spectra, and the per-step push/field calls.

    ``steps`` is any object with ``kind`` (STEPS_*), ``n_steps`` and, by kind,
    ``z_start``/``z_end``/``n_shell``/``z_edges``.
    """

    def __init__(self, n: int, box: float, omega_m: float, h: float, steps, subsamples: int = 4,
                 history: int = HISTORY_FP32, normalise: int = 1, out_unit: float = 1.0, stream=None,
                 kernel=None, near_mode: int = NEAR_NGP, deposit: int = DEPOSIT_NGP,
                 horizon_mode: int = HORIZON_EQ15, n_shell_max: int = 0):
        L = _lib()
        self.n, self.box = int(n), float(box)
        self._cos = _Cosmology(float(omega_m), float(h))
        self._steps, self._zkeep = _steps_struct(steps, subsamples, history, normalise, out_unit, kernel, near_mode,
                                                 deposit, horizon_mode, n_shell_max)
        self._stream = _stream_ptr(stream)
        h_ = ctypes.c_void_p()
        _check(L.lc_plan_create(self.n, self.box, ctypes.byref(self._cos), ctypes.byref(self._steps),
                                self._stream, ctypes.byref(h_)), "lc_plan_create")
        self._h = h_
        info = _Info()
        _check(L.lc_plan_info(self._h, ctypes.byref(info)), "lc_plan_info")
        self.n_steps = info.n_steps
        self.n_ring = info.n_ring
        self.history = info.history
        self.wedge_size = info.wedge_size
        self.z_edges = np.array([info.z_edges[i] for i in range(self.n_steps + 1)])

    @classmethod
    def from_workload(cls, w, stream=None, **kw):
        args = dict(n=w.n, box=w.box, omega_m=w.omega_m, h=w.h, steps=w.steps, subsamples=w.subsamples,
                    history=w.history, normalise=w.normalise, out_unit=w.out_unit, stream=stream,
                    kernel=getattr(w, "kernel", None), near_mode=getattr(w, "near_mode", 0),
                    deposit=getattr(w, "deposit", DEPOSIT_NGP), horizon_mode=getattr(w, "horizon_mode", HORIZON_EQ15),
                    n_shell_max=getattr(w, "n_shell_max", 0))
        args.update(kw)
        return cls(**args)

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None):
            _lib().lc_plan_destroy(self._h)  # also destroys its step graphs
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- calls
    def prepare(self, begin: int = 0, end: Optional[int] = None):
        _check(_lib().lc_plan_prepare(self._h, int(begin), int(self.n_steps if end is None else end)),
               "lc_plan_prepare")

    def push(self, step: int, pos, lum):
        n = int(lum.shape[0]) if lum is not None else 0
        pp, k1 = _ptr(pos, np.float64)
        lp, k2 = _ptr(lum, np.float64)
        _check(_lib().lc_push_sources(self._h, int(step), n, pp if n else None, lp if n else None),
               "lc_push_sources")

    def field(self, step: int, out=None):
        """Retarded field at the end of `step` into `out` (torch CUDA tensor or
        numpy array of N^3 float32); a new CUDA tensor if out is None."""
        if out is None:
            torch = _torch()
            out = torch.empty((self.n,) * 3, dtype=torch.float32, device="cuda")
        if isinstance(out, np.ndarray):
            assert out.dtype == np.float32 and out.flags.c_contiguous and out.size == self.n ** 3
            ptr = out.ctypes.data
        else:
            assert out.dtype.itemsize == 4 and out.is_contiguous() and out.numel() == self.n ** 3
            ptr = out.data_ptr()
        _check(_lib().lc_retarded_field(self._h, int(step), ptr), "lc_retarded_field")
        return out

    def field_async(self, step: int, out) -> int:
        """Enqueue the retarded field of `step` into `out` and return a ticket.
        A host `out` (numpy, or a pinned torch CPU tensor) is filled by a copy
        that overlaps the next steps' work: read it only after wait(ticket).
        A CUDA `out` is stream-ordered (ticket 0)."""
        if isinstance(out, np.ndarray):
            assert out.dtype == np.float32 and out.flags.c_contiguous and out.size == self.n ** 3
            ptr = out.ctypes.data
        else:
            assert out.dtype.itemsize == 4 and out.is_contiguous() and out.numel() == self.n ** 3
            ptr = out.data_ptr()
        t = ctypes.c_uint64()
        _check(_lib().lc_retarded_field_async(self._h, int(step), ptr, ctypes.byref(t)), "lc_retarded_field_async")
        return int(t.value)

    def wait(self, ticket: int):
        """Block until the output of `ticket` (from field_async) is in place."""
        _check(_lib().lc_plan_wait(self._h, int(ticket)), "lc_plan_wait")

    def poll(self, ticket: int) -> bool:
        """True once the output of `ticket` (from field_async) is in place; never blocks."""
        d = ctypes.c_int()
        _check(_lib().lc_plan_poll(self._h, int(ticket), ctypes.byref(d)), "lc_plan_poll")
        return bool(d.value)

    def instant_field(self, step: int, out=None):
        """Action-at-a-distance field of Eq. 18: every shell sees the sources
        of `step` itself (the last pushed step)."""
        if out is None:
            torch = _torch()
            out = torch.empty((self.n,) * 3, dtype=torch.float32, device="cuda")
        ptr = out.ctypes.data if isinstance(out, np.ndarray) else out.data_ptr()
        _check(_lib().lc_instant_field(self._h, int(step), ptr), "lc_instant_field")
        return out

    def reset(self):
        _check(_lib().lc_plan_reset(self._h), "lc_plan_reset")

    def check(self):
        _check(_lib().lc_plan_check(self._h), "lc_plan_check")

    def set_stream(self, stream):
        self._stream = _stream_ptr(stream)
        _check(_lib().lc_plan_set_stream(self._h, self._stream), "lc_plan_set_stream")

    @property
    def device_bytes(self) -> int:
        return int(_lib().lc_plan_device_bytes(self._h))

    def shells(self, step: int, integrals: bool = False):
        k = step + 1
        lo, hi, I = np.zeros(k), np.zeros(k), np.zeros(k)
        rh = ctypes.c_double()
        A = ctypes.c_int()
        dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
        _check(_lib().lc_step_shells(self._h, int(step), ctypes.byref(A), dp(lo), dp(hi), ctypes.byref(rh),
                                     dp(I) if integrals else ctypes.POINTER(ctypes.c_double)()), "lc_step_shells")
        a = A.value
        return (lo[:a], hi[:a], rh.value, I[:a]) if integrals else (lo[:a], hi[:a], rh.value)

    def graph(self, step: int, pos, lum, out) -> "StepGraph":
        """Capture push(step) + field(step) on device buffers as one CUDA graph."""
        return StepGraph(self, step, pos, lum, out)

    def set_timing(self, enable: bool = True):
        _check(_lib().lc_plan_set_timing(self._h, int(bool(enable))), "lc_plan_set_timing")

    def timing(self, reset: bool = False):
        """Accumulated per-phase device milliseconds and launch counts."""
        ms = np.zeros(len(PHASES))
        cnt = np.zeros(len(PHASES), dtype=np.int64)
        _check(_lib().lc_plan_timing(self._h, ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), int(reset)), "lc_plan_timing")
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(PHASES)}

    def set_table_budget(self, nbytes: int):
        """Keep the Green's-function tables under nbytes (0: no limit)."""
        _check(_lib().lc_plan_set_table_budget(self._h, int(nbytes)), "lc_plan_set_table_budget")

    @property
    def table_bytes(self) -> int:
        return int(_lib().lc_plan_table_bytes(self._h))

    def checkpoint_bytes(self) -> int:
        return int(_lib().lc_plan_checkpoint_bytes(self._h))

    def save(self, buf=None):
        """Write the plan's history state into `buf` (numpy uint8 array or torch
        uint8 tensor, host or device); a new numpy array if buf is None."""
        n = self.checkpoint_bytes()
        if buf is None:
            buf = np.empty(n, dtype=np.uint8)
        ptr = buf.ctypes.data if isinstance(buf, np.ndarray) else buf.data_ptr()
        size = buf.nbytes if isinstance(buf, np.ndarray) else buf.numel() * buf.element_size()
        _check(_lib().lc_plan_save(self._h, ptr, size), "lc_plan_save")
        return buf

    def load(self, buf):
        """Restore a state written by save() of a plan with the same parameters."""
        ptr = buf.ctypes.data if isinstance(buf, np.ndarray) else buf.data_ptr()
        size = buf.nbytes if isinstance(buf, np.ndarray) else buf.numel() * buf.element_size()
        _check(_lib().lc_plan_load(self._h, ptr, size), "lc_plan_load")

    def green_wedge(self, step: int, lookback: int):
        out = np.zeros(self.wedge_size, dtype=np.float32)
        g0 = ctypes.c_double()
        _check(_lib().lc_plan_green_wedge(self._h, int(step), int(lookback), out.ctypes.data, ctypes.byref(g0)),
               "lc_plan_green_wedge")
        return out, g0.value


class StepGraph:
    """A whole step (deposit, forward transform into the ring, shell MAC,
    inverse transform) replayed with one launch; inputs/output are the device
    tensors given at capture."""

    def __init__(self, plan: Plan, step: int, pos, lum, out):
        n = int(lum.shape[0])
        self.plan, self.step = plan, int(step)
        self._keep = (pos, lum, out)
        h = ctypes.c_void_p()
        _check(_lib().lc_graph_create(plan._h, self.step, n, pos.data_ptr() if n else None,
                                      lum.data_ptr() if n else None, out.data_ptr(), ctypes.byref(h)),
               "lc_graph_create")
        self._g = h

    def launch(self):
        _check(_lib().lc_graph_launch(self._g), "lc_graph_launch")

    def close(self):
        if getattr(self, "_g", None) and self.plan._h:
            _lib().lc_graph_destroy(self._g)
        self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchGraph:
    """One step of several (uneven) plans captured as one CUDA graph whose
    branches run concurrently; `sources[i]` = (pos, lum) device tensors,
    `outs[i]` a device float32 tensor of plans[i].n ** 3."""

    def __init__(self, plans, steps, sources, outs):
        n = len(plans)
        self.plans = list(plans)
        self._keep = (list(sources), list(outs))
        hp = (ctypes.c_void_p * n)(*[p._h for p in plans])
        st = (ctypes.c_int * n)(*[int(s) for s in steps])
        ns = (ctypes.c_int64 * n)(*[int(src[1].shape[0]) for src in sources])
        pp = (ctypes.c_void_p * n)(*[src[0].data_ptr() if src[1].shape[0] else None for src in sources])
        lp = (ctypes.c_void_p * n)(*[src[1].data_ptr() if src[1].shape[0] else None for src in sources])
        op = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
        h = ctypes.c_void_p()
        _check(_lib().lc_batch_graph_create(hp, n, st, ns, pp, lp, op, ctypes.byref(h)), "lc_batch_graph_create")
        self._g = h

    def launch(self, stream=None):
        _check(_lib().lc_batch_graph_launch(self._g, _stream_ptr(stream)), "lc_batch_graph_launch")

    def close(self):
        if getattr(self, "_g", None):
            _lib().lc_batch_graph_destroy(self._g)
        self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_step(plans, steps, sources, outs):
    """Push (if sources[i] is not None) and evaluate several plans at once."""
    n = len(plans)
    hp = (ctypes.c_void_p * n)(*[p._h for p in plans])
    st = (ctypes.c_int * n)(*[int(s) for s in steps])
    ns = (ctypes.c_int64 * n)()
    pp = (ctypes.c_void_p * n)()
    lp = (ctypes.c_void_p * n)()
    op = (ctypes.c_void_p * n)()
    keep = []
    for i in range(n):
        if sources[i] is None:
            ns[i] = -1
        else:
            pos, lum = sources[i]
            ns[i] = int(lum.shape[0])
            a, k1 = _ptr(pos, np.float64)
            b, k2 = _ptr(lum, np.float64)
            keep += [k1, k2]
            pp[i], lp[i] = a, b
        op[i] = outs[i].data_ptr()
    _check(_lib().lc_batch_step(hp, n, st, ns, pp, lp, op), "lc_batch_step")


def estimate_bytes(n, steps, omega_m, h, history=HISTORY_FP32, kernel=None, horizon_mode=HORIZON_EQ15,
                   n_shell_max=0) -> Tuple[int, int]:
    st, keep = _steps_struct(steps, 4, history, kernel=kernel, horizon_mode=horizon_mode, n_shell_max=n_shell_max)
    c = _Cosmology(omega_m, h)
    b = ctypes.c_size_t()
    t = ctypes.c_size_t()
    _check(_lib().lc_plan_estimate(int(n), ctypes.byref(st), ctypes.byref(c), ctypes.byref(b), ctypes.byref(t)),
           "lc_plan_estimate")
    return int(b.value), int(t.value)


def fdiff_map(j_retarded, j_instant, out=None, stream=None):
    """f_diff = (J_instant - J) / J per cell (torch CUDA float32 tensors)."""
    torch = _torch()
    assert j_retarded.dtype == torch.float32 and j_instant.dtype == torch.float32
    assert j_retarded.is_contiguous() and j_instant.is_contiguous() and j_retarded.numel() == j_instant.numel()
    if out is None:
        out = torch.empty_like(j_retarded)
    _check(_lib().lc_fdiff_map(j_retarded.numel(), j_retarded.data_ptr(), j_instant.data_ptr(), out.data_ptr(),
                               _stream_ptr(stream)), "lc_fdiff_map")
    return out


def deposit_grid(n: int, box: float, pos, lum, out=None, stream=None, deposit: int = DEPOSIT_NGP):
    """Fixed-point deposit (nearest grid point or cloud in cell) on the device:
    returns (int64 grid, scale, total)."""
    nsrc = int(lum.shape[0])
    if out is None:
        out = np.zeros((n, n, n), dtype=np.int64)
    pp, k1 = _ptr(pos, np.float64)
    lp, k2 = _ptr(lum, np.float64)
    optr = out.ctypes.data if isinstance(out, np.ndarray) else out.data_ptr()
    S = ctypes.c_double()
    tot = ctypes.c_int64()
    _check(_lib().lc_deposit_grid(int(n), float(box), int(deposit), nsrc, pp if nsrc else None, lp if nsrc else None, optr,
                                  ctypes.byref(S), ctypes.byref(tot), _stream_ptr(stream)), "lc_deposit_grid")
    return out, S.value, tot.value


def fft_r2c(x, stream=None):
    """3D real-to-complex forward transform (Eq. 12 sign) of a cubic float32 CUDA tensor."""
    torch = _torch()
    n = x.shape[0]
    x = x.contiguous().to(torch.float32)
    out = torch.empty((n, n, n // 2 + 1), dtype=torch.complex64, device=x.device)
    _check(_lib().lc_fft_r2c(n, x.data_ptr(), out.data_ptr(), _stream_ptr(stream)), "lc_fft_r2c")
    return out


def fft_r2c_static(x, out=None, stream=None):
    """fft_r2c without device allocation inside the library (N <= 96); the
    result is enqueued on the stream, not waited for.

    `x` must be a cubic CUDA tensor; it is made a contiguous float32 tensor
    first (which may copy it, on the caller's side).  `out`, if given, must be
    a contiguous complex64 CUDA tensor of shape (N, N, N/2 + 1) on x's device;
    anything else raises ValueError before the library is called."""
    torch = _torch()
    if not getattr(x, "is_cuda", False):
        raise ValueError("fft_r2c_static: x must be a CUDA tensor")
    if x.dim() != 3 or not (x.shape[0] == x.shape[1] == x.shape[2]):
        raise ValueError(f"fft_r2c_static: x must be cubic (N, N, N), got {tuple(x.shape)}")
    n = int(x.shape[0])
    x = x.contiguous().to(torch.float32)
    if out is None:
        out = torch.empty((n, n, n // 2 + 1), dtype=torch.complex64, device=x.device)
    elif (not getattr(out, "is_cuda", False) or out.device != x.device or out.dtype != torch.complex64
          or not out.is_contiguous() or tuple(out.shape) != (n, n, n // 2 + 1)):
        raise ValueError("fft_r2c_static: out must be a contiguous complex64 CUDA tensor of shape "
                         f"({n}, {n}, {n // 2 + 1}) on {x.device}")
    _check(_lib().lc_fft_r2c_static(n, x.data_ptr(), out.data_ptr(), _stream_ptr(stream)), "lc_fft_r2c_static")
    return out


def fft_c2r(X, scale: Optional[float] = None, stream=None):
    """Inverse of Eq. 12 (times `scale`, default 1/N^3) of a (N, N, N/2+1) complex64 CUDA tensor."""
    torch = _torch()
    n = X.shape[0]
    X = X.contiguous().to(torch.complex64)
    out = torch.empty((n, n, n), dtype=torch.float32, device=X.device)
    s = 1.0 / n ** 3 if scale is None else float(scale)
    _check(_lib().lc_fft_c2r(n, X.data_ptr(), out.data_ptr(), ctypes.c_float(s), _stream_ptr(stream)), "lc_fft_c2r")
    return out


__all__ = ["Plan", "StepGraph", "BatchGraph", "batch_step", "deposit_grid", "fft_r2c", "fft_r2c_static", "fft_c2r",
           "build", "estimate_bytes", "LCError",
           "SIGNATURES", "LIB_PATH", "SUPPORTED_N", "STEPS_EXPLICIT", "STEPS_EQUAL_TIME", "STEPS_EQUAL_TAU",
           "HISTORY_FP32", "HISTORY_BF16", "DEPOSIT_NGP", "DEPOSIT_CIC", "HORIZON_EQ15", "HORIZON_ROUGH"]
