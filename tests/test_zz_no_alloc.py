"""lc_fft_r2c_static, the allocation-free transform, through the C ABI.

It serves callers that cannot allocate device memory (a pool that owns the
device, a host that forbids cudaMalloc, a loop that must not synchronise):
its scratch is a static device array inside the library.  Checked against
the allocating lc_fft_r2c on two calls in a row (different sizes and data,
so the second call cannot lean on what the first left in the shared array),
within the transform tolerance the other tests use: once with a wait after
each call, once with both calls queued on one stream and a single wait at
the end (calls ordered on one stream share the array safely), and once
through the Python wrapper.  Kept in the last test file so that a failure
here stops a -x run only after everything else.
"""
import ctypes

import numpy as np
import pytest

import paper_1502_02294_gb300 as lc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = (96, 64)


@pytest.fixture(scope="module")
def static_fft():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    lc.build()
    return lc._lib().lc_fft_r2c_static


def _inputs(seed):
    rng = np.random.default_rng(seed)
    return [torch.from_numpy(rng.standard_normal((n, n, n)).astype(np.float32)).cuda() for n in SIZES]


def _call(f, x, out, stream):
    n = x.shape[0]
    return f(n, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))


def _nan_out(n):
    return torch.full((n, n, n // 2 + 1), float("nan"), dtype=torch.complex64, device="cuda")


def _check_against_allocating(x, out):
    ref = lc.fft_r2c(x).cpu().numpy().astype(np.complex128)
    got = out.cpu().numpy().astype(np.complex128)
    assert np.isfinite(got).all()
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 2e-6, (x.shape[0], err)


def test_static_scratch_fft_matches_allocating_fft_twice(static_fft):
    stream = torch.cuda.current_stream()
    for x in _inputs(2024):
        out = _nan_out(x.shape[0])
        assert _call(static_fft, x, out, stream) == lc.LC_OK
        torch.cuda.synchronize()
        _check_against_allocating(x, out)
    # grids beyond the static array are refused with a clear status
    big = torch.zeros((128, 128, 128), dtype=torch.float32, device="cuda")
    bout = torch.empty((128, 128, 65), dtype=torch.complex64, device="cuda")
    assert static_fft(128, ctypes.c_void_p(big.data_ptr()), ctypes.c_void_p(bout.data_ptr()), None) == \
        lc.LC_ERR_UNSUPPORTED_SIZE


def test_static_scratch_calls_queued_on_one_stream(static_fft):
    # two calls back to back on one stream, no wait between them: the second
    # reuses the array the first is still working in, which stream order makes safe
    stream = torch.cuda.current_stream()
    xs = _inputs(7)
    outs = [_nan_out(x.shape[0]) for x in xs]
    for x, o in zip(xs, outs):
        assert _call(static_fft, x, o, stream) == lc.LC_OK
    torch.cuda.synchronize()
    for x, o in zip(xs, outs):
        _check_against_allocating(x, o)


def test_static_scratch_through_python_wrapper(static_fft):
    for x in _inputs(11):
        out = lc.fft_r2c_static(x)
        torch.cuda.synchronize()
        _check_against_allocating(x, out)
