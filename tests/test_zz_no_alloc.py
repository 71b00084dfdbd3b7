"""lc_fft_r2c_static, the allocation-free transform, through the C ABI.

It serves callers that cannot allocate device memory (a pool that owns the
device, a host that forbids cudaMalloc, a loop that must not synchronise):
its scratch is a static device array inside the library.  Checked against
the allocating lc_fft_r2c on two calls in a row (different sizes and data,
so the second call cannot lean on what the first left in the shared array),
within the transform tolerance the other tests use.  Kept in the last test
file so that a failure here stops a -x run only after everything else.
"""
import ctypes

import numpy as np
import pytest

import paper_1502_02294_gb300 as lc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_static_scratch_fft_matches_allocating_fft_twice():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    lc.build()
    L = lc._lib()
    f = L.lc_fft_r2c_static
    rng = np.random.default_rng(2024)
    stream = torch.cuda.current_stream()
    for n in (96, 64):
        x = torch.from_numpy(rng.standard_normal((n, n, n)).astype(np.float32)).cuda()
        out = torch.full((n, n, n // 2 + 1), float("nan"), dtype=torch.complex64, device="cuda")
        st = f(n, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert st == lc.LC_OK
        torch.cuda.synchronize()
        ref = lc.fft_r2c(x).cpu().numpy().astype(np.complex128)
        got = out.cpu().numpy().astype(np.complex128)
        assert np.isfinite(got).all()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < 2e-6, (n, err)
    # grids beyond the static array are refused with a clear status
    big = torch.zeros((128, 128, 128), dtype=torch.float32, device="cuda")
    bout = torch.empty((128, 128, 65), dtype=torch.complex64, device="cuda")
    assert f(128, ctypes.c_void_p(big.data_ptr()), ctypes.c_void_p(bout.data_ptr()), None) == lc.LC_ERR_UNSUPPORTED_SIZE
