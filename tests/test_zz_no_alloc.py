"""fch_fft_r2c_noalloc: the standalone R2C transform for callers that must not
allocate device memory once running (another component owns the device memory
budget, cudaMalloc/cudaFree could synchronize the device and stall other work,
or their rules forbid allocation after start-up). Its work array is a fixed
array inside the library, so this test checks, through the C ABI, that two
calls in a row give the same spectra as fch_fft_r2c (which uses a plan's own
work array) and as the FP64 oracle's transform at the largest size, on the
legacy default stream and on a caller's stream with work queued ahead, and that
sizes beyond the fixed array are refused.

Collected last on purpose (file name), so a run that stops at the first
failure has run every other test first; it also passes alone in a fresh process.
"""
import ctypes as C
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
from paper_2006_04784_gb300 import build as B  # noqa: E402

B.build()
from paper_2006_04784_gb300 import fch  # noqa: E402

DEV = torch.device("cuda:0")


def noalloc_fn():
    L = fch.lib()
    f = L.fch_fft_r2c_noalloc
    f.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
    f.restype = C.c_int
    return f


@pytest.mark.parametrize("n,prec", [(512, 0), (512, 1), (128, 0), (64, 1)])
def test_noalloc_r2c_matches_plan_twice(n, prec):
    f = noalloc_fn()
    dt = torch.float64 if prec == 0 else torch.float32
    cdt = torch.complex128 if prec == 0 else torch.complex64
    tol = 1e-13 if prec == 0 else 2e-6  # the transform tolerances of the parity tests
    plan = fch.FFTPlan(n, prec)
    for call in range(2):  # two calls in a row share (and reuse) the fixed array
        batch = 3 if call == 0 else 2
        rng = np.random.default_rng(100 * n + 10 * prec + call)
        x = torch.tensor(rng.standard_normal((batch, n, n)), dtype=dt, device=DEV)
        ref = torch.empty((batch, n // 2 + 1, n), dtype=cdt, device=DEV)
        got = torch.full((batch, n // 2 + 1, n), float("nan"), dtype=cdt, device=DEV)
        torch.cuda.synchronize()
        plan.r2c(x, ref)
        rc = f(n, prec, C.c_void_p(x.data_ptr()), C.c_void_p(got.data_ptr()), batch, None)
        assert rc == 0, fch.lib().fch_last_cuda_error(None)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.isfinite(g).all()
        assert np.abs(g - r).max() <= tol * np.abs(r).max() * math.log2(n)
        if n == 512 and call == 1:
            # the oracle's radix-2 FFT of the last field (kx-major half spectrum)
            o = O.fft2(x[-1].double().cpu().numpy(), -1)[:, : n // 2 + 1].T
            assert np.abs(g[-1] - o).max() <= tol * np.abs(o).max() * math.log2(n)


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_on_a_caller_stream_after_queued_work(prec):
    # the input is produced on the caller's stream behind a long matrix product; the
    # transform enqueued on that stream must see it (stream order, no host wait)
    f = noalloc_fn()
    n, batch = 256, 2
    dt = torch.float64 if prec == 0 else torch.float32
    cdt = torch.complex128 if prec == 0 else torch.complex64
    rng = np.random.default_rng(7 + prec)
    x0 = torch.tensor(rng.standard_normal((batch, n, n)), dtype=dt, device=DEV)
    ref = torch.empty((batch, n // 2 + 1, n), dtype=cdt, device=DEV)
    plan = fch.FFTPlan(n, prec)
    plan.r2c(x0, ref)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    big = torch.ones((4096, 4096), device=DEV)
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(4):
            big = big @ big * (1.0 / 4096)  # queued work ahead of the transform
        x = x0 * 1.0 + big[0, 0].to(dt) * 0.0  # produced on s, after the products
        got = torch.full((batch, n // 2 + 1, n), float("nan"), dtype=cdt, device=DEV)
        rc = f(n, prec, C.c_void_p(x.data_ptr()), C.c_void_p(got.data_ptr()), batch,
               C.c_void_p(s.cuda_stream))
        assert rc == 0, fch.lib().fch_last_cuda_error(None)
    s.synchronize()
    tol = 1e-13 if prec == 0 else 2e-6
    r, g = ref.cpu().numpy(), got.cpu().numpy()
    assert np.isfinite(g).all()
    assert np.abs(g - r).max() <= tol * np.abs(r).max() * math.log2(n)


def test_noalloc_rejects_sizes_beyond_the_fixed_array():
    f = noalloc_fn()
    x = torch.zeros((1, 1024, 1024), dtype=torch.float64, device=DEV)
    X = torch.zeros((1, 513, 1024), dtype=torch.complex128, device=DEV)
    rc = f(1024, 0, C.c_void_p(x.data_ptr()), C.c_void_p(X.data_ptr()), 1, None)
    assert rc == 1
    assert b"exceeds" in fch.lib().fch_last_cuda_error(None)
    assert f(100, 0, C.c_void_p(x.data_ptr()), C.c_void_p(X.data_ptr()), 1, None) == 1
