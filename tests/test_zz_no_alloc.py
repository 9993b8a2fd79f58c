"""The allocation-free <Z> entry point (qsim_expval_z_noalloc), called through the C ABI.

Some callers cannot let a library allocate device memory (their memory belongs to another allocator,
or an allocation in a steady-state loop is not acceptable). This entry point keeps its partial sums
in a fixed device array instead; here its results are compared with the allocating qsim_expval_z on
two calls in a row (the second must not see the first call's leftovers), and an oversized request
must be refused. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_09213_gb300 import build
    build.build()
    from paper_2404_09213_gb300 import _lib
    return _lib.lib()


def _states(rng, B, n, dt):
    s = rng.normal(size=(B, 2 ** n)) + 1j * rng.normal(size=(B, 2 ** n))
    s /= np.linalg.norm(s, axis=1, keepdims=True)
    return torch.tensor(s, dtype=dt, device="cuda")


def _call(fn, st, B, n, code):
    z = torch.full((B, n), float("nan"), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(ctypes.c_void_p(st.data_ptr()), B, n, code, ctypes.c_void_p(z.data_ptr()), stream)
    torch.cuda.synchronize()
    return rc, z.cpu().numpy()


@pytest.mark.parametrize("n,B,dt", [(3, 5, torch.complex64), (12, 4, torch.complex128), (16, 3, torch.complex64),
                                    (20, 2, torch.complex64)])
def test_noalloc_matches_allocating_entry_point_twice(lib, n, B, dt):
    rng = np.random.default_rng(n * 7 + B)
    code = 1 if dt == torch.complex128 else 0
    tol = 1e-12 if dt == torch.complex128 else 1e-6
    for call in range(2):   # two calls in a row, different states
        st = _states(rng, B, n, dt)
        rc0, z0 = _call(lib.qsim_expval_z, st, B, n, code)
        rc1, z1 = _call(lib.qsim_expval_z_noalloc, st, B, n, code)
        assert rc0 == 0 and rc1 == 0, lib.qsim_last_error()
        np.testing.assert_allclose(z1, z0, atol=tol, rtol=0)


def test_noalloc_rejects_oversized_requests(lib):
    n, B = 24, 16          # 16 * 2^12 * 13 partial sums > 524288
    st = torch.zeros(1, dtype=torch.complex64, device="cuda")   # never read: rejected before launch
    z = torch.zeros((B, n), dtype=torch.float64, device="cuda")
    rc = lib.qsim_expval_z_noalloc(ctypes.c_void_p(st.data_ptr()), B, n, 0, ctypes.c_void_p(z.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -9
    assert b"fixed scratch" in lib.qsim_last_error()
    assert torch.count_nonzero(z).item() == 0
