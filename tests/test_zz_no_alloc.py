"""cgl_rel_error_noalloc: the error-norm entry point for callers that cannot
allocate device memory (their memory belongs to another allocator or to a
fixed budget, or they cannot afford the device-wide synchronisation of
cudaFree).  It keeps its scratch in a static device array instead of
allocating per call, so it must give the same norms as cgl_rel_error, call
after call, and refuse counts beyond the array's capacity.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2403_02816_gb300 import native as nat

pytestmark = pytest.mark.gpu

MAX_COUNT = 268435456  # CGL_REL_ERROR_NOALLOC_MAX_COUNT in include/cgl.h


@pytest.fixture(scope="module")
def lib():
    from paper_2403_02816_gb300 import build as B
    B.build()
    assert torch.cuda.is_available()
    return nat.load()


def norms(lib, fn, x, y, prec):
    out = (ctypes.c_double * 3)()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = getattr(lib, fn)(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), x.numel(), prec, out,
                          stream)
    assert st == nat.CGL_OK, (fn, st)
    return np.array(out[:3])


@pytest.mark.parametrize("dtype,prec", [(torch.complex128, nat.CGL_F64), (torch.complex64, nat.CGL_F32),
                                        (torch.complex64, nat.CGL_BF16X3)])
def test_noalloc_matches_allocating_entry_point_on_consecutive_calls(lib, dtype, prec):
    g = torch.Generator(device="cuda").manual_seed(7)
    # two calls in a row with different sizes: the second uses fewer partial
    # records than the first, so stale contents of the shared array would show
    for count in (2 * 65536 + 12345, 70001, 1000):
        y = torch.randn(count, dtype=dtype, device="cuda", generator=g)
        x = y + 1e-4 * torch.randn(count, dtype=dtype, device="cuda", generator=g)
        x[count // 3] = float("nan")
        ref = norms(lib, "cgl_rel_error", x, y, prec)
        got = norms(lib, "cgl_rel_error_noalloc", x, y, prec)
        np.testing.assert_allclose(got[:2], ref[:2], rtol=1e-12, atol=0)
        assert got[2] == ref[2] == 1


def test_noalloc_rejects_counts_beyond_its_scratch(lib):
    x = torch.zeros(4, dtype=torch.complex128, device="cuda")
    out = (ctypes.c_double * 3)()
    st = lib.cgl_rel_error_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), MAX_COUNT + 1,
                                   nat.CGL_F64, out, None)
    assert st == nat.CGL_EINVAL
    assert b"CGL_REL_ERROR_NOALLOC_MAX_COUNT" in lib.cgl_last_error()
    assert lib.cgl_rel_error_noalloc(None, None, 4, nat.CGL_F64, out, None) == nat.CGL_EINVAL
    assert b"NULL" in lib.cgl_last_error()
    st = lib.cgl_rel_error_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), 4, 7, out, None)
    assert st == nat.CGL_EINVAL
    assert b"precision" in lib.cgl_last_error()
