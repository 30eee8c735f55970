"""The paper's fourth-order finite-difference matrices and plans with
caller-supplied direction matrices (cgl_fd4_matrix, cgl_plan_create_ex)."""
import ctypes

import numpy as np
import pytest

from oracle import cgl_oracle as O
from paper_2403_02816_gb300 import build as B
from paper_2403_02816_gb300 import native as nat


@pytest.fixture(scope="module")
def lib():
    B.build()
    return nat.load()


@pytest.mark.parametrize("n,lo,hi", [(6, 0.0, 1.0), (17, -3.0, 5.0), (64, -50.0, 50.0)])
@pytest.mark.parametrize("right", [O.DIRICHLET, O.NEUMANN])
def test_fd4_matrix_matches_oracle(lib, n, lo, hi, right):
    got = nat.cgl_fd4_matrix(n, lo, hi, right)
    ref = O.fd4_laplacian(n, lo, hi, right)
    np.testing.assert_allclose(got, ref, rtol=1e-14, atol=1e-14 * np.abs(ref).max())


def test_fd4_matrix_validation(lib):
    out = (ctypes.c_double * 64)()
    assert lib.cgl_fd4_matrix(5, 0.0, 1.0, nat.CGL_BC_DIRICHLET, out) == nat.CGL_EINVAL
    assert lib.cgl_fd4_matrix(8, 1.0, 1.0, nat.CGL_BC_DIRICHLET, out) == nat.CGL_EINVAL
    assert lib.cgl_fd4_matrix(8, 0.0, 1.0, nat.CGL_BC_PERIODIC, out) == nat.CGL_EINVAL
    assert lib.cgl_fd4_matrix(8, 0.0, 1.0, nat.CGL_BC_DIRICHLET, None) == nat.CGL_EINVAL


def test_plan_create_ex_validation_before_any_cuda_call(lib):
    A = [np.eye(8, dtype=complex), np.eye(8, dtype=complex)]
    st, h = nat.cgl_plan_create_ex(A, -1.0, 1.0, 0.0, 0.0, 0.01, nat.CGL_RK4, nat.CGL_F64, stream=0)
    assert st == nat.CGL_EUNSUPPORTED and not h.value
    bad = [np.eye(8, dtype=complex), np.full((8, 8), np.nan, dtype=complex)]
    st, h = nat.cgl_plan_create_ex(bad, -1.0, 1.0, 0.0, 0.0, 0.01, nat.CGL_STRANG, nat.CGL_F64, stream=0)
    assert st == nat.CGL_EINVAL and not h.value
    st, h = nat.cgl_plan_create_ex(A, -1.0, 1.0, 0.0, 0.0, -1.0, nat.CGL_STRANG, nat.CGL_F64, stream=0)
    assert st == nat.CGL_EINVAL and not h.value
    hh = ctypes.c_void_p()
    n = (ctypes.c_int64 * 2)(8, 8)
    assert lib.cgl_plan_create_ex(ctypes.byref(hh), 2, n, None, -1.0, 1.0, 0.0, 0.0, 0.01, 0, 0, None) \
        == nat.CGL_EINVAL
