"""The C-ABI library loads and exports every symbol include/cgl.h declares;
argument validation that happens before any CUDA call (no GPU needed)."""
import ctypes

import pytest

from paper_2403_02816_gb300 import build as B
from paper_2403_02816_gb300 import native as nat


@pytest.fixture(scope="module")
def lib():
    B.build()
    return nat.load()


def test_header_declares_the_entry_points():
    names = nat.header_functions()
    for need in ["cgl_plan_create", "cgl_step", "cgl_plan_destroy", "cgl_step_host", "cgl_linear_flow",
                 "cgl_rel_error", "cgl_strerror"]:
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in nat.header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror(lib):
    assert lib.cgl_strerror(0) == b"ok"
    assert lib.cgl_strerror(nat.CGL_EINVAL) == b"invalid argument"
    assert lib.cgl_strerror(nat.CGL_ENONFINITE) == b"non-finite value produced"
    assert lib.cgl_strerror(12345) == b"unknown status"


def create(**kw):
    base = dict(d=2, n=[8, 8], bc=[0, 0], lo=[-1.0, -1.0], hi=[1.0, 1.0], a1=1.0, b1=0.5, a2=1.0, a3=-1.0,
                b3=1.2, a4=0.0, b4=0.0, tau=0.01, scheme=nat.CGL_STRANG, precision=nat.CGL_F64)
    base.update(kw)
    return nat.cgl_plan_create(base["d"], base["n"], base["bc"], base["lo"], base["hi"], base["a1"], base["b1"],
                               base["a2"], base["a3"], base["b3"], base["a4"], base["b4"], base["tau"],
                               base["scheme"], base["precision"], stream=0)


@pytest.mark.parametrize("kw,status", [
    (dict(d=0, n=[], bc=[], lo=[], hi=[]), nat.CGL_EINVAL),
    (dict(d=4, n=[2] * 4, bc=[0] * 4, lo=[0.0] * 4, hi=[1.0] * 4), nat.CGL_EINVAL),
    (dict(n=[1, 8]), nat.CGL_EINVAL),
    (dict(a1=0.0), nat.CGL_EINVAL),
    (dict(a1=-1.0), nat.CGL_EINVAL),
    (dict(tau=0.0), nat.CGL_EINVAL),
    (dict(tau=float("nan")), nat.CGL_EINVAL),
    (dict(b3=float("inf")), nat.CGL_EINVAL),
    (dict(lo=[1.0, -1.0]), nat.CGL_EINVAL),
    (dict(bc=[0, 7]), nat.CGL_EINVAL),
    (dict(scheme=99), nat.CGL_EINVAL),
    (dict(precision=7), nat.CGL_EINVAL),
    (dict(bc=[2, 0]), nat.CGL_EUNSUPPORTED),
    (dict(bc=[2, 2], n=[8, 22]), nat.CGL_EUNSUPPORTED),
    (dict(bc=[2, 2], n=[8, 4096]), nat.CGL_EUNSUPPORTED),
    (dict(n=[8, 2048]), nat.CGL_EUNSUPPORTED),
    (dict(scheme=8), nat.CGL_EINVAL),
    (dict(bc=[2, 2], precision=nat.CGL_BF16X3), nat.CGL_EUNSUPPORTED),
    (dict(n=[24, 300], precision=nat.CGL_BF16X3), nat.CGL_EUNSUPPORTED),
])
def test_invalid_arguments_are_rejected_before_any_cuda_call(lib, kw, status):
    st, h = create(**kw)
    assert st == status
    assert not h.value
    assert lib.cgl_last_error() != b""


def test_null_arguments(lib):
    assert lib.cgl_plan_create(None, 2, None, None, None, None, 1, 0, 1, -1, 1, 0, 0, 0.1, 0, 0, None) \
        == nat.CGL_EINVAL
    assert lib.cgl_step(None, None, 1, None) == nat.CGL_EINVAL
    assert lib.cgl_step_host(None, None, 1, None) == nat.CGL_EINVAL
    assert lib.cgl_plan_destroy(None) == nat.CGL_OK
    assert lib.cgl_rel_error(None, None, 4, 0, None, None) == nat.CGL_EINVAL
    assert lib.cgl_plan_info(None, None, None, None) == nat.CGL_EINVAL
    assert lib.cgl_measure_fma_peak(nat.CGL_F64, 16, None, None) == nat.CGL_EINVAL
    out = ctypes.c_double()
    assert lib.cgl_measure_fma_peak(nat.CGL_F64, 0, ctypes.byref(out), None) == nat.CGL_EINVAL
    assert lib.cgl_measure_fma_peak(nat.CGL_BF16X3, 16, ctypes.byref(out), None) == nat.CGL_EINVAL


def test_batch_validation_before_any_cuda_call(lib):
    import ctypes
    probs = [nat.to_cgl_problem(type("P", (), dict(d=2, n=(8, 8), bc=(2, 2), lo=(0, 0), hi=(1, 1), a1=1.0, b1=0.0,
                                                   a2=1.0, a3=-1.0, b3=1.0, a4=0.0, b4=0.0))())]
    arr = (nat.cgl_problem * 1)(*probs)
    h = ctypes.c_void_p()
    assert lib.cgl_batch_create(ctypes.byref(h), 1, arr, 0.01, nat.CGL_LAWSON4, nat.CGL_F32, None) \
        == nat.CGL_EUNSUPPORTED  # periodic
    assert lib.cgl_batch_create(ctypes.byref(h), 0, arr, 0.01, nat.CGL_LAWSON4, nat.CGL_F32, None) == nat.CGL_EINVAL
    assert lib.cgl_batch_create(ctypes.byref(h), 1, arr, 0.01, nat.CGL_RK4, nat.CGL_F32, None) \
        == nat.CGL_EUNSUPPORTED
    assert lib.cgl_batch_create(ctypes.byref(h), 1, arr, 0.01, nat.CGL_LAWSON4, 7, None) == nat.CGL_EINVAL
    assert lib.cgl_batch_destroy(None) == nat.CGL_OK
    assert lib.cgl_autotune_mode_tile(1, 1, 0, 1, None, None) == nat.CGL_EINVAL


def test_fault_injection_hooks_validate_their_arguments(lib):
    assert lib.cgl_batch_inject_wait_failure(None, 1) == nat.CGL_EINVAL
    assert lib.cgl_inject_alloc_failure(-2) == nat.CGL_EINVAL
    # arming and disarming the allocation failure touches no device
    assert lib.cgl_inject_alloc_failure(3) == nat.CGL_OK
    assert lib.cgl_inject_alloc_failure(-1) == nat.CGL_OK


def coupled_create(**kw):
    base = dict(d=2, n=[70, 35], lo=[0.0, 0.0], hi=[70.0, 35.0], a0=-0.4, a1=0.125, b1=0.5, a2=-0.9, a3=1.0,
                b3=0.8, a4=-0.1, b4=-0.6, a5=0.5, tau=0.01, scheme=nat.CGL_SPLIT4, precision=nat.CGL_F64)
    base.update(kw)
    lib = nat.load()
    h = ctypes.c_void_p()
    d = base["d"]
    st = lib.cgl_plan_create_coupled(ctypes.byref(h), d, (ctypes.c_int64 * max(d, 1))(*base["n"]),
                                     (ctypes.c_double * max(d, 1))(*base["lo"]),
                                     (ctypes.c_double * max(d, 1))(*base["hi"]), base["a0"], base["a1"], base["b1"],
                                     base["a2"], base["a3"], base["b3"], base["a4"], base["b4"], base["a5"],
                                     base["tau"], base["scheme"], base["precision"], None)
    return st, h


@pytest.mark.parametrize("kw,status", [
    (dict(a0=float("nan")), nat.CGL_EINVAL),
    (dict(a5=float("inf")), nat.CGL_EINVAL),
    (dict(d=4, n=[8] * 4, lo=[0.0] * 4, hi=[1.0] * 4), nat.CGL_EINVAL),
    (dict(scheme=nat.CGL_SPLIT4_3T), nat.CGL_EUNSUPPORTED),
    (dict(scheme=nat.CGL_STRANG3T), nat.CGL_EUNSUPPORTED),
    (dict(precision=nat.CGL_BF16X3), nat.CGL_EUNSUPPORTED),
    (dict(n=[70, 22]), nat.CGL_EUNSUPPORTED),
    (dict(a1=0.0), nat.CGL_EINVAL),
])
def test_coupled_plan_validation_before_any_cuda_call(lib, kw, status):
    st, h = coupled_create(**kw)
    assert st == status
    assert not h.value
