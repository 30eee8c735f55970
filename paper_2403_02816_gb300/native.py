"""Thin ctypes binding of libcgl (include/cgl.h): argument marshalling only.

Every step of the integrators runs in the library's CUDA kernels; there is no
Python or CPU fallback.  Loading fails loudly when ``lib/libcgl.so`` has not
been built (``__graft_entry__.build()`` or ``python -m
paper_2403_02816_gb300.build``).

Function names match the C ABI.  ``Plan`` wraps a plan handle for torch
tensors: a field is a contiguous complex tensor of shape (n_d, ..., n_1)
(so that n_1 runs fastest, the paper's vec order), complex128 for F64 plans
and complex64 for F32 plans, on the current CUDA device.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libcgl.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "cgl.h")

CGL_BC_DIRICHLET, CGL_BC_NEUMANN, CGL_BC_PERIODIC = 0, 1, 2
CGL_STRANG, CGL_SPLIT4, CGL_LAWSON4, CGL_RK4, CGL_LAWSON2, CGL_RK2 = 0, 1, 2, 3, 4, 5
CGL_STRANG3T, CGL_SPLIT4_3T = 6, 7
CGL_F64, CGL_F32, CGL_BF16X3, CGL_F64_TC = 0, 1, 2, 3
CGL_OK, CGL_EINVAL, CGL_ENOMEM, CGL_ECUDA, CGL_EUNSUPPORTED, CGL_ETIMEOUT, CGL_ENONFINITE = 0, -1, -2, -3, -4, -5, -6

SCHEMES = {"strang": CGL_STRANG, "split4": CGL_SPLIT4, "lawson4": CGL_LAWSON4, "rk4": CGL_RK4,
           "lawson2": CGL_LAWSON2, "rk2": CGL_RK2, "strang3t": CGL_STRANG3T, "split4_3t": CGL_SPLIT4_3T}
PRECISIONS = {"f64": CGL_F64, "f32": CGL_F32, "bf16x3": CGL_BF16X3, "f64tc": CGL_F64_TC}


class CglError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__("%s failed: %s (%d): %s" % (where, _strerror(status), status, msg))
        self.status = status


class cgl_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


class cgl_problem(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("n", ctypes.c_int64 * 3), ("bc", ctypes.c_int * 3),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("a1", ctypes.c_double), ("b1", ctypes.c_double), ("a2", ctypes.c_double),
                ("a3", ctypes.c_double), ("b3", ctypes.c_double), ("a4", ctypes.c_double),
                ("b4", ctypes.c_double)]


def to_cgl_problem(prob) -> cgl_problem:
    q = cgl_problem()
    q.d = prob.d
    for m in range(prob.d):
        q.n[m] = int(prob.n[m])
        q.bc[m] = int(prob.bc[m])
        q.lo[m] = float(prob.lo[m])
        q.hi[m] = float(prob.hi[m])
    for k in ("a1", "b1", "a2", "a3", "b3", "a4", "b4"):
        setattr(q, k, float(getattr(prob, k)))
    return q


_lib = None


def load() -> ctypes.CDLL:
    """Load lib/libcgl.so (once) and declare the signatures of include/cgl.h."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libcgl.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P, I, I64, D, VP, SZ = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p,
                            ctypes.c_size_t)
    sig = {
        "cgl_plan_create": (I, [ctypes.POINTER(P), I, ctypes.POINTER(I64), ctypes.POINTER(I), ctypes.POINTER(D),
                                ctypes.POINTER(D), D, D, D, D, D, D, D, D, I, I, VP]),
        "cgl_plan_create_ex": (I, [ctypes.POINTER(P), I, ctypes.POINTER(I64), ctypes.POINTER(VP), D, D, D, D, D, I,
                                   I, VP]),
        "cgl_plan_create_coupled": (I, [ctypes.POINTER(P), I, ctypes.POINTER(I64), ctypes.POINTER(D),
                                        ctypes.POINTER(D), D, D, D, D, D, D, D, D, D, D, I, I, VP]),
        "cgl_fd4_matrix": (I, [I, D, D, I, ctypes.POINTER(D)]),
        "cgl_step": (I, [P, VP, I64, VP]),
        "cgl_step_host": (I, [P, VP, I64, VP]),
        "cgl_plan_destroy": (I, [P]),
        "cgl_linear_flow": (I, [P, D, VP, VP]),
        "cgl_plan_factor": (I, [P, D, I, ctypes.POINTER(D)]),
        "cgl_plan_info": (I, [P, ctypes.POINTER(SZ), ctypes.POINTER(SZ), ctypes.POINTER(I)]),
        "cgl_last_device_status": (I, [P, VP]),
        "cgl_profile_step": (I, [P, VP, I64, VP, ctypes.POINTER(cgl_kernel_time), I, ctypes.POINTER(I)]),
        "cgl_rel_error": (I, [VP, VP, I64, I, ctypes.POINTER(D), VP]),
        "cgl_rel_error_noalloc": (I, [VP, VP, I64, I, ctypes.POINTER(D), VP]),
        "cgl_measure_fma_peak": (I, [I, I, ctypes.POINTER(D), VP]),
        "cgl_batch_create": (I, [ctypes.POINTER(P), I, ctypes.POINTER(cgl_problem), D, I, I, VP]),
        "cgl_batch_info": (I, [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(SZ),
                               ctypes.POINTER(I)]),
        "cgl_batch_step": (I, [P, VP, I64, VP]),
        "cgl_batch_last_device_status": (I, [P, VP]),
        "cgl_batch_destroy": (I, [P]),
        "cgl_batch_inject_wait_failure": (I, [P, I]),
        "cgl_inject_alloc_failure": (I, [ctypes.c_longlong]),
        "cgl_autotune_mode_tile": (I, [I, I, I, I, ctypes.POINTER(I), ctypes.POINTER(D)]),
        "cgl_corrector_create": (I, [ctypes.POINTER(P), I, I, I, I, I, ctypes.c_uint64, VP]),
        "cgl_corrector_num_params": (I, [P, ctypes.POINTER(I64)]),
        "cgl_corrector_set_weights": (I, [P, ctypes.POINTER(ctypes.c_float), I64]),
        "cgl_corrector_get_weights": (I, [P, ctypes.POINTER(ctypes.c_float), I64]),
        "cgl_corrector_forward": (I, [P, VP, VP, VP, VP, I, VP, VP]),
        "cgl_corrector_gradients": (I, [P, VP, VP, VP, VP, VP, I, ctypes.POINTER(ctypes.c_float),
                                        ctypes.POINTER(D), VP]),
        "cgl_corrector_train_step": (I, [P, VP, VP, VP, VP, VP, I, ctypes.c_float, ctypes.POINTER(D), VP]),
        "cgl_corrector_apply": (I, [P, VP, VP, VP, I, VP, VP]),
        "cgl_corrector_destroy": (I, [P]),
        "cgl_corrector_last_device_status": (I, [P, VP]),
        "cgl_conv3x3": (I, [VP, VP, VP, VP, I, I, I, I, I, I, VP, VP]),
        "cgl_corrector_set_output_scale": (I, [P, ctypes.c_float]),
        "cgl_corrector_layer_state": (I, [P, I, I, VP, I64, VP]),
        "cgl_corrector_apply_c128": (I, [P, VP, VP, VP, I, VP, VP]),
        "cgl_corrector_set_target_mode": (I, [P, I]),
        "cgl_corrector_set_scale_mode": (I, [P, I]),
        "cgl_strerror": (ctypes.c_char_p, [I]),
        "cgl_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def header_functions() -> list:
    """Names of the functions include/cgl.h declares."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cgl_[a-z0-9_]+)\s*\(", text)))


def _strerror(status: int) -> str:
    try:
        return load().cgl_strerror(status).decode()
    except Exception:
        return "status"


def check(status: int, where: str):
    if status != CGL_OK:
        msg = load().cgl_last_error().decode()
        raise CglError(status, where, msg)
    return status


def _stream_handle(stream) -> ctypes.c_void_p:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))


def cgl_plan_create(d, n, bc, lo, hi, a1, b1, a2, a3, b3, a4, b4, tau, scheme, precision, stream=None):
    lib = load()
    h = ctypes.c_void_p()
    arr = lambda t, v: (t * len(v))(*v)
    st = lib.cgl_plan_create(ctypes.byref(h), int(d), arr(ctypes.c_int64, n), arr(ctypes.c_int, bc),
                             arr(ctypes.c_double, lo), arr(ctypes.c_double, hi), a1, b1, a2, a3, b3, a4, b4,
                             tau, int(scheme), int(precision), _stream_handle(stream))
    return st, h


def cgl_plan_create_ex(mats, a3, b3, a4, b4, tau, scheme, precision, stream=None):
    """Plan with caller-supplied direction matrices (complex n_mu x n_mu numpy
    arrays); returns (status, handle)."""
    import numpy as np
    lib = load()
    h = ctypes.c_void_p()
    cols = [np.asfortranarray(np.asarray(A, dtype=np.complex128)) for A in mats]
    bufs = [np.frombuffer(c.tobytes(order="F"), dtype=np.float64).copy() for c in cols]
    ptrs = (ctypes.c_void_p * len(bufs))(*[b.ctypes.data for b in bufs])
    n = (ctypes.c_int64 * len(cols))(*[c.shape[0] for c in cols])
    st = lib.cgl_plan_create_ex(ctypes.byref(h), len(cols), n, ptrs, a3, b3, a4, b4, tau, int(scheme), int(precision),
                                _stream_handle(stream))
    return st, h


def cgl_fd4_matrix(n, lo, hi, right_bc):
    """The paper's fourth-order d^2/dx^2 matrix (n x n numpy array)."""
    import numpy as np
    out = (ctypes.c_double * (n * n))()
    check(load().cgl_fd4_matrix(int(n), float(lo), float(hi), int(right_bc), out), "cgl_fd4_matrix")
    return np.frombuffer(out, dtype=np.float64).reshape((n, n), order="F").copy()


def cgl_conv3x3(x, w_bf16, bias, y, relu, status=None, stream=None):
    """One tensor-core 3x3 circular convolution: x float32 [B][Cin][H][W],
    w_bf16 int16/uint16 bit patterns [Cout][Cin][3][3], bias float32 [Cout]
    or None, y float32 [B][Cout][H][W] (device tensors)."""
    B, cin, H, W = x.shape
    cout = w_bf16.shape[0]
    ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    check(load().cgl_conv3x3(ptr(x), ptr(w_bf16), ptr(bias), ptr(y), B, cin, cout, H, W, int(relu), ptr(status),
                             _stream_handle(stream)), "cgl_conv3x3")
    return y


def cgl_rel_error(x, y, precision, stream=None):
    """Relative L2 and inf errors of device tensor x against y (FP64 accumulation)."""
    out = (ctypes.c_double * 3)()
    check(load().cgl_rel_error(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), x.numel(),
                               int(precision), out, _stream_handle(stream)), "cgl_rel_error")
    return out[0], out[1], int(out[2])


def cgl_measure_fma_peak(precision, iters, stream=None):
    """Measured FMA throughput of the current device in TFLOP/s ("f64" or "f32")."""
    out = ctypes.c_double()
    check(load().cgl_measure_fma_peak(PRECISIONS[precision], int(iters), ctypes.byref(out), _stream_handle(stream)),
          "cgl_measure_fma_peak")
    return out.value


class Plan:
    """A libcgl plan for one problem, step size, scheme and precision."""

    nfield = 1  # fields in the state (the coupled system has two)

    def __init__(self, prob, tau: float, scheme: str, precision: str = "f64", stream=None):
        self.prob = prob
        self.scheme = scheme
        self.precision = precision
        self.prec = PRECISIONS[precision]
        st, self.handle = cgl_plan_create(prob.d, prob.n, prob.bc, prob.lo, prob.hi, prob.a1, prob.b1, prob.a2,
                                          prob.a3, prob.b3, prob.a4, prob.b4, tau, SCHEMES[scheme], self.prec,
                                          stream)
        check(st, "cgl_plan_create")

    @classmethod
    def from_matrices(cls, mats, a3, b3, a4, b4, tau: float, scheme: str, precision: str = "f64", stream=None):
        """Plan whose direction matrices A_mu are given (cgl_plan_create_ex)."""
        from . import inputs
        self = cls.__new__(cls)
        d = len(mats)
        n = tuple(int(A.shape[0]) for A in mats)
        self.prob = inputs.Problem(n, (CGL_BC_DIRICHLET,) * d, (0.0,) * d, (1.0,) * d, 1.0, 0.0, 0.0, a3, b3, a4, b4)
        self.scheme = scheme
        self.precision = precision
        self.prec = PRECISIONS[precision]
        st, self.handle = cgl_plan_create_ex(mats, a3, b3, a4, b4, tau, SCHEMES[scheme], self.prec, stream)
        check(st, "cgl_plan_create_ex")
        return self

    # torch helpers -------------------------------------------------------
    @property
    def shape(self):
        n = tuple(reversed(self.prob.n))
        return n if self.nfield == 1 else (self.nfield,) + n

    @property
    def dtype(self):
        import torch
        return torch.complex128 if self.prec in (CGL_F64, CGL_F64_TC) else torch.complex64

    def _field(self, u):
        count = self.nfield * self.prob.N
        if not u.is_cuda or not u.is_contiguous() or u.dtype != self.dtype or u.numel() != count:
            raise ValueError("field must be a contiguous %s CUDA tensor with %d elements" % (self.dtype, count))
        return ctypes.c_void_p(u.data_ptr())

    def step(self, u, nsteps: int, stream=None):
        check(load().cgl_step(self.handle, self._field(u), int(nsteps), _stream_handle(stream)), "cgl_step")
        return u

    def step_host(self, u_host, nsteps: int, stream=None):
        """u_host: a CPU tensor (pinned or pageable), advanced in place."""
        if u_host.is_cuda or not u_host.is_contiguous() or u_host.dtype != self.dtype:
            raise ValueError("u_host must be a contiguous CPU tensor of %s" % self.dtype)
        check(load().cgl_step_host(self.handle, ctypes.c_void_p(u_host.data_ptr()), int(nsteps),
                                   _stream_handle(stream)), "cgl_step_host")
        return u_host

    def linear_flow(self, u, c: float, stream=None):
        check(load().cgl_linear_flow(self.handle, float(c), self._field(u), _stream_handle(stream)),
              "cgl_linear_flow")
        return u

    def factor(self, c: float, mu: int):
        import numpy as np
        n = self.prob.n[mu]
        count = n if self.prob.periodic else n * n
        buf = (ctypes.c_double * (2 * count))()
        check(load().cgl_plan_factor(self.handle, float(c), int(mu), buf), "cgl_plan_factor")
        a = np.frombuffer(buf, dtype=np.complex128).copy()
        return a if self.prob.periodic else a.reshape((n, n), order="F")

    def info(self):
        fb, wb, nl = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_int()
        check(load().cgl_plan_info(self.handle, ctypes.byref(fb), ctypes.byref(wb), ctypes.byref(nl)),
              "cgl_plan_info")
        return {"field_bytes": fb.value, "workspace_bytes": wb.value, "launches_per_step": nl.value}

    def device_status(self, stream=None) -> int:
        return load().cgl_last_device_status(self.handle, _stream_handle(stream))

    def profile(self, u, nsteps: int, stream=None):
        recs = (cgl_kernel_time * 16)()
        cnt = ctypes.c_int()
        check(load().cgl_profile_step(self.handle, self._field(u), int(nsteps), _stream_handle(stream), recs, 16,
                                      ctypes.byref(cnt)), "cgl_profile_step")
        return [{"name": r.name.decode(), "launches": r.launches, "total_ms": r.total_ms, "flops": r.flops,
                 "bytes": r.bytes} for r in recs[:cnt.value]]

    def close(self):
        if getattr(self, "handle", None):
            load().cgl_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def inject_alloc_failure(after: int):
    """Test hook: the (after + 1)-th device allocation from now by a plan,
    batch or corrector fails with CGL_ENOMEM; -1 disarms."""
    check(load().cgl_inject_alloc_failure(int(after)), "cgl_inject_alloc_failure")


def to_device(U, dtype, device="cuda"):
    """numpy array of shape (n_1..n_d) -> contiguous torch tensor (n_d..n_1)."""
    import numpy as np
    import torch
    t = torch.from_numpy(np.ascontiguousarray(U.T))
    return t.to(dtype).to(device).contiguous()


def to_device_pair(W, dtype, device="cuda"):
    """numpy (2, n_1..n_d) (u, v) -> contiguous torch tensor (2, n_d..n_1)."""
    import torch
    return torch.stack([to_device(W[0], dtype, device), to_device(W[1], dtype, device)]).contiguous()


def from_device_pair(t):
    """torch tensor (2, n_d..n_1) -> complex128 numpy array (2, n_1..n_d)."""
    import numpy as np
    return np.stack([from_device(t[0]), from_device(t[1])])


class CoupledPlan(Plan):
    """Plan of the coupled two-field system (cgl_plan_create_coupled).  `prob`
    carries n, lo, hi and a0, a1, b1, a2, a3, b3, a4, b4, a5; the state is a
    tensor of shape (2, n_d, ..., n_1): u, then v."""

    nfield = 2

    def __init__(self, prob, tau: float, scheme: str, precision: str = "f64", stream=None):
        self.prob = prob
        self.scheme = scheme
        self.precision = precision
        self.prec = PRECISIONS[precision]
        lib = load()
        h = ctypes.c_void_p()
        d = len(prob.n)
        st = lib.cgl_plan_create_coupled(ctypes.byref(h), d, (ctypes.c_int64 * d)(*prob.n),
                                         (ctypes.c_double * d)(*prob.lo), (ctypes.c_double * d)(*prob.hi),
                                         prob.a0, prob.a1, prob.b1, prob.a2, prob.a3, prob.b3, prob.a4, prob.b4,
                                         prob.a5, float(tau), SCHEMES[scheme], self.prec, _stream_handle(stream))
        self.handle = h
        check(st, "cgl_plan_create_coupled")


def from_device(t):
    """torch tensor (n_d..n_1) -> complex128 numpy array (n_1..n_d)."""
    import torch
    return t.to(torch.complex128).cpu().numpy().T.copy()


def cgl_batch_create(probs, tau, scheme, precision, stream=None):
    arr = (cgl_problem * len(probs))(*[to_cgl_problem(p) for p in probs])
    h = ctypes.c_void_p()
    st = load().cgl_batch_create(ctypes.byref(h), len(probs), arr, float(tau), int(scheme), int(precision),
                                 _stream_handle(stream))
    return st, h


def cgl_autotune_mode_tile(n, contiguous, precision, nrhs):
    tb, ms = ctypes.c_int(), ctypes.c_double()
    check(load().cgl_autotune_mode_tile(int(n), int(contiguous), int(precision), int(nrhs), ctypes.byref(tb),
                                        ctypes.byref(ms)), "cgl_autotune_mode_tile")
    return tb.value, ms.value


class Batch:
    """Many independent finite-difference problems advanced together.  The
    field is one packed complex tensor; instance i occupies
    [offsets[i], offsets[i] + N_i) in the layout of a single plan."""

    def __init__(self, probs, tau: float, scheme: str, precision: str = "f32", stream=None):
        self.probs = list(probs)
        self.prec = PRECISIONS[precision]
        st, self.handle = cgl_batch_create(self.probs, tau, SCHEMES[scheme], self.prec, stream)
        check(st, "cgl_batch_create")
        total = ctypes.c_int64()
        offs = (ctypes.c_int64 * len(self.probs))()
        nl = ctypes.c_int()
        check(load().cgl_batch_info(self.handle, ctypes.byref(total), offs, None, ctypes.byref(nl)),
              "cgl_batch_info")
        self.total = total.value
        self.offsets = list(offs)
        self.launches_per_step = nl.value

    @property
    def dtype(self):
        import torch
        return torch.complex128 if self.prec in (CGL_F64, CGL_F64_TC) else torch.complex64

    def pack(self, fields, device="cuda"):
        """numpy arrays (n_1..n_d), one per instance -> packed device tensor."""
        import numpy as np
        import torch
        flat = np.concatenate([np.ascontiguousarray(U.T).reshape(-1) for U in fields])
        return torch.from_numpy(flat).to(self.dtype).to(device)

    def unpack(self, t):
        """packed tensor -> list of complex128 numpy arrays (n_1..n_d)."""
        import torch
        host = t.to(torch.complex128).cpu().numpy()
        out = []
        for p, off in zip(self.probs, self.offsets):
            N = int(p.N) if hasattr(p, "N") else int(__import__("numpy").prod(p.n))
            out.append(host[off:off + N].reshape(tuple(reversed(p.n))).T.copy())
        return out

    def step(self, u, nsteps: int, stream=None):
        if not u.is_cuda or not u.is_contiguous() or u.dtype != self.dtype or u.numel() != self.total:
            raise ValueError("packed field must be a contiguous %s CUDA tensor of %d values" % (self.dtype,
                                                                                               self.total))
        check(load().cgl_batch_step(self.handle, ctypes.c_void_p(u.data_ptr()), int(nsteps),
                                    _stream_handle(stream)), "cgl_batch_step")
        return u

    def device_status(self, stream=None) -> int:
        return load().cgl_batch_last_device_status(self.handle, _stream_handle(stream))

    def inject_wait_failure(self, on: bool):
        """Test hook: make every dependency wait of the step unreachable
        (FP64 / FP32 batches); the next steps report CGL_ETIMEOUT."""
        check(load().cgl_batch_inject_wait_failure(self.handle, 1 if on else 0), "cgl_batch_inject_wait_failure")

    def close(self):
        if getattr(self, "handle", None):
            load().cgl_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


class Corrector:
    """Residual CNN corrector of a coarse 2D periodic step (cgl_corrector_*).
    Fields are complex64 CUDA tensors [P, H, W]; params float32 [P, 5];
    idx int32 [batch] (or None)."""

    def __init__(self, height, width, hidden=32, layers=6, max_batch=32, seed=2403028164, stream=None):
        self.handle = ctypes.c_void_p()
        check(load().cgl_corrector_create(ctypes.byref(self.handle), int(height), int(width), int(hidden),
                                          int(layers), int(max_batch), ctypes.c_uint64(seed),
                                          _stream_handle(stream)), "cgl_corrector_create")
        n = ctypes.c_int64()
        check(load().cgl_corrector_num_params(self.handle, ctypes.byref(n)), "cgl_corrector_num_params")
        self.nparams = n.value
        self.hw = (int(height), int(width))

    def set_output_scale(self, scale):
        check(load().cgl_corrector_set_output_scale(self.handle, ctypes.c_float(scale)),
              "cgl_corrector_set_output_scale")

    def set_weights(self, flat):
        import numpy as np
        a = np.ascontiguousarray(flat, dtype=np.float32)
        check(load().cgl_corrector_set_weights(self.handle, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                               a.size), "cgl_corrector_set_weights")

    def get_weights(self):
        import numpy as np
        a = np.empty(self.nparams, dtype=np.float32)
        check(load().cgl_corrector_get_weights(self.handle, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                               a.size), "cgl_corrector_get_weights")
        return a

    def forward(self, coarse, un, params, idx=None, batch=None, stream=None):
        import torch
        batch = int(batch if batch is not None else (idx.numel() if idx is not None else coarse.shape[0]))
        out = torch.empty((batch, 2) + self.hw, dtype=torch.float32, device=coarse.device)
        check(load().cgl_corrector_forward(self.handle, _ptr(coarse), _ptr(un), _ptr(params), _ptr(idx), batch,
                                           _ptr(out), _stream_handle(stream)), "cgl_corrector_forward")
        return out

    def gradients(self, coarse, un, target, params, idx=None, batch=None, stream=None):
        import numpy as np
        batch = int(batch if batch is not None else (idx.numel() if idx is not None else coarse.shape[0]))
        g = np.empty(self.nparams, dtype=np.float32)
        loss = ctypes.c_double()
        check(load().cgl_corrector_gradients(self.handle, _ptr(coarse), _ptr(un), _ptr(target), _ptr(params),
                                             _ptr(idx), batch, g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                             ctypes.byref(loss), _stream_handle(stream)), "cgl_corrector_gradients")
        return loss.value, g

    def train_step(self, coarse, un, target, params, idx, lr, want_loss=False, stream=None):
        loss = ctypes.c_double()
        check(load().cgl_corrector_train_step(self.handle, _ptr(coarse), _ptr(un), _ptr(target), _ptr(params),
                                              _ptr(idx), int(idx.numel()), ctypes.c_float(lr),
                                              ctypes.byref(loss) if want_loss else None,
                                              _stream_handle(stream)), "cgl_corrector_train_step")
        return loss.value if want_loss else None

    def apply(self, coarse, un, params, out, stream=None):
        check(load().cgl_corrector_apply(self.handle, _ptr(coarse), _ptr(un), _ptr(params), int(coarse.shape[0]),
                                         _ptr(out), _stream_handle(stream)), "cgl_corrector_apply")
        return out

    def apply_c128(self, coarse, un, params, out, stream=None):
        """out = coarse + N(x) for complex128 fields [B, H, W]."""
        check(load().cgl_corrector_apply_c128(self.handle, _ptr(coarse), _ptr(un), _ptr(params),
                                              int(coarse.shape[0]), _ptr(out), _stream_handle(stream)),
              "cgl_corrector_apply_c128")
        return out

    def set_target_mode(self, mode):
        check(load().cgl_corrector_set_target_mode(self.handle, int(mode)), "cgl_corrector_set_target_mode")

    def set_scale_mode(self, mode):
        check(load().cgl_corrector_set_scale_mode(self.handle, int(mode)), "cgl_corrector_set_scale_mode")

    def layer_state(self, kind, layer, batch, channels, stream=None):
        """Per-layer buffer of the last call (cgl_corrector_layer_state):
        kind 0 = activation feeding layer `layer`, 1 = loss gradient w.r.t.
        layer `layer`'s output; a float32 CUDA tensor [batch, channels, H, W]."""
        import torch
        out = torch.empty((batch, channels) + self.hw, dtype=torch.float32, device="cuda")
        check(load().cgl_corrector_layer_state(self.handle, int(kind), int(layer), _ptr(out), out.numel(),
                                               _stream_handle(stream)), "cgl_corrector_layer_state")
        return out

    def device_status(self, stream=None) -> int:
        return load().cgl_corrector_last_device_status(self.handle, _stream_handle(stream))

    def close(self):
        if getattr(self, "handle", None):
            load().cgl_corrector_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
