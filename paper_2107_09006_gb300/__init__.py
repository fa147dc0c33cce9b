"""Python binding of libls_schwarz.so: two-level Schwarz PCG for sparse least squares.

The functions below carry the C ABI's names (include/ls_schwarz.h) and only marshal
arguments: torch tensors and numpy arrays become raw pointers, status codes become
exceptions.  Every computation runs in the CUDA library; importing this package
fails loudly if the library is missing or cannot be loaded.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LS_SCHWARZ_BOUNDS=1 loads the bounds-checked build (_build.build(debug_bounds=True)):
# its kernels check their indices and report an out-of-range one as LS_ERR_INVALID
_LIB_PATH = os.path.join(_HERE, "libls_schwarz_dbg.so" if os.environ.get("LS_SCHWARZ_BOUNDS") == "1"
                         else "libls_schwarz.so")

LS_OK, LS_ERR_INVALID, LS_ERR_OOM, LS_ERR_CUDA, LS_ERR_FACTOR, LS_ERR_EIGEN, LS_ERR_NOT_CONVERGED, \
    LS_ERR_NONFINITE, LS_ERR_DEVICE_TIMEOUT, LS_ERR_UNSUPPORTED = range(10)
LS_PREC_F64, LS_PREC_F32, LS_PREC_BF16 = 0, 1, 2
LS_Q_SIZES, LS_Q_OMEGA, LS_Q_XI, LS_Q_EIGVALS, LS_Q_ZBAR, LS_Q_EIGSTEPS, LS_Q_STORAGE, LS_Q_BATCH, LS_Q_NORMAL = range(9)
_PREC = {"f64": LS_PREC_F64, "f32": LS_PREC_F32, "bf16": LS_PREC_BF16}


class ls_options(ctypes.Structure):
    _fields_ = [("nev_max", ctypes.c_int), ("delta_rel", ctypes.c_double),
                ("s_rel", ctypes.c_double), ("factor_prec", ctypes.c_int), ("maxit", ctypes.c_int),
                ("coarse", ctypes.c_int), ("fixed_iters", ctypes.c_int), ("eig_maxit", ctypes.c_int),
                ("eig_tol", ctypes.c_double), ("use_graph", ctypes.c_int), ("time_kernels", ctypes.c_int),
                ("equilibrate", ctypes.c_int), ("variant", ctypes.c_int), ("solver", ctypes.c_int),
                ("restart", ctypes.c_int), ("spmv", ctypes.c_int), ("test_stall", ctypes.c_int),
                ("block_kernel", ctypes.c_int), ("normal_product", ctypes.c_int),
                ("normal_kernel", ctypes.c_int), ("local_config", ctypes.c_int)]


class ls_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("restarts", ctypes.c_int), ("relres_recursive", ctypes.c_double),
                ("relres_true", ctypes.c_double), ("kappa_lanczos", ctypes.c_double), ("n0", ctypes.c_int),
                ("kmin", ctypes.c_int), ("kmax", ctypes.c_int), ("tau_used", ctypes.c_double),
                ("delta", ctypes.c_double), ("t_setup", ctypes.c_double), ("t_eig", ctypes.c_double),
                ("t_solve", ctypes.c_double), ("bad_subdomain", ctypes.c_int), ("eig_steps_max", ctypes.c_int),
                ("ms_local", ctypes.c_double), ("ms_spmv", ctypes.c_double), ("ms_coarse", ctypes.c_double),
                ("local_launches", ctypes.c_int), ("launches", ctypes.c_int), ("ms_iter", ctypes.c_double),
                ("lanes_csr", ctypes.c_int), ("lanes_csc", ctypes.c_int), ("local_kernel", ctypes.c_int),
                ("normal_product", ctypes.c_int), ("local_config", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class LSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"ls status {status}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is missing: run __graft_entry__.build() (nvcc, sm_103a) first")
    lib = ctypes.CDLL(_LIB_PATH)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    sig = {
        "ls_default_options": (None, [ctypes.POINTER(ls_options)]),
        "ls_setup": (ctypes.c_int, [i64, i64, vp, vp, vp, i32, vp, ctypes.c_int, dbl, ctypes.POINTER(ls_options), vp,
                                    ctypes.POINTER(vp)]),
        "ls_setup_batched": (ctypes.c_int, [i32, vp, vp, vp, vp, vp, i32, vp, ctypes.c_int, dbl,
                                            ctypes.POINTER(ls_options), vp, ctypes.POINTER(vp)]),
        "ls_solve": (ctypes.c_int, [vp, vp, ctypes.c_int, dbl, vp, ctypes.POINTER(ls_info), vp]),
        "ls_backward": (ctypes.c_int, [vp, vp, vp, vp, ctypes.c_int, dbl, vp, vp, ctypes.POINTER(ls_info), vp]),
        "ls_free": (None, [vp]),
        "ls_last_error": (ctypes.c_char_p, []),
        "ls_handle_info": (ctypes.c_int, [vp, ctypes.POINTER(ls_info)]),
        "ls_apply_preconditioner": (ctypes.c_int, [vp, vp, vp, ctypes.c_int]),
        "ls_apply_normal": (ctypes.c_int, [vp, vp, vp]),
        "ls_query": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp, i64]),
        "ls_build_index_sets": (ctypes.c_int, [i64, i64, vp, vp, i32, vp, vp, vp, vp, vp, vp, vp, vp]),
        "ls_update_values": (ctypes.c_int, [vp, vp]),
        "ls_normal_product_noalloc": (ctypes.c_int, [i64, i64, vp, vp, vp, vp, vp, vp, i64, vp, vp, vp]),
        "ls_noalloc_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()
LIBRARY_PATH = _LIB_PATH
EXPORTED = ("ls_default_options", "ls_setup", "ls_setup_batched", "ls_solve", "ls_backward", "ls_free", "ls_last_error",
            "ls_handle_info", "ls_apply_preconditioner", "ls_apply_normal", "ls_query", "ls_build_index_sets",
            "ls_normal_product_noalloc", "ls_noalloc_last_error", "ls_update_values")


def _ptr(a) -> int | None:
    """Raw address of a contiguous torch tensor or numpy array (None stays NULL)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy arrays passed to the library must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors passed to the library must be contiguous")
        return a.data_ptr()
    raise TypeError(f"cannot pass {type(a)} to the library")


def _check(status: int):
    if status != LS_OK:
        raise LSError(status, _lib.ls_last_error().decode())


def ls_default_options(**kw) -> ls_options:
    o = ls_options()
    _lib.ls_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if k == "factor_prec" and isinstance(v, str):
            v = _PREC[v]
        setattr(o, k, v)
    return o


def ls_setup(m, n, row_ptr, col, val, nparts, part, overlap=1, tau=0.0, opt=None, stream=None):
    """Build the two-level preconditioner (threshold tau; tau <= 0: automatic); returns
    the opaque handle (an int)."""
    h = ctypes.c_void_p()
    o = opt if opt is not None else ls_default_options()
    _check(_lib.ls_setup(int(m), int(n), _ptr(row_ptr), _ptr(col), _ptr(val), int(nparts), _ptr(part),
                         int(overlap), float(tau), ctypes.byref(o), stream, ctypes.byref(h)))
    return h.value


def ls_setup_batched(m_off, n_off, row_ptr, col, val, nparts, part, overlap=1, tau=0.0, opt=None, stream=None):
    """Batched setup of independent problems given as one block-diagonal CSR matrix;
    m_off, n_off: host int64 offsets of the problems' rows and columns."""
    mo = np.ascontiguousarray(m_off, dtype=np.int64)
    no = np.ascontiguousarray(n_off, dtype=np.int64)
    h = ctypes.c_void_p()
    o = opt if opt is not None else ls_default_options()
    _check(_lib.ls_setup_batched(int(len(mo) - 1), _ptr(mo), _ptr(no), _ptr(row_ptr), _ptr(col), _ptr(val),
                                 int(nparts), _ptr(part), int(overlap), float(tau), ctypes.byref(o), stream,
                                 ctypes.byref(h)))
    return h.value


def ls_solve(h, b, nrhs, rtol, x, raise_on_fail=True, stream=None) -> dict:
    """``stream``: the caller's raw cudaStream_t to order the call against (None: the
    legacy default stream)."""
    info = ls_info()
    st = _lib.ls_solve(h, _ptr(b), int(nrhs), float(rtol), _ptr(x), ctypes.byref(info), stream)
    if raise_on_fail:
        _check(st)
    d = info.as_dict()
    d["status"] = st
    return d


def ls_backward(h, b, x, grad_x, nrhs, rtol, grad_b=None, grad_vals=None, stream=None) -> dict:
    info = ls_info()
    _check(_lib.ls_backward(h, _ptr(b), _ptr(x), _ptr(grad_x), int(nrhs), float(rtol), _ptr(grad_b),
                            _ptr(grad_vals), ctypes.byref(info), stream))
    return info.as_dict()


def ls_update_values(h, val):
    """New values of A (same pattern, caller's CSR order) for the operator; the
    preconditioner is kept."""
    _check(_lib.ls_update_values(h, _ptr(val)))


def ls_free(h):
    _lib.ls_free(h)


def ls_last_error() -> str:
    return _lib.ls_last_error().decode()


def ls_handle_info(h) -> dict:
    info = ls_info()
    _check(_lib.ls_handle_info(h, ctypes.byref(info)))
    return info.as_dict()


def ls_apply_preconditioner(h, r, z, which=0):
    _check(_lib.ls_apply_preconditioner(h, _ptr(r), _ptr(z), int(which)))


def ls_apply_normal(h, p, w):
    _check(_lib.ls_apply_normal(h, _ptr(p), _ptr(w)))


def ls_query(h, kind, i, out):
    _check(_lib.ls_query(h, int(kind), int(i), _ptr(out), int(out.size if isinstance(out, np.ndarray) else out.numel())))
    return out


def _check_noalloc_args(m, n, nnz, row_ptr, col, val, col_ptr, row, cval, p, w, require_cuda=True):
    """The C call checks only sizes and NULL pointers and launches its kernels on the raw
    addresses, so a host array, a wrong dtype or a short array would be read or written
    out of bounds on the device.  Every array must be a contiguous torch tensor of the
    exact dtype and length below, all on the current CUDA device; ValueError otherwise."""
    import torch
    m, n, nnz = int(m), int(n), int(nnz)
    spec = (("row_ptr", row_ptr, torch.int64, m + 1), ("col", col, torch.int32, nnz),
            ("val", val, torch.float64, nnz), ("col_ptr", col_ptr, torch.int64, n + 1),
            ("row", row, torch.int32, nnz), ("cval", cval, torch.float64, nnz),
            ("p", p, torch.float64, n), ("w", w, torch.float64, n))
    for name, t, dt, length in spec:
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name}: a torch tensor is required, got {type(t).__name__}")
        if t.dtype != dt:
            raise ValueError(f"{name}: dtype {t.dtype}, expected {dt}")
        if t.dim() != 1 or t.numel() != length:
            raise ValueError(f"{name}: shape {tuple(t.shape)}, expected ({length},)")
        if not t.is_contiguous():
            raise ValueError(f"{name}: must be contiguous")
    if require_cuda:
        cur = torch.cuda.current_device() if torch.cuda.is_available() else None
        for name, t, _, _ in spec:
            if t.device.type != "cuda" or t.device.index != cur:
                raise ValueError(f"{name}: on {t.device}, expected the current CUDA device (cuda:{cur})")


def ls_normal_product_noalloc(m, n, row_ptr, col, val, col_ptr, row, cval, nnz, p, w, stream=None):
    """w = A^T (A p) with no allocation by the library, for callers that cannot call
    cudaMalloc (device memory owned by a framework pool or a fixed budget, real-time
    loops).  Every array is a contiguous CUDA tensor on the current device: row_ptr
    int64[m+1], col int32[nnz], val float64[nnz] (CSR), col_ptr int64[n+1], row
    int32[nnz], cval float64[nnz] (CSC), p and w float64[n]; anything else raises
    ValueError before the call.  Asynchronous on ``stream`` (a raw cudaStream_t handle
    or None)."""
    _check_noalloc_args(m, n, nnz, row_ptr, col, val, col_ptr, row, cval, p, w)
    st = _lib.ls_normal_product_noalloc(int(m), int(n), _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(col_ptr),
                                        _ptr(row), _ptr(cval), int(nnz), _ptr(p), _ptr(w), stream)
    if st != LS_OK:
        raise LSError(st, _lib.ls_noalloc_last_error().decode())


def ls_build_index_sets(m, n, row_ptr, col, nparts, part):
    """Host-only index sets: returns (omega_off, omega, n_interior, xi_off, xi) as numpy arrays."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cc = np.ascontiguousarray(col, dtype=np.int32)
    pp = np.ascontiguousarray(part, dtype=np.int32)
    ot, xt = ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.ls_build_index_sets(int(m), int(n), _ptr(rp), _ptr(cc), int(nparts), _ptr(pp), ctypes.byref(ot),
                                    ctypes.byref(xt), None, None, None, None, None))
    om_off = np.zeros(nparts + 1, np.int64)
    om = np.zeros(max(ot.value, 1), np.int32)
    nI = np.zeros(nparts, np.int32)
    xi_off = np.zeros(nparts + 1, np.int64)
    xi = np.zeros(max(xt.value, 1), np.int32)
    _check(_lib.ls_build_index_sets(int(m), int(n), _ptr(rp), _ptr(cc), int(nparts), _ptr(pp), None, None,
                                    _ptr(om_off), _ptr(om), _ptr(nI), _ptr(xi_off), _ptr(xi)))
    return om_off, om[: ot.value], nI, xi_off, xi[: xt.value]


from .solver import Solver, LSSolve  # noqa: E402,F401
