"""B300-native restarted reflected-Halpern PDHG for LP (cuPDLPx, arXiv 2507.14051).

Thin ctypes binding over the C ABI declared in ``include/lp.h`` (``libpdhg.so``, built
in-tree by ``paper_2507_14051_b300.build``).  The functions here only marshal arguments:
every step of the solve runs in the library's CUDA kernels.  There is no CPU fallback;
if the library cannot be loaded, the first call raises.

Low level (same names and arguments as the C ABI):
    lp_default_params, lp_create, lp_set_params, lp_solve, lp_get, lp_get_info,
    lp_get_trace, lp_destroy, lp_last_error, lp_time_kernels, lp_debug_spmv, lp_debug_layout
High level:
    Solver(lp_or_arrays, **params) -> .solve(tol, max_iter, stream) -> .result()
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpdhg.so")

LP_OK = 0
LP_ERR_INVALID_ARG = -1
LP_ERR_INVALID_INPUT = -2
LP_ERR_CUDA = -3
LP_ERR_OUT_OF_MEMORY = -4
LP_ERR_NOT_SOLVED = -5
LP_ERR_TOO_LARGE = -6
LP_SOLVE_OPTIMAL, LP_SOLVE_ITER_LIMIT, LP_SOLVE_NUMERICAL, LP_SOLVE_INFEASIBLE = 1, 2, 3, 4
LP_SOLVE_STALLED, LP_SOLVE_INTERNAL_ERROR = 5, 6
LP_HOST, LP_DEVICE = 0, 1

EXPORTED = ("lp_default_params", "lp_create", "lp_set_params", "lp_solve", "lp_get",
            "lp_get_info", "lp_get_trace", "lp_destroy", "lp_last_error", "lp_time_kernels",
            "lp_debug_spmv", "lp_debug_layout", "lp_power_norm_noalloc")


class lp_params(C.Structure):
    """Mirror of ``lp_params`` in include/lp.h (field order and types must match)."""
    _fields_ = [
        ("gamma", C.c_double),
        ("beta_sufficient", C.c_double),
        ("beta_necessary", C.c_double),
        ("beta_artificial", C.c_double),
        ("k_p", C.c_double),
        ("k_i", C.c_double),
        ("k_d", C.c_double),
        ("eta", C.c_double),
        ("omega0", C.c_double),
        ("check_every", C.c_int64),
        ("restart_enabled", C.c_int32),
        ("pid_enabled", C.c_int32),
        ("power_tol", C.c_double),
        ("power_max_iter", C.c_int64),
        ("power_seed", C.c_uint64),
        ("ruiz_iters", C.c_int32),
        ("pc_enabled", C.c_int32),
        ("pc_alpha", C.c_double),
        ("trace_cap", C.c_int64),
        ("unroll", C.c_int32),
        ("lane_target", C.c_int32),
        ("persistent", C.c_int32),
        ("precision", C.c_int32),
        ("switch_tol", C.c_double),
        ("fp32_patience", C.c_int32),
    ]


class LPError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where} failed with status {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def load(path: str | None = None) -> C.CDLL:
    """Loads libpdhg.so (building it first if it is missing or stale and nvcc exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if path is None:
            from . import build as _build
            try:
                _build.build()
            except (OSError, FileNotFoundError) as e:  # no nvcc: only an existing library will do
                if not os.path.exists(p):
                    raise RuntimeError(f"CUDA library {p} is missing and cannot be built: {e}")
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library {p} is missing; run paper_2507_14051_b300.build")
        L = C.CDLL(p)
        vp, dp, i32p, i64p = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_int64)
        L.lp_default_params.argtypes = [C.POINTER(lp_params)]
        L.lp_create.argtypes = [C.c_int32, C.c_int32, C.c_int64, vp, vp, vp, vp, vp, vp, vp, vp,
                                C.c_int32, C.POINTER(lp_params), C.POINTER(C.c_void_p)]
        L.lp_set_params.argtypes = [vp, C.POINTER(lp_params)]
        L.lp_solve.argtypes = [vp, C.c_double, C.c_int64, vp]
        L.lp_get.argtypes = [vp, vp, vp, i32p, dp, i64p]
        L.lp_get_info.argtypes = [vp, dp]
        L.lp_get_trace.argtypes = [vp, dp, C.c_int64, i64p]
        L.lp_destroy.argtypes = [vp]
        L.lp_destroy.restype = None
        L.lp_last_error.argtypes = []
        L.lp_last_error.restype = C.c_char_p
        L.lp_time_kernels.argtypes = [vp, C.c_int64, vp, dp]
        L.lp_debug_spmv.argtypes = [vp, C.c_int32, vp, vp]
        L.lp_debug_layout.argtypes = [vp, i32p, i32p, dp, dp]
        L.lp_power_norm_noalloc.argtypes = [C.c_int32, C.c_int32, C.c_int64, vp, vp, vp, C.c_double,
                                            C.c_int64, C.c_uint64, vp, dp, i64p]
        for name in EXPORTED:
            if name not in ("lp_destroy", "lp_last_error"):
                getattr(L, name).restype = C.c_int32
        _lib = L
        return L


def lp_last_error() -> str:
    return load().lp_last_error().decode()


def _check(code: int, where: str) -> None:
    if code != LP_OK:
        raise LPError(code, where, lp_last_error())


def lp_default_params(**overrides) -> lp_params:
    p = lp_params()
    _check(load().lp_default_params(C.byref(p)), "lp_default_params")
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _ptr(a) -> int | None:
    """Address of a contiguous numpy array or torch tensor (None for None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()  # torch.Tensor


def lp_create(m, n, nnz, row_ptr, col_idx, val, c, l_c, u_c, l_v, u_v, where=LP_HOST,
              params: lp_params | None = None) -> int:
    """Returns an opaque handle (int).  Arrays: numpy (LP_HOST) or torch CUDA tensors
    (LP_DEVICE), contiguous, dtypes int64 / int32 / float64 as in include/lp.h."""
    h = C.c_void_p()
    _check(load().lp_create(m, n, nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(val), _ptr(c), _ptr(l_c),
                            _ptr(u_c), _ptr(l_v), _ptr(u_v), where,
                            C.byref(params) if params is not None else None, C.byref(h)),
           "lp_create")
    return h.value


def lp_set_params(h, params: lp_params) -> None:
    _check(load().lp_set_params(h, C.byref(params)), "lp_set_params")


def lp_solve(h, tol: float, max_iter: int, stream: int | None = None) -> None:
    """stream: a cudaStream_t as an int (e.g. torch.cuda.current_stream().cuda_stream)."""
    _check(load().lp_solve(h, tol, int(max_iter), stream), "lp_solve")


def lp_get(h, x=None, y=None):
    """Writes xhat/yhat into x/y (numpy float64 or torch CUDA float64, or None) and returns
    (solve_status, kkt[4], iters)."""
    st = C.c_int32(0)
    kkt = np.zeros(4)
    it = C.c_int64(0)
    _check(load().lp_get(h, _ptr(x), _ptr(y), C.byref(st), kkt.ctypes.data_as(C.POINTER(C.c_double)),
                         C.byref(it)), "lp_get")
    return st.value, kkt, it.value


def lp_get_info(h) -> np.ndarray:
    out = np.zeros(9)
    _check(load().lp_get_info(h, out.ctypes.data_as(C.POINTER(C.c_double))), "lp_get_info")
    return out


def lp_get_trace(h, cap: int) -> np.ndarray:
    out = np.zeros((max(cap, 1), 4))
    rows = C.c_int64(0)
    _check(load().lp_get_trace(h, out.ctypes.data_as(C.POINTER(C.c_double)), cap, C.byref(rows)),
           "lp_get_trace")
    return out[: rows.value]


def lp_destroy(h) -> None:
    if h:
        load().lp_destroy(h)


def lp_time_kernels(h, iters: int, stream: int | None = None) -> np.ndarray:
    """[ms per launch of the row (or loop) kernel, ms per launch of the column kernel (0 for
    the loop kernel), iterations per launch, launches timed]."""
    out = np.zeros(4)
    _check(load().lp_time_kernels(h, int(iters), stream, out.ctypes.data_as(C.POINTER(C.c_double))),
           "lp_time_kernels")
    return out


def lp_debug_spmv(h, which: int, x_dev, y_dev) -> None:
    _check(load().lp_debug_spmv(h, which, _ptr(x_dev), _ptr(y_dev)), "lp_debug_spmv")


def lp_debug_layout(h, m: int, n: int):
    rp = np.zeros(m, np.int32)
    cp = np.zeros(n, np.int32)
    dr = np.zeros(m)
    dc = np.zeros(n)
    _check(load().lp_debug_layout(h, rp.ctypes.data_as(C.POINTER(C.c_int32)),
                                  cp.ctypes.data_as(C.POINTER(C.c_int32)),
                                  dr.ctypes.data_as(C.POINTER(C.c_double)),
                                  dc.ctypes.data_as(C.POINTER(C.c_double))), "lp_debug_layout")
    return rp, cp, dr, dc


def lp_power_norm_noalloc(m, n, nnz, row_ptr, col_idx, val, tol=1e-7, max_iter=10000, seed=0,
                          stream: int | None = None):
    """||A||_2 estimate for a device CSR (torch CUDA tensors) without device allocation;
    returns (norm, steps).  See include/lp.h for the limits and the shared scratch."""
    out = C.c_double(0.0)
    it = C.c_int64(0)
    _check(load().lp_power_norm_noalloc(m, n, nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(val), tol,
                                        int(max_iter), seed, stream, C.byref(out), C.byref(it)),
           "lp_power_norm_noalloc")
    return out.value, it.value


class Solver:
    """Owns one handle.  ``lp`` is any object with m, n, row_ptr, col_idx, val, c, l_c, u_c,
    l_v, u_v (numpy, host)."""

    def __init__(self, lp, **params):
        self.m, self.n = int(lp.m), int(lp.n)
        arrs = [np.ascontiguousarray(lp.row_ptr, dtype=np.int64),
                np.ascontiguousarray(lp.col_idx, dtype=np.int32),
                np.ascontiguousarray(lp.val, dtype=np.float64)]
        arrs += [np.ascontiguousarray(getattr(lp, k), dtype=np.float64)
                 for k in ("c", "l_c", "u_c", "l_v", "u_v")]
        self.params = lp_default_params(**params)
        self.h = lp_create(self.m, self.n, int(arrs[0][-1]), *arrs, where=LP_HOST, params=self.params)

    def set_params(self, **params):
        for k, v in params.items():
            if not hasattr(self.params, k):
                raise KeyError(k)
            setattr(self.params, k, v)
        lp_set_params(self.h, self.params)

    def solve(self, tol=1e-8, max_iter=100000, stream=None):
        lp_solve(self.h, tol, max_iter, stream)
        return self

    def result(self):
        x, y = np.zeros(self.n), np.zeros(self.m)
        st, kkt, it = lp_get(self.h, x, y)
        info = lp_get_info(self.h)
        return dict(x=x, y=y, status=st, kkt=kkt, iters=it, eta=info[0], omega=info[1],
                    restarts=int(info[2]), norm_A=info[3], power_iters=int(info[4]),
                    pobj=info[5], dobj=info[6], persistent=bool(info[7]), iters_fp32=int(info[8]))

    def trace(self):
        return lp_get_trace(self.h, int(self.params.trace_cap))

    def close(self):
        if self.h:
            lp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
