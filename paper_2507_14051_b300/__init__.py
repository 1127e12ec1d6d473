"""B300-native restarted reflected-Halpern PDHG for LP (cuPDLPx, arXiv 2507.14051).

Thin ctypes binding over the C ABI declared in ``include/lp.h`` (``libpdhg.so``, built
in-tree by ``paper_2507_14051_b300.build``).  The functions here only marshal arguments:
every step of the solve runs in the library's CUDA kernels.  There is no CPU fallback;
if the library cannot be loaded, the first call raises.

Low level (same names and arguments as the C ABI):
    lp_default_params, lp_create, lp_set_params, lp_solve, lp_get, lp_get_info,
    lp_get_trace, lp_destroy, lp_last_error, lp_time_kernels, lp_debug_spmv, lp_debug_layout,
    lp_power_norm_noalloc, lp_tune_schedule
High level:
    solve(A, c, l_c, u_c, l_v, u_v, tol, max_iter, stream, **params): one call, scipy CSR on the
        host or torch sparse CSR on the device
    Solver(lp, **params) -> .solve(tol, max_iter, stream) -> .result()
    BatchSolver(lps, eta=None, tiles=None, **params): many LPs in one persistent loop
        (include/lp_batch.h), plus the differentiable unrolled map (include/lp_diff.h) that
        paper_2507_14051_b300.diff.UnrolledLPBatch wraps as a torch.autograd.Function
    tune_batch(lps): per-instance tile schedules from lp_tune_schedule
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
            "lp_debug_spmv", "lp_debug_layout", "lp_power_norm_noalloc",
            "lp_batch_create", "lp_batch_solve", "lp_batch_get", "lp_batch_get_all",
            "lp_batch_time_loop", "lp_batch_schedule", "lp_batch_destroy", "lp_tune_schedule",
            "lp_batch_set_data", "lp_batch_unroll", "lp_batch_unroll_vjp", "lp_batch_get_trace",
            "lp_batch_time_unroll")


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
        ("rescale", C.c_int32),
        ("tile_rows", C.c_int32),
        ("batch_local_nnz", C.c_int64),
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
        pp = C.POINTER(C.c_void_p)
        L.lp_batch_create.argtypes = [C.c_int32, vp, vp, vp, pp, pp, pp, pp, pp, pp, pp, pp, vp, vp,
                                      C.POINTER(lp_params), C.POINTER(C.c_void_p)]
        L.lp_tune_schedule.argtypes = [C.c_int32, C.c_int32, C.c_int64, vp, vp, vp, C.c_char_p, i32p, i32p, dp]
        L.lp_batch_set_data.argtypes = [vp, vp, vp, vp, vp, vp, C.c_int32]
        L.lp_batch_unroll.argtypes = [vp, C.c_int64, C.c_int64, vp, vp, vp]
        L.lp_batch_unroll_vjp.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.lp_batch_get_trace.argtypes = [vp, C.c_int32, dp, C.c_int64, i64p]
        L.lp_batch_time_unroll.argtypes = [vp, C.c_int32, vp, dp]
        L.lp_batch_solve.argtypes = [vp, C.c_double, C.c_int64, vp]
        L.lp_batch_get.argtypes = [vp, C.c_int32, vp, vp, i32p, dp, i64p]
        L.lp_batch_get_all.argtypes = [vp, vp, vp, vp, vp, vp]
        L.lp_batch_time_loop.argtypes = [vp, C.c_int64, C.c_int32, vp, dp]
        L.lp_batch_schedule.argtypes = [vp, vp]
        L.lp_batch_destroy.argtypes = [vp]
        L.lp_batch_destroy.restype = None
        for name in EXPORTED:
            if name not in ("lp_destroy", "lp_last_error", "lp_batch_destroy"):
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
    returns (norm, steps).  See include/lp.h for the limits and the shared scratch.

    The arrays must be contiguous torch tensors on the current CUDA device with dtypes int64
    (row_ptr, m + 1 entries), int32 (col_idx, nnz) and float64 (val, nnz); anything else is
    refused here (ValueError) before the library reads a byte of it."""
    if nnz > 0:
        import torch
        want = ((row_ptr, torch.int64, m + 1, "row_ptr"), (col_idx, torch.int32, nnz, "col_idx"),
                (val, torch.float64, nnz, "val"))
        for t, dt, length, name in want:
            if not isinstance(t, torch.Tensor):
                raise ValueError(f"{name} must be a torch tensor on the current CUDA device")
            if t.dtype != dt:
                raise ValueError(f"{name} must have dtype {dt}, got {t.dtype}")
        for t, dt, length, name in want:
            if not t.is_contiguous():
                raise ValueError(f"{name} must be contiguous")
            if t.numel() < length:
                raise ValueError(f"{name} has {t.numel()} entries, needs {length}")
        for t, dt, length, name in want:
            if not t.is_cuda or t.device.index != torch.cuda.current_device():
                raise ValueError(f"{name} must live on the current CUDA device")
    out = C.c_double(0.0)
    it = C.c_int64(0)
    _check(load().lp_power_norm_noalloc(m, n, nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(val), tol,
                                        int(max_iter), seed, stream, C.byref(out), C.byref(it)),
           "lp_power_norm_noalloc")
    return out.value, it.value


def solve(A, c, l_c, u_c, l_v, u_v, tol=1e-8, max_iter=1_000_000, stream=None, **params):
    """Solves one LP (Section 2.1: min c^T x, l_c <= A x <= u_c, l_v <= x <= u_v) in one call.

    A is a scipy.sparse matrix with numpy vectors (host input), or a torch sparse CSR tensor on
    a CUDA device with CUDA tensors (device input; passed by pointer).  The data are copied by
    lp_create, solved on `stream` (a cudaStream_t as an int; None: the legacy default stream)
    and the handle is destroyed.  Returns a dict with x and y in the original variables (numpy
    for host input, CUDA float64 tensors for device input), status, kkt (relative gap, primal
    and dual residuals, their maximum) and iters.  ``params`` are lp_params fields."""
    prm = lp_default_params(**params)
    if hasattr(A, "is_cuda") and A.is_cuda:
        import torch
        if A.layout != torch.sparse_csr:
            A = A.to_sparse_csr()
        m, n = int(A.shape[0]), int(A.shape[1])
        rp = A.crow_indices().to(torch.int64).contiguous()
        ci = A.col_indices().to(torch.int32).contiguous()
        val = A.values().to(torch.float64).contiguous()
        vecs = [torch.as_tensor(v, dtype=torch.float64, device=A.device).contiguous()
                for v in (c, l_c, u_c, l_v, u_v)]
        where = LP_DEVICE
        x = torch.zeros(n, dtype=torch.float64, device=A.device)
        y = torch.zeros(m, dtype=torch.float64, device=A.device)
    else:
        import scipy.sparse as sp
        A = sp.csr_matrix(A)
        A.sum_duplicates()
        m, n = int(A.shape[0]), int(A.shape[1])
        rp = np.ascontiguousarray(A.indptr, dtype=np.int64)
        ci = np.ascontiguousarray(A.indices, dtype=np.int32)
        val = np.ascontiguousarray(A.data, dtype=np.float64)
        vecs = [np.ascontiguousarray(v, dtype=np.float64) for v in (c, l_c, u_c, l_v, u_v)]
        where = LP_HOST
        x, y = np.zeros(n), np.zeros(m)
    h = lp_create(m, n, int(rp[-1]), rp, ci, val, *vecs, where=where, params=prm)
    try:
        lp_solve(h, tol, max_iter, stream)
        st, kkt, it = lp_get(h, x, y)
    finally:
        lp_destroy(h)
    return dict(x=x, y=y, status=st, kkt=kkt, iters=it)


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


class BatchSolver:
    """Owns one batch handle (include/lp_batch.h) over a list of LPs (objects as for Solver).
    ``eta``: None (power iteration per instance, or params' eta) or a sequence of per-instance
    step sizes."""

    def __init__(self, lps, eta=None, tiles=None, **params):
        self.count = len(lps)
        self.shapes = [(int(lp.m), int(lp.n)) for lp in lps]
        cols = {"row_ptr": np.int64, "col_idx": np.int32, "val": np.float64, "c": np.float64,
                "l_c": np.float64, "u_c": np.float64, "l_v": np.float64, "u_v": np.float64}
        keep = {k: [np.ascontiguousarray(getattr(lp, k), dtype=dt) for lp in lps] for k, dt in cols.items()}
        ptrs = {k: (C.c_void_p * self.count)(*[a.ctypes.data for a in v]) for k, v in keep.items()}
        m = np.array([s[0] for s in self.shapes], np.int32)
        n = np.array([s[1] for s in self.shapes], np.int32)
        nnz = np.array([int(a[-1]) for a in keep["row_ptr"]], np.int64)
        eta_arr = None if eta is None else np.ascontiguousarray(eta, dtype=np.float64)
        lt_arr = None if tiles is None else np.ascontiguousarray(np.asarray(tiles, dtype=np.int32).reshape(-1))
        self.params = lp_default_params(**params)
        h = C.c_void_p()
        _check(load().lp_batch_create(self.count, m.ctypes.data, n.ctypes.data, nnz.ctypes.data,
                                      ptrs["row_ptr"], ptrs["col_idx"], ptrs["val"], ptrs["c"],
                                      ptrs["l_c"], ptrs["u_c"], ptrs["l_v"], ptrs["u_v"],
                                      None if eta_arr is None else eta_arr.ctypes.data,
                                      None if lt_arr is None else lt_arr.ctypes.data,
                                      C.byref(self.params), C.byref(h)), "lp_batch_create")
        self.h = h.value

    def solve(self, tol=1e-8, max_iter=100000, stream=None):
        _check(load().lp_batch_solve(self.h, tol, int(max_iter), stream), "lp_batch_solve")
        return self

    def get(self, k):
        m, n = self.shapes[k]
        x, y = np.zeros(n), np.zeros(m)
        st = C.c_int32(0)
        kkt = np.zeros(4)
        it = C.c_int64(0)
        _check(load().lp_batch_get(self.h, k, x.ctypes.data, y.ctypes.data, C.byref(st),
                                   kkt.ctypes.data_as(C.POINTER(C.c_double)), C.byref(it)), "lp_batch_get")
        return dict(x=x, y=y, status=st.value, kkt=kkt, iters=it.value)

    def summary(self):
        st = np.zeros(self.count, np.int32)
        kkt = np.zeros((self.count, 4))
        it = np.zeros(self.count, np.int64)
        it32 = np.zeros(self.count, np.int64)
        eta = np.zeros(self.count)
        _check(load().lp_batch_get_all(self.h, st.ctypes.data, kkt.ctypes.data, it.ctypes.data,
                                       it32.ctypes.data, eta.ctypes.data), "lp_batch_get_all")
        return dict(status=st, kkt=kkt, iters=it, iters_fp32=it32, eta=eta)

    def schedule(self):
        """Where each instance runs: 0 grid loop, 1 cluster of 8 blocks, 2 one block, 3 the
        shared-memory cluster loop (include/lp_batch.h, lp_batch_schedule)."""
        where = np.zeros(self.count, np.int32)
        _check(load().lp_batch_schedule(self.h, where.ctypes.data), "lp_batch_schedule")
        return where

    def set_data(self, c=None, l_c=None, u_c=None, l_v=None, u_v=None):
        """Replaces objectives / bounds (concatenated over instances, original order): numpy
        arrays (host) or torch CUDA float64 tensors (device), all of one kind."""
        arrs = [a for a in (c, l_c, u_c, l_v, u_v) if a is not None]
        where = LP_HOST if all(isinstance(a, np.ndarray) for a in arrs) else LP_DEVICE
        conv = (lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)) if where == LP_HOST \
            else (lambda a: a)
        keep = [conv(a) for a in (c, l_c, u_c, l_v, u_v)]
        _check(load().lp_batch_set_data(self.h, *[_ptr(a) for a in keep], where), "lp_batch_set_data")

    def unroll(self, K, checkpoint_every, x=None, y=None, stream=None):
        """Forward of the differentiable unrolled solve; x, y: device float64 outputs or None."""
        _check(load().lp_batch_unroll(self.h, int(K), int(checkpoint_every), _ptr(x), _ptr(y), stream),
               "lp_batch_unroll")

    def unroll_vjp(self, dl_dx=None, dl_dy=None, dl_dc=None, dl_dlc=None, dl_duc=None, dl_dlv=None,
                   dl_duv=None, stream=None):
        _check(load().lp_batch_unroll_vjp(self.h, _ptr(dl_dx), _ptr(dl_dy), _ptr(dl_dc), _ptr(dl_dlc),
                                          _ptr(dl_duc), _ptr(dl_dlv), _ptr(dl_duv), stream), "lp_batch_unroll_vjp")

    def trace(self, k, cap):
        out = np.zeros((max(int(cap), 1), 4))
        rows = C.c_int64(0)
        _check(load().lp_batch_get_trace(self.h, k, out.ctypes.data_as(C.POINTER(C.c_double)), int(cap),
                                         C.byref(rows)), "lp_batch_get_trace")
        return out[: rows.value]

    def time_unroll(self, reps=3, stream=None):
        """After unroll(): mean ms per launch of the forward segment kernel without and with clamp
        codes and of the adjoint segment kernel, and the iterations per launch."""
        out = np.zeros(4)
        _check(load().lp_batch_time_unroll(self.h, int(reps), stream, out.ctypes.data_as(C.POINTER(C.c_double))),
               "lp_batch_time_unroll")
        return float(out[0]), float(out[1]), float(out[2]), int(out[3])

    def time_loop(self, iters, fp64=True, stream=None):
        """(ms per launch of the batch loop kernel, iterations per launch)."""
        out = np.zeros(2)
        _check(load().lp_batch_time_loop(self.h, int(iters), 1 if fp64 else 0, stream,
                                         out.ctypes.data_as(C.POINTER(C.c_double))), "lp_batch_time_loop")
        return float(out[0]), int(out[1])

    def close(self):
        if self.h:
            load().lp_batch_destroy(self.h)
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


TUNE_CANDIDATES = [(8, 1), (16, 1), (32, 1), (8, 8), (16, 8), (32, 8), (8, 32), (16, 32), (32, 32)]


def lp_tune_schedule(lp, cache_path: str | None = None, timings: bool = False):
    """Fastest tile schedule (lane_target, tile_rows) for lp's matrix in the batch loop, cached per
    shape class (see include/lp_batch.h).  Returns the pair, or (pair, ms per iteration of each
    of TUNE_CANDIDATES)."""
    rp = np.ascontiguousarray(lp.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(lp.col_idx, dtype=np.int32)
    v = np.ascontiguousarray(lp.val, dtype=np.float64)
    lt, tr = C.c_int32(0), C.c_int32(0)
    ms = np.zeros(len(TUNE_CANDIDATES))
    _check(load().lp_tune_schedule(int(lp.m), int(lp.n), int(rp[-1]), rp.ctypes.data, ci.ctypes.data, v.ctypes.data,
                                   None if cache_path is None else cache_path.encode(), C.byref(lt), C.byref(tr),
                                   ms.ctypes.data_as(C.POINTER(C.c_double)) if timings else None),
           "lp_tune_schedule")
    return ((lt.value, tr.value), ms) if timings else (lt.value, tr.value)


def tune_batch(lps, cache_path: str | None = None):
    """Per-instance tile schedules for a batch (for BatchSolver(tiles=...)): one tuning run per
    shape class, the library caching by class."""
    return [lp_tune_schedule(lp, cache_path) for lp in lps]
