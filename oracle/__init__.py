"""FP64 CPU oracle for restarted reflected-Halpern PDHG (arXiv 2507.14051).

TEST INFRASTRUCTURE ONLY: tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may load it; the CUDA library never does.

The arithmetic lives in ``pdhg_oracle.c`` (plain sequential C, double
precision).  This module compiles it with gcc on first use and exposes each
function through ctypes with numpy arguments.  Parameter defaults here are
the oracle's own copy of the values read from the paper (Section 3): the
reflection gamma, the three restart betas and the PID gains are not printed
there, so the chosen values are readings, listed in the design notes.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pdhg_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OPTIMAL, ITER_LIMIT, NUMERICAL = 1, 2, 3


class Params(C.Structure):
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
        ("rescale", C.c_int32),
    ]


DEFAULTS = dict(gamma=1.0, beta_sufficient=0.2, beta_necessary=0.8, beta_artificial=0.36,
                k_p=0.5, k_i=0.001, k_d=0.0, eta=0.0, omega0=1.0, check_every=64,
                restart_enabled=1, pid_enabled=1, power_tol=1e-7, power_max_iter=10000,
                power_seed=0, ruiz_iters=10, pc_enabled=1, pc_alpha=1.0, rescale=0)


def make_params(**kw) -> Params:
    d = dict(DEFAULTS)
    for k, v in kw.items():
        if k not in d:
            raise KeyError(k)
        d[k] = v
    return Params(**d)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O3, no fast-math)."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            tmp = _LIB_PATH + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                                   "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def compile_variant(source_text: str, out_path: str) -> str:
    """Compiles a modified copy of the oracle source (used by tests that plant a mistake)."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                           "-ffp-contract=off", "-o", out_path, src, "-lm"])
    return out_path


def source() -> str:
    with open(_SRC) as f:
        return f.read()


@contextlib.contextmanager
def using_library(path: str):
    """Temporarily routes every function of this module to another build of the oracle."""
    global _lib
    saved = _lib
    _lib = _configure(C.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = _configure(C.CDLL(_LIB_PATH))
    return _lib


def _configure(L):
    """Declares argument and result types of every exported oracle function."""
    dp, ip64, ip32 = C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int32)
    L.orc_spmv.argtypes = [C.c_int32, ip64, ip32, dp, dp, dp]
    L.orc_spmv_t.argtypes = [C.c_int32, C.c_int32, ip64, ip32, dp, dp, dp]
    L.orc_pdhg_step.argtypes = [C.c_int32, C.c_int32, ip64, ip32, dp, dp, dp, dp, dp, dp,
                                C.c_double, C.c_double, dp, dp, dp, dp, dp]
    L.orc_p_norm_sq.restype = C.c_double
    L.orc_p_norm_sq.argtypes = [C.c_int32, C.c_int32, ip64, ip32, dp, C.c_double, C.c_double, dp, dp]
    L.orc_kkt.argtypes = [C.c_int32, C.c_int32, ip64, ip32, dp, dp, dp, dp, dp, dp, dp, dp, dp]
    L.orc_restart_decide.restype = C.c_int32
    L.orc_restart_decide.argtypes = [C.c_int64, C.c_int64, C.c_double, C.c_double, C.c_double,
                                     C.c_double, C.c_double, C.c_double]
    L.orc_pid_update.restype = C.c_double
    L.orc_pid_update.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                 C.c_double, dp]
    L.orc_start_entry.restype = C.c_double
    L.orc_start_entry.argtypes = [C.c_uint64, C.c_uint64]
    L.orc_power_norm.restype = C.c_double
    L.orc_power_norm.argtypes = [C.c_int32, C.c_int32, ip64, ip32, dp, C.c_double, C.c_int64,
                                 C.c_uint64, ip64]
    L.orc_scale.argtypes = [C.c_int32, C.c_int32, ip64, ip32, dp, C.c_int32, C.c_int32,
                            C.c_double, dp, dp]
    L.orc_solve.restype = C.c_int32
    L.orc_solve.argtypes = [C.c_int32, C.c_int32, ip64, ip32, dp, dp, dp, dp, dp, dp,
                            C.POINTER(Params), C.c_double, C.c_int64, dp, dp, dp, ip64, dp, dp,
                            C.c_int64, dp]
    return L


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _csr(lp):
    rp = np.ascontiguousarray(lp.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(lp.col_idx, dtype=np.int32)
    v = np.ascontiguousarray(lp.val, dtype=np.float64)
    return (rp, ci, v), (rp.ctypes.data_as(C.POINTER(C.c_int64)),
                         ci.ctypes.data_as(C.POINTER(C.c_int32)),
                         v.ctypes.data_as(C.POINTER(C.c_double)))


def spmv(lp, x):
    keep, (rp, ci, v) = _csr(lp)
    xa, xp = _d(x)
    out = np.zeros(lp.m)
    lib().orc_spmv(lp.m, rp, ci, v, xp, _d(out)[1])
    return out


def spmv_t(lp, y):
    keep, (rp, ci, v) = _csr(lp)
    ya, yp = _d(y)
    out = np.zeros(lp.n)
    lib().orc_spmv_t(lp.m, lp.n, rp, ci, v, yp, _d(out)[1])
    return out


def _vecs(lp):
    arrs = [_d(a) for a in (lp.c, lp.l_c, lp.u_c, lp.l_v, lp.u_v)]
    return [a for a, _ in arrs], [p for _, p in arrs]


def pdhg_step(lp, eta, omega, x, y):
    """One PDHG step T(x, y) (Section 2.2, eq. pdhg)."""
    keep, (rp, ci, v) = _csr(lp)
    kv, (c, lc, uc, lv, uv) = _vecs(lp)
    xa, xp_ = _d(x)
    ya, yp_ = _d(y)
    xo, yo = np.zeros(lp.n), np.zeros(lp.m)
    work = np.zeros(lp.n + lp.m)
    lib().orc_pdhg_step(lp.m, lp.n, rp, ci, v, c, lc, uc, lv, uv, eta, omega, xp_, yp_,
                        _d(xo)[1], _d(yo)[1], _d(work)[1])
    return xo, yo


def p_norm_sq(lp, eta, omega, dx, dy):
    keep, (rp, ci, v) = _csr(lp)
    a, ap = _d(dx)
    b, bp = _d(dy)
    return lib().orc_p_norm_sq(lp.m, lp.n, rp, ci, v, eta, omega, ap, bp)


def kkt(lp, x, y):
    """[rel_gap, rel_pres, rel_dres, rel_kkt, pobj, dobj, pres, dres] (Section 4)."""
    keep, (rp, ci, v) = _csr(lp)
    kv, (c, lc, uc, lv, uv) = _vecs(lp)
    xa, xp_ = _d(x)
    ya, yp_ = _d(y)
    out = np.zeros(8)
    lib().orc_kkt(lp.m, lp.n, rp, ci, v, c, lc, uc, lv, uv, xp_, yp_, _d(out)[1])
    return out


def restart_decide(k, t, r, r0, r_prev, beta_s=0.2, beta_n=0.8, beta_a=0.36) -> bool:
    return bool(lib().orc_restart_decide(k, t, r, r0, r_prev, beta_s, beta_n, beta_a))


class PID:
    """Stateful wrapper over orc_pid_update (integral, previous error)."""

    def __init__(self, kp, ki, kd):
        self.kp, self.ki, self.kd = kp, ki, kd
        self.state = np.zeros(3)

    def update(self, omega, dx_norm, dy_norm):
        return lib().orc_pid_update(omega, dx_norm, dy_norm, self.kp, self.ki, self.kd,
                                    self.state.ctypes.data_as(C.POINTER(C.c_double)))


def start_entry(seed, i):
    return lib().orc_start_entry(seed, i)


def power_norm(lp, tol=1e-7, max_iter=10000, seed=0):
    keep, (rp, ci, v) = _csr(lp)
    it = C.c_int64(0)
    val = lib().orc_power_norm(lp.m, lp.n, rp, ci, v, tol, max_iter, seed, C.byref(it))
    return val, it.value


def scale(lp, ruiz_iters=10, pc_enabled=1, pc_alpha=1.0):
    """Diagonal preconditioning: returns (scaled values, d_r, d_c)."""
    keep, (rp, ci, v) = _csr(lp)
    val = np.array(lp.val, dtype=np.float64, copy=True)
    dr, dc = np.zeros(lp.m), np.zeros(lp.n)
    lib().orc_scale(lp.m, lp.n, rp, ci, _d(val)[1], ruiz_iters, pc_enabled, pc_alpha,
                    _d(dr)[1], _d(dc)[1])
    return val, dr, dc


def solve(lp, tol=1e-8, max_iter=100000, trace=False, **params):
    """Run the oracle's solve.  Returns a dict with x, y, status, kkt, iters,
    eta, omega and (if trace) an array of rows (r_t, omega_t, restart_t, k_t)."""
    keep, (rp, ci, v) = _csr(lp)
    kv, (c, lc, uc, lv, uv) = _vecs(lp)
    prm = make_params(**params)
    x, y = np.zeros(lp.n), np.zeros(lp.m)
    kk = np.zeros(8)
    iters = C.c_int64(0)
    eta = C.c_double(0)
    om = C.c_double(0)
    cap = int(max_iter) if trace else 0
    tr = np.zeros((max(cap, 1), 4))
    st = lib().orc_solve(lp.m, lp.n, rp, ci, v, c, lc, uc, lv, uv, C.byref(prm), tol, int(max_iter),
                         _d(x)[1], _d(y)[1], _d(kk)[1], C.byref(iters), C.byref(eta), C.byref(om),
                         cap, _d(tr)[1] if trace else None)
    out = dict(x=x, y=y, status=int(st), kkt=kk, iters=int(iters.value), eta=eta.value,
               omega=om.value)
    if trace:
        out["trace"] = tr[: out["iters"]]
    return out
