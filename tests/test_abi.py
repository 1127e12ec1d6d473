"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, exports every entry
point include/lp.h declares, the Python mirror of lp_params matches the C layout, and input
validation rejects bad problems before any CUDA call."""
import ctypes as C
import glob
import math
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2507_14051_b300 as lpx
from paper_2507_14051_b300 import gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


def declared_entry_points():
    names = []
    for h in HEADERS:
        with open(h) as f:
            names += re.findall(r"LP_API\s+[\w\s\*]+?\b(lp_\w+)\s*\(", f.read())
    return names


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for required in ("lp_create", "lp_solve", "lp_get", "lp_set_params", "lp_destroy", "lp_last_error"):
        assert required in names
    assert set(names) == set(lpx.EXPORTED)


def test_library_loads_and_exports_every_declared_symbol():
    L = lpx.load()
    out = subprocess.run(["nm", "-D", "--defined-only", lpx.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(lp_\w+)$", out, flags=re.M))
    for name in declared_entry_points():
        assert name in exported, name
        assert getattr(L, name) is not None


def test_params_layout_matches_header(tmp_path):
    fields = [f for f, _ in lpx.lp_params._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "lp.h"\nint main(void){\n'
                   '  printf("%zu\\n", sizeof(lp_params));\n'
                   + "".join(f'  printf("%zu\\n", offsetof(lp_params, {f}));\n' for f in fields)
                   + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert vals[0] == C.sizeof(lpx.lp_params)
    for f, off in zip(fields, vals[1:]):
        assert getattr(lpx.lp_params, f).offset == off, f


def test_default_params_match_documentation_and_oracle():
    import oracle
    p = lpx.lp_default_params()
    assert (p.gamma, p.beta_sufficient, p.beta_necessary, p.beta_artificial) == (1.0, 0.2, 0.8, 0.36)
    assert p.eta == 0.0 and p.omega0 == 1.0 and p.check_every == 64
    assert p.unroll == 32 and p.lane_target == 0 and p.trace_cap == 0 and p.persistent == -1
    for k, v in oracle.DEFAULTS.items():
        assert getattr(p, k) == v, k


def _arrays(lp):
    return [np.ascontiguousarray(lp.row_ptr, np.int64), np.ascontiguousarray(lp.col_idx, np.int32),
            np.ascontiguousarray(lp.val, np.float64)] + \
           [np.ascontiguousarray(getattr(lp, k), np.float64) for k in ("c", "l_c", "u_c", "l_v", "u_v")]


def _create(lp, arrs=None, **kw):
    arrs = arrs or _arrays(lp)
    return lpx.lp_create(lp.m, lp.n, int(arrs[0][-1]), *arrs, **kw)


# arrays: 0 row_ptr, 1 col_idx, 2 val, 3 c, 4 l_c, 5 u_c, 6 l_v, 7 u_v
BAD_INPUTS = {
    "lower_above_upper": lambda a: a[6].__setitem__(0, a[7][0] + 1.0),
    "nan_row_bound": lambda a: a[4].__setitem__(1, math.nan),
    "plus_inf_lower": lambda a: a[6].__setitem__(2, math.inf),
    "minus_inf_upper": lambda a: a[5].__setitem__(0, -math.inf),
    "col_out_of_range": lambda a: a[1].__setitem__(0, 10 ** 6),
    "negative_col": lambda a: a[1].__setitem__(0, -1),
    "nan_value": lambda a: a[2].__setitem__(0, math.nan),
    "inf_objective": lambda a: a[3].__setitem__(0, math.inf),
    "row_lower_above_upper": lambda a: a[4].__setitem__(0, a[5][0] + 1.0),
    "row_ptr_decreasing": lambda a: a[0].__setitem__(1, a[0][2] + 1),
    "row_ptr_start": lambda a: a[0].__setitem__(0, 1),
}


@pytest.mark.parametrize("case", sorted(BAD_INPUTS))
def test_create_rejects_invalid_input(case):
    lp = gen.small_lp(0)
    arrs = _arrays(lp)
    BAD_INPUTS[case](arrs)
    with pytest.raises(lpx.LPError) as e:
        _create(lp, arrs)
    assert e.value.code == lpx.LP_ERR_INVALID_INPUT
    assert lpx.lp_last_error()


def test_create_rejects_invalid_arguments():
    lp = gen.small_lp(0)
    arrs = _arrays(lp)
    L = lpx.load()
    h = C.c_void_p()
    ptrs = [a.ctypes.data for a in arrs]
    assert L.lp_create(-1, lp.n, 0, *ptrs, 0, None, C.byref(h)) == lpx.LP_ERR_INVALID_ARG
    assert L.lp_create(lp.m, lp.n, lp.nnz, *ptrs, 7, None, C.byref(h)) == lpx.LP_ERR_INVALID_ARG
    assert L.lp_create(lp.m, lp.n, lp.nnz, *ptrs, 0, None, None) == lpx.LP_ERR_INVALID_ARG
    assert L.lp_create(lp.m, lp.n, lp.nnz, None, *ptrs[1:], 0, None, C.byref(h)) == lpx.LP_ERR_INVALID_ARG
    assert L.lp_create(lp.m, lp.n, 1 << 31, *ptrs, 0, None, C.byref(h)) == lpx.LP_ERR_TOO_LARGE
    for field, value in (("gamma", 1.5), ("check_every", 0), ("unroll", 0), ("omega0", -1.0),
                         ("lane_target", -1), ("lane_target", 65), ("pc_alpha", 3.0), ("persistent", 4)):
        p = lpx.lp_default_params(**{field: value})
        with pytest.raises(lpx.LPError) as e:
            _create(lp, arrs, params=p)
        assert e.value.code == lpx.LP_ERR_INVALID_ARG, field
    assert L.lp_solve(None, 1e-8, 10, None) == lpx.LP_ERR_INVALID_ARG
    assert L.lp_get(None, None, None, None, None, None) == lpx.LP_ERR_INVALID_ARG
    L.lp_destroy(None)


def test_valid_create_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lpx.LPError) as e:
        _create(gen.small_lp(0))
    assert e.value.code in (lpx.LP_ERR_CUDA, lpx.LP_ERR_OUT_OF_MEMORY)


# ------------------------------------------------------------------------- batch (lp_batch.h)

def _batch(seed=0, count=3):
    return gen.batch_uneven(seed, count=count, m_min=20, m_max=60, density=0.05)


@pytest.mark.parametrize("case", sorted(BAD_INPUTS))
def test_batch_create_rejects_invalid_instance(case):
    import copy
    lps = [copy.deepcopy(lp) for lp in _batch()]
    bad = lps[2]
    arrs = _arrays(bad)
    BAD_INPUTS[case](arrs)
    for k, a in zip(("row_ptr", "col_idx", "val", "c", "l_c", "u_c", "l_v", "u_v"), arrs):
        setattr(bad, k, a)
    with pytest.raises(lpx.LPError) as e:
        lpx.BatchSolver(lps)
    assert e.value.code == lpx.LP_ERR_INVALID_INPUT
    assert "instance 2" in lpx.lp_last_error()


def test_batch_create_rejects_invalid_arguments():
    lps = _batch()
    with pytest.raises(lpx.LPError) as e:
        lpx.BatchSolver(lps, eta=[0.1, -1.0, 0.1])
    assert e.value.code == lpx.LP_ERR_INVALID_ARG
    with pytest.raises(lpx.LPError) as e:
        lpx.BatchSolver(lps, gamma=2.0)
    assert e.value.code == lpx.LP_ERR_INVALID_ARG
    L = lpx.load()
    h = C.c_void_p()
    assert L.lp_batch_create(0, None, None, None, None, None, None, None, None, None, None, None, None,
                             None, None, C.byref(h)) == lpx.LP_ERR_INVALID_ARG
    with pytest.raises(lpx.LPError) as e:
        lpx.BatchSolver(lps, tiles=[(8, 1), (0, 1), (8, 1)])
    assert e.value.code == lpx.LP_ERR_INVALID_ARG
    assert L.lp_batch_solve(None, 1e-8, 10, None) == lpx.LP_ERR_INVALID_ARG
    assert L.lp_batch_get(None, 0, None, None, None, None, None) == lpx.LP_ERR_INVALID_ARG
    assert L.lp_batch_get_all(None, None, None, None, None, None) == lpx.LP_ERR_INVALID_ARG
    assert L.lp_batch_schedule(None, None) == lpx.LP_ERR_INVALID_ARG
    assert L.lp_batch_unroll(None, 10, 5, None, None, None) == lpx.LP_ERR_INVALID_ARG
    assert L.lp_batch_unroll_vjp(None, None, None, None, None, None, None, None, None) == lpx.LP_ERR_INVALID_ARG
    assert L.lp_batch_time_unroll(None, 1, None, None) == lpx.LP_ERR_INVALID_ARG
    L.lp_batch_destroy(None)


def test_batch_valid_create_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lpx.LPError) as e:
        lpx.BatchSolver(_batch())
    assert e.value.code in (lpx.LP_ERR_CUDA, lpx.LP_ERR_OUT_OF_MEMORY)


def test_tune_rejects_invalid_input_before_any_cuda_call():
    lp = gen.small_lp(0)
    bad = lp.col_idx.copy()
    bad[0] = lp.n + 5
    L = lpx.load()
    lt, tr = C.c_int32(0), C.c_int32(0)
    rp = np.ascontiguousarray(lp.row_ptr, np.int64)
    v = np.ascontiguousarray(lp.val)
    assert L.lp_tune_schedule(lp.m, lp.n, lp.nnz, rp.ctypes.data, bad.ctypes.data, v.ctypes.data, None,
                              C.byref(lt), C.byref(tr), None) == lpx.LP_ERR_INVALID_INPUT
    assert L.lp_tune_schedule(lp.m, lp.n, lp.nnz, rp.ctypes.data, bad.ctypes.data, v.ctypes.data, None,
                              None, None, None) == lpx.LP_ERR_INVALID_ARG


def test_one_call_solve_refuses_invalid_input_before_any_cuda_call():
    """lpx.solve marshals a scipy CSR matrix into lp_create, whose validation runs before the
    first CUDA call: a crossed variable bound and a NaN objective entry are refused on a host
    without a GPU."""
    import scipy.sparse as sp
    lp = gen.small_lp(1)
    A = sp.csr_matrix((lp.val, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n))
    lv, uv = lp.l_v.copy(), lp.u_v.copy()
    lv[3], uv[3] = 2.0, 1.0
    with pytest.raises(lpx.LPError) as e:
        lpx.solve(A, lp.c, lp.l_c, lp.u_c, lv, uv)
    assert e.value.code == lpx.LP_ERR_INVALID_INPUT
    c = lp.c.copy()
    c[0] = np.nan
    with pytest.raises(lpx.LPError) as e:
        lpx.solve(A, c, lp.l_c, lp.u_c, lp.l_v, lp.u_v)
    assert e.value.code == lpx.LP_ERR_INVALID_INPUT
