"""Mixed precision (FP32 matrix and iterates, FP64 reductions and control; then FP64 refinement)
against the FP64 oracle, through the C ABI (include/lp.h, lp_params.precision).

The FP32 phase is not the oracle's arithmetic, so it is held to an error bound rather than to
rounding-order parity:
  * fixed map (restarts and PID off, scaling off): after t iterations of the FP32 path,
    max |x32 - x64| <= t * u32 * (Lmax + 4) * max(1, max |z64|), u32 = 2^-24, Lmax the longest
    row or column.  Each iteration evaluates a dot product of at most Lmax terms (relative error
    <= Lmax u32 of the sum of absolute terms) and four more rounded operations per entry; the
    reflected Halpern step with gamma <= 1 is nonexpansive, so per-step errors add up at most
    linearly.
  * solves: the returned point is checked by the oracle's own FP64 KKT evaluation (Section 4) --
    for the refined solve at the FP64 tolerance, for the FP32-only solve at its own tolerance.
"""
import numpy as np
import pytest

import oracle
import paper_2507_14051_b300 as lpx
from paper_2507_14051_b300 import gen

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
NO_SCALING = dict(ruiz_iters=0, pc_enabled=0)


def gpu(lp, tol, max_iter, **params):
    with lpx.Solver(lp, **params) as s:
        s.solve(tol, max_iter)
        return s.result()


def max_len(lp):
    rows = np.diff(lp.row_ptr).max(initial=0)
    cols = np.bincount(lp.col_idx, minlength=lp.n).max(initial=0)
    return int(max(rows, cols))


@pytest.mark.parametrize("persistent", [-1, 1, 2])
@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("iters", [1, 64, 400])
def test_fp32_fixed_map_error_bound(cuda_device, seed, iters, persistent):
    """persistent -1 runs these small LPs on the shared-memory cluster loop, 1 on the grid-wide
    loop, 2 on the cluster loop."""
    lp = gen.small_lp(seed)
    kw = dict(restart_enabled=0, pid_enabled=0, **NO_SCALING)
    eta = oracle.solve(lp, tol=0.0, max_iter=1, **kw)["eta"]
    o = oracle.solve(lp, tol=0.0, max_iter=iters, eta=eta, **kw)
    g = gpu(lp, 0.0, iters, eta=eta, precision=2, persistent=persistent, **kw)
    assert g["iters"] == g["iters_fp32"] == iters
    bound = iters * U32 * (max_len(lp) + 4)
    for a, b in ((g["x"], o["x"]), (g["y"], o["y"])):
        scale = max(1.0, float(np.abs(b).max()))
        err = float(np.abs(a - b).max())
        assert err <= bound * scale, (err, bound * scale)
        assert err > 0.0 or iters == 1  # the phase really ran in FP32


@pytest.mark.parametrize("seed", range(6))
def test_mixed_solve_reaches_fp64_tolerance(cuda_device, seed):
    """FP32 to the switch level, FP64 refinement to 1e-8: the oracle evaluates the returned point
    and finds it optimal to 1e-8 with the planted objective."""
    lp = gen.small_lp(seed)
    g = gpu(lp, 1e-8, 200000, precision=1, switch_tol=1e-5)
    assert g["status"] == oracle.OPTIMAL
    assert 0 < g["iters_fp32"] < g["iters"]
    k = oracle.kkt(lp, g["x"], g["y"])
    assert k[3] <= 1e-8
    np.testing.assert_allclose(g["kkt"], k[:4], rtol=1e-7, atol=1e-13)
    pstar = float(lp.c @ lp.x_star)
    assert abs(k[4] - pstar) <= 1e-7 * (1 + abs(pstar))


@pytest.mark.parametrize("make", [lambda: gen.miplib_like(7, 4000, 8000, 2000),
                                  lambda: gen.free_and_boxed_mix(2, 300, 500),
                                  lambda: gen.ragged_rows(5, 400, 3000)])
def test_mixed_solve_structured(cuda_device, make):
    """Structured LPs with planted optima: the mixed solve meets 1e-6 (oracle-evaluated) and
    its objective matches the planted optimum (the MIPLIB-shaped one runs the grid-wide
    loop)."""
    lp = make()
    g = gpu(lp, 1e-6, 1_000_000, precision=1)
    assert g["status"] == oracle.OPTIMAL
    k = oracle.kkt(lp, g["x"], g["y"])
    assert k[3] <= 1e-6
    pstar = float(lp.c @ lp.x_star)
    assert abs(k[4] - pstar) <= 1e-5 * (1 + abs(pstar))


@pytest.mark.parametrize("seed", range(3))
def test_fp32_only_solve(cuda_device, seed):
    """precision 2 stops when its own (FP64-reduced) KKT test passes; the oracle's evaluation of
    the returned point agrees within FP32 rounding of the inputs (a few u32 relative to the
    norms in the KKT denominators)."""
    lp = gen.small_lp(seed)
    g = gpu(lp, 1e-4, 200000, precision=2)
    assert g["status"] == oracle.OPTIMAL
    assert g["iters_fp32"] == g["iters"]
    k = oracle.kkt(lp, g["x"], g["y"])
    assert k[3] <= 1e-4 * (1 + 1e-2)


def test_handover_after_first_check(cuda_device):
    """A switch level every point meets hands over at the first check iteration exactly."""
    lp = gen.small_lp(1)
    g = gpu(lp, 1e-8, 200000, precision=1, switch_tol=1e300, check_every=64)
    assert g["iters_fp32"] == 64
    assert g["status"] == oracle.OPTIMAL
    assert oracle.kkt(lp, g["x"], g["y"])[3] <= 1e-8


def test_mixed_iteration_limit_counts_both_phases(cuda_device):
    lp = gen.small_lp(2)
    g = gpu(lp, 1e-12, 100, precision=1, switch_tol=1e-12)
    # neither phase reaches 1e-12 in 100 iterations: FP32 stops at 100, then FP64 runs 100 more
    assert g["iters_fp32"] == 100
    assert g["iters"] == 200
    assert g["status"] == oracle.ITER_LIMIT


@pytest.mark.parametrize("precision", [1, 2])
def test_mixed_drivers_and_repeat(cuda_device, precision):
    """Same result from the cooperative loop kernel and the per-phase kernels (the per-entry FP32
    arithmetic is identical; only the order of the FP64 block sums differs), and bitwise the
    same result when a handle solves twice."""
    lp = gen.miplib_like(5, 3000, 6000, 2000)
    with lpx.Solver(lp, precision=precision, persistent=1) as s:
        a = s.solve(1e-6, 20000).result()
        a2 = s.solve(1e-6, 20000).result()
    b = gpu(lp, 1e-6, 20000, precision=precision, persistent=0)
    assert a["persistent"] and not b["persistent"]
    assert np.array_equal(a["x"], a2["x"]) and np.array_equal(a["y"], a2["y"])
    assert a["iters"] == a2["iters"]
    ref = max(1.0, float(np.abs(a["x"]).max()))
    if a["iters"] == b["iters"]:
        assert float(np.abs(a["x"] - b["x"]).max()) <= 1e-5 * ref


@pytest.mark.parametrize("make,tol", [(lambda: gen.small_lp(3), 1e-10),
                                      (lambda: gen.miplib_like(7, 4000, 8000, 2000), 1e-6)])
def test_fp32_stall_guard(cuda_device, make, tol):
    """A level below the FP32 rounding floor (1e-10): the FP32-only solve ends STALLED well before
    max_iter; a mixed solve with that switch level hands over at the same stall and its FP64 phase
    meets the tolerance."""
    lp = make()
    g2 = gpu(lp, 1e-10, 400000, precision=2)
    assert g2["status"] == lpx.LP_SOLVE_STALLED
    assert g2["iters"] < 400000 and g2["iters"] % 64 == 0
    # the returned point is the best check's; its KKT values are reported (evaluated in FP32
    # arithmetic, so the FP64 evaluation agrees to the FP32 floor only)
    k2 = oracle.kkt(lp, g2["x"], g2["y"])
    assert k2[3] <= max(10.0 * g2["kkt"][3], 1e-6)
    g1 = gpu(lp, tol, 1_000_000, precision=1, switch_tol=1e-10)
    assert g1["iters_fp32"] == g2["iters"]  # same FP32 phase, stopped by the same guard
    assert g1["status"] == oracle.OPTIMAL
    assert oracle.kkt(lp, g1["x"], g1["y"])[3] <= tol
    off = gpu(lp, 1e-10, 3000, precision=2, fp32_patience=0)
    assert off["status"] == oracle.ITER_LIMIT and off["iters"] == 3000


def test_fp32_numerical_status(cuda_device):
    """A cost that overflows FP32 ends the FP32 phase NUMERICAL; the refinement does not run."""
    bad = gen.free_and_boxed_mix(0, 30, 40)
    free = int(np.argmax(~np.isfinite(bad.l_v) & ~np.isfinite(bad.u_v)))
    bad.c = bad.c.copy()
    bad.c[free] = 1e300
    for precision in (1, 2):
        g = gpu(bad, 1e-8, 100, eta=0.1, precision=precision, **NO_SCALING)
        assert g["status"] == oracle.NUMERICAL
        assert g["iters"] == 1


def test_precision_is_fixed_at_create(cuda_device):
    lp = gen.small_lp(0)
    with lpx.Solver(lp) as s:
        s.set_params(precision=1)  # ignored: the FP32 buffers are made at create
        r = s.solve(1e-6, 100000).result()
    assert r["iters_fp32"] == 0


@pytest.mark.parametrize("persistent", [0, 1])
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_kernel_timing_in_the_first_stage_precision(cuda_device, precision, persistent):
    """lp_time_kernels times the kernels of the solve's first stage; after an FP32 timing the
    handle holds no result until the next solve, which is unchanged by the timing."""
    lp = gen.small_lp(1)
    with lpx.Solver(lp, precision=precision, persistent=persistent) as s:
        ref = s.solve(1e-6, 20000).result()
        kt = lpx.lp_time_kernels(s.h, 64)
        assert kt[0] > 0.0 and kt[3] >= 1
        assert (kt[1] == 0.0) == bool(persistent)
        if precision == 0:
            assert lpx.lp_get(s.h)[2] == 64
        else:
            with pytest.raises(lpx.LPError) as e:
                lpx.lp_get(s.h)
            assert e.value.code == lpx.LP_ERR_NOT_SOLVED
        again = s.solve(1e-6, 20000).result()
    assert again["status"] == ref["status"] and again["iters"] == ref["iters"]
    assert np.array_equal(again["x"], ref["x"]) and np.array_equal(again["y"], ref["y"])
