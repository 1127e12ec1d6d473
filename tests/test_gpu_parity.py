"""GPU path against the FP64 oracle, through the C ABI (include/lp.h).

Tolerances (FP64 on both sides; the two differ only in rounding order: tree vs sequential sums
in the SpMVs and reductions, fused multiply-adds, y * (1/sigma) instead of y / sigma, and the
maintained A x / A^T y which carry the Halpern recursion's rounding for at most one restart
epoch):
  * iterates after a fixed count:  max |gpu - oracle| <= 1e-10 * max(1, max |oracle|)
    (the paper-level parity target; T is nonexpansive, so per-step rounding of ~1e-15 does not
    grow past ~iterations * 1e-15);
  * restart iterations, status and iteration count: identical;
  * residual trace r_t: relative 1e-9 plus 1e-12 * max_t r_t (r = ||z - T z||_P is a difference
    of iterates, so its absolute rounding error stays near eps * ||z|| while r shrinks);
  * relative KKT values: 1e-8 relative (they are ratios of nearly cancelling sums).
Restart decisions compare r against beta * r0 and against the previous r.  When such a margin
is inside the rounding error of r (a floating-point tie), either outcome is a correct
evaluation of the paper's rule, and after a differing decision the trajectories part.  The
harness therefore finds the oracle's first near-tie decision and compares both sides over the
iterations before it (the run is cut so that the tied decision is never taken).  A cut must not
hide the comparison: it is accepted only when it leaves at least 90 % of the requested
iterations, or when the tie comes after the run has converged to the rounding floor
(r_tie <= 1e-9 max_t r_t, where every later decision compares residuals of ~1e-16 relative
differences); the uncut runs are then still compared at the requested count, both sides within
1e-6 of each other (a decision taken differently that late moves the iterates by about r_tie).
Any other cut fails the test with its position.
"""
import numpy as np
import pytest

import oracle
import paper_2507_14051_b300 as lpx
from paper_2507_14051_b300 import gen

pytestmark = pytest.mark.gpu

SHARED = ("gamma", "beta_sufficient", "beta_necessary", "beta_artificial", "k_p", "k_i", "k_d",
          "eta", "omega0", "check_every", "restart_enabled", "pid_enabled", "power_tol",
          "power_max_iter", "power_seed", "ruiz_iters", "pc_enabled", "pc_alpha", "rescale")
RTOL_ITER = 1e-10


def gpu_solve(lp, tol, max_iter, trace=False, **params):
    if trace:
        params = dict(params, trace_cap=max_iter)
    with lpx.Solver(lp, **params) as s:
        s.solve(tol, max_iter)
        res = s.result()
        if trace:
            res["trace"] = s.trace()
    return res


def oracle_solve(lp, tol, max_iter, trace=False, **params):
    return oracle.solve(lp, tol=tol, max_iter=max_iter, trace=trace,
                        **{k: v for k, v in params.items() if k in SHARED})


def oracle_eta(lp, **params):
    return oracle_solve(lp, 0.0, 1, **params)["eta"]


def assert_iterates_close(a, b, rtol=RTOL_ITER):
    scale = max(1.0, float(np.max(np.abs(b))) if b.size else 1.0)
    err = float(np.max(np.abs(a - b))) if b.size else 0.0
    assert err <= rtol * scale, (err, scale)


def first_near_tie(trace, beta_s=0.2, beta_n=0.8, rel=1e-9, floor=1e-12):
    """First iteration whose restart decision lies within rounding of a threshold."""
    r, k = trace[:, 0], trace[:, 3]
    atol = floor * float(np.max(r)) if len(r) else 0.0
    r0 = r_prev = 0.0
    for t in range(len(r)):
        if k[t] == 0:
            r0 = r[t]
        else:
            tol = rel * r[t] + atol
            if abs(r[t] - beta_s * r0) <= tol or abs(r[t] - beta_n * r0) <= tol:
                return t
            if r[t] <= beta_n * r0 + tol and abs(r[t] - r_prev) <= tol:
                return t
        r_prev = r[t]
    return None


TIE_CONVERGED = 1e-9  # a restart near-tie is tolerated once r_t <= this * max r


def tie_is_late(trace, tie):
    """True if the near-tie decision at `tie` comes after the run converged to the rounding floor."""
    r = trace[:, 0]
    return bool(r[tie] <= TIE_CONVERGED * float(np.max(r)))


def compare_fixed(lp, iters, **params):
    """Both sides run `iters` iterations (tol = 0) with the same explicit step size, cut
    before the first near-tie restart decision if there is one; a cut that leaves less than
    90 % of the iterations is accepted only after convergence (module docstring), and then the
    full runs are also compared at 1e-6."""
    params = dict(params)
    params.setdefault("eta", oracle_eta(lp, **params))
    requested = iters
    o = oracle_solve(lp, 0.0, iters, trace=True, **params)
    tie = first_near_tie(o["trace"], params.get("beta_sufficient", 0.2), params.get("beta_necessary", 0.8))
    if tie is not None and tie < iters - 1:
        late = tie_is_late(o["trace"], tie)
        assert tie + 1 >= 0.9 * requested or late, (
            f"restart near-tie at iteration {tie} (r/max r = {o['trace'][tie, 0] / np.max(o['trace'][:, 0]):.2e}) "
            f"would cut the comparison to {tie + 1} of {requested} iterations")
        if late:
            full_g = gpu_solve(lp, 0.0, requested, **params)
            assert full_g["iters"] == o["iters"] == requested
            assert_iterates_close(full_g["x"], o["x"], rtol=1e-6)
            assert_iterates_close(full_g["y"], o["y"], rtol=1e-6)
        iters = tie + 1
        o = oracle_solve(lp, 0.0, iters, trace=True, **params)
    g = gpu_solve(lp, 0.0, iters, trace=True, **params)
    assert g["status"] == o["status"] == oracle.ITER_LIMIT
    assert g["iters"] == o["iters"] == iters
    np.testing.assert_array_equal(g["trace"][:, 2], o["trace"][:, 2])   # restart iterations
    np.testing.assert_array_equal(g["trace"][:, 3], o["trace"][:, 3])   # epoch step k
    np.testing.assert_allclose(g["trace"][:, 0], o["trace"][:, 0], rtol=1e-9,
                               atol=1e-12 * float(np.max(o["trace"][:, 0])))
    # omega comes from |xhat - x0| and |yhat - y0| at restarts, differences whose relative rounding
    # error grows like |z| / |z - z0| ~ r_max / r_t as the run converges
    r = o["trace"][:, 0]
    w_tol = 1e-13 * float(np.max(r)) / np.maximum(r, 1e-300) + 1e-12
    w_err = np.abs(g["trace"][:, 1] - o["trace"][:, 1]) / o["trace"][:, 1]
    assert np.all(w_err <= w_tol), (float(np.max(w_err / w_tol)), int(np.argmax(w_err / w_tol)))
    assert_iterates_close(g["x"], o["x"])
    assert_iterates_close(g["y"], o["y"])
    np.testing.assert_allclose(g["kkt"], o["kkt"][:4], rtol=1e-8, atol=1e-14)
    return g, o


# --------------------------------------------------------------------------- SpMV schedule

def _spmv_case(lp, scaled):
    import torch
    params = {} if scaled else dict(ruiz_iters=0, pc_enabled=0)
    with lpx.Solver(lp, **params) as s:
        rperm, cperm, dr, dc = lpx.lp_debug_layout(s.h, lp.m, lp.n)
        rng = np.random.default_rng(5)
        x = rng.standard_normal(lp.n)
        y = rng.standard_normal(lp.m)
        xd = torch.tensor(x[cperm], dtype=torch.float64, device="cuda")
        yd = torch.tensor(y[rperm], dtype=torch.float64, device="cuda")
        ax = torch.zeros(lp.m, dtype=torch.float64, device="cuda")
        aty = torch.zeros(lp.n, dtype=torch.float64, device="cuda")
        lpx.lp_debug_spmv(s.h, 0, xd, ax)
        lpx.lp_debug_spmv(s.h, 1, yd, aty)
        g_ax = np.empty(lp.m); g_ax[rperm] = ax.cpu().numpy()
        g_aty = np.empty(lp.n); g_aty[cperm] = aty.cpu().numpy()
    # stored matrix is D_r A D_c
    ref_ax = dr * oracle.spmv(lp, dc * x)
    ref_aty = dc * oracle.spmv_t(lp, dr * y)
    np.testing.assert_allclose(g_ax, ref_ax, rtol=1e-12, atol=1e-12 * max(1, np.abs(ref_ax).max()))
    np.testing.assert_allclose(g_aty, ref_aty, rtol=1e-12, atol=1e-12 * max(1, np.abs(ref_aty).max()))


@pytest.mark.parametrize("make", [lambda: gen.ragged_rows(0, 300, 2500), lambda: gen.small_lp(1),
                                  lambda: gen.miplib_like(0, 3000, 6000, 2000),
                                  lambda: gen.multicommodity(0, 300, 1500, 3)])
@pytest.mark.parametrize("scaled", [False, True])
def test_spmv_matches_oracle(cuda_device, make, scaled):
    _spmv_case(make(), scaled)


def test_layout_is_a_permutation_and_scaling_matches_oracle(cuda_device):
    lp = gen.miplib_like(1, 2000, 4000, 1000)
    with lpx.Solver(lp) as s:
        rperm, cperm, dr, dc = lpx.lp_debug_layout(s.h, lp.m, lp.n)
    assert np.array_equal(np.sort(rperm), np.arange(lp.m))
    assert np.array_equal(np.sort(cperm), np.arange(lp.n))
    _, odr, odc = oracle.scale(lp, 10, 1, 1.0)
    np.testing.assert_allclose(dr, odr, rtol=1e-13)
    np.testing.assert_allclose(dc, odc, rtol=1e-13)


@pytest.mark.parametrize("make", [lambda: gen.small_lp(0), lambda: gen.ragged_rows(1, 200, 300),
                                  lambda: gen.miplib_like(2, 2000, 4000, 1000)])
def test_power_iteration_step_size(cuda_device, make):
    """eta = 0.998 / ||A~||_2 (Section 3), ||A~|| by power iteration on the device."""
    lp = make()
    g = gpu_solve(lp, 0.0, 1)
    assert g["eta"] == pytest.approx(oracle_eta(lp), rel=1e-6)   # same stopping rule, same start
    tight = gpu_solve(lp, 0.0, 1, power_tol=1e-13, power_max_iter=200000)
    val, dr, dc = oracle.scale(lp, 10, 1, 1.0)
    scaled = gen.LP(lp.m, lp.n, lp.row_ptr, lp.col_idx, val, lp.c, lp.l_c, lp.u_c, lp.l_v, lp.u_v)
    assert tight["norm_A"] == pytest.approx(np.linalg.norm(scaled.dense(), 2), rel=1e-6)
    assert tight["eta"] * np.linalg.norm(scaled.dense(), 2) < 1.0


# --------------------------------------------------------------------------- iterates

@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("iters", [10, 100, 1000])
def test_small_lp_iterates(cuda_device, seed, iters):
    """Small LP (m=200, n=500, 2 % density), seeds 0-9: iterates after 10/100/1000 steps."""
    compare_fixed(gen.small_lp(seed), iters)


@pytest.mark.parametrize("variant", [dict(gamma=0.0), dict(gamma=0.5), dict(restart_enabled=0),
                                     dict(pid_enabled=0), dict(ruiz_iters=0, pc_enabled=0),
                                     dict(k_p=0.3, k_i=0.05, k_d=0.2), dict(check_every=1),
                                     dict(check_every=7, unroll=3), dict(lane_target=1), dict(lane_target=16),
                                     dict(persistent=0), dict(persistent=0, check_every=5, unroll=2),
                                     dict(persistent=1, unroll=5), dict(tile_rows=32), dict(tile_rows=4, lane_target=2),
                                     dict(tile_rows=32, persistent=0), dict(persistent=2), dict(persistent=2, gamma=0.5),
                                     dict(persistent=2, check_every=1, unroll=3), dict(persistent=2, tile_rows=32),
                                     dict(persistent=3, check_every=1, unroll=3), dict(persistent=3, pid_enabled=0),
                                     dict(persistent=3, restart_enabled=0, unroll=64), dict(persistent=3, gamma=0.5)])
def test_variants_iterates(cuda_device, variant):
    compare_fixed(gen.free_and_boxed_mix(3, 300, 450), 400, **variant)


@pytest.mark.parametrize("make", [lambda: gen.ragged_rows(4, 500, 3000), lambda: gen.miplib_like(3, 4000, 8000, 2000),
                                  lambda: gen.multicommodity(1, 500, 3000, 4), lambda: gen.tiny_bounded(2, 3, 4)])
def test_structured_iterates(cuda_device, make):
    compare_fixed(make(), 300)


def test_full_size_miplib_like_iterates(cuda_device):
    """The benchmark workload (m=50k, n=100k, nnz~600k, default parameters, the benchmark's
    launch configuration): 200 iterations against the oracle, element by element."""
    compare_fixed(gen.miplib_like(0), 200)


# --------------------------------------------------------------------------- to tolerance

@pytest.mark.parametrize("seed", range(10))
def test_small_lp_to_tolerance(cuda_device, seed):
    """Both sides stop at the same iteration with OPTIMAL (Section 4, eps = 1e-8); the GPU's
    point has oracle-evaluated relative KKT <= 1e-8 and the planted optimal objective."""
    lp = gen.small_lp(seed)
    eta = oracle_eta(lp)
    g = gpu_solve(lp, 1e-8, 100000, eta=eta)
    o = oracle_solve(lp, 1e-8, 100000, eta=eta, trace=True)
    assert g["status"] == o["status"] == oracle.OPTIMAL
    tie = first_near_tie(o["trace"])
    if tie is None or tie >= o["iters"] - 1:
        assert g["iters"] == o["iters"]
    else:  # only a converged-regime tie may move the stopping check, and by one period at most
        assert tie_is_late(o["trace"], tie), (tie, o["iters"])
        assert abs(g["iters"] - o["iters"]) <= 64, (g["iters"], o["iters"])
    k = oracle.kkt(lp, g["x"], g["y"])
    assert k[3] <= 1e-8
    np.testing.assert_allclose(g["kkt"], k[:4], rtol=1e-7, atol=1e-13)
    pstar = float(lp.c @ lp.x_star)
    assert abs(k[4] - pstar) <= 1e-7 * (1 + abs(pstar))


def test_numerical_status(cuda_device):
    bad = gen.free_and_boxed_mix(0, 30, 40)
    free = int(np.argmax(~np.isfinite(bad.l_v) & ~np.isfinite(bad.u_v)))
    bad.c = bad.c.copy()
    bad.c[free] = 1e308
    kw = dict(eta=0.1, ruiz_iters=0, pc_enabled=0)
    g = gpu_solve(bad, 1e-8, 100, **kw)
    o = oracle_solve(bad, 1e-8, 100, **kw)
    assert g["status"] == o["status"] == oracle.NUMERICAL
    assert g["iters"] == o["iters"] == 1


def test_single_iteration_and_degenerate_shapes(cuda_device):
    compare_fixed(gen.small_lp(0), 1)
    # no rows: the LP is a box-constrained linear function
    rng = np.random.default_rng(0)
    n = 37
    lp = gen.LP(0, n, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0), rng.standard_normal(n),
                np.zeros(0), np.zeros(0), -np.ones(n), np.ones(n))
    g = gpu_solve(lp, 1e-10, 1000)
    assert g["status"] == oracle.OPTIMAL
    np.testing.assert_allclose(g["x"], -np.sign(lp.c))
    # empty columns and rows
    compare_fixed(gen.ragged_rows(9, 64, 5000), 150)


@pytest.mark.parametrize("persistent", [1, 0, 2, 3])
def test_deterministic_and_reusable(cuda_device, persistent):
    lp = gen.miplib_like(4, 3000, 6000, 2000)
    with lpx.Solver(lp, persistent=persistent) as s:
        a = s.solve(0.0, 500).result()
        b = s.solve(0.0, 500).result()
    assert a["persistent"] == bool(persistent)
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["y"], b["y"])
    assert a["iters"] == b["iters"] == 500


def test_both_drivers_agree(cuda_device):
    """The cooperative loop kernel and the one-kernel-per-phase driver run the same device
    functions; only the grid size (hence the order of the block sums) differs."""
    lp = gen.miplib_like(5, 3000, 6000, 2000)
    eta = oracle_eta(lp)
    a = gpu_solve(lp, 0.0, 300, eta=eta, persistent=1)
    b = gpu_solve(lp, 0.0, 300, eta=eta, persistent=0)
    assert a["persistent"] and not b["persistent"]
    assert_iterates_close(a["x"], b["x"])
    assert_iterates_close(a["y"], b["y"])


@pytest.mark.parametrize("gamma", [1.0, 0.5])
def test_three_drivers_agree_on_a_small_lp(cuda_device, gamma):
    """The small LP (200 x 500) picks by itself the shared-memory cluster loop (persistent
    -1 -> 3, reported as 3 in lp_get_info) with gamma = 1, the cluster loop (2) otherwise; the
    cluster loop, the grid-wide loop kernel (1) and one kernel per phase (0) run the same
    iteration.  With gamma = 1 the loop kernels run the reflected form, the split kernels the
    plain one."""
    lp = gen.small_lp(2)
    eta = oracle_eta(lp)
    with lpx.Solver(lp, eta=eta, gamma=gamma) as s:
        auto = s.solve(0.0, 500).result()
        info = lpx.lp_get_info(s.h)
    want = 3 if gamma == 1.0 else 2
    assert info[7] == float(want)
    runs = {p: gpu_solve(lp, 0.0, 500, eta=eta, gamma=gamma, persistent=p) for p in (0, 1, 2, 3)}
    o = oracle_solve(lp, 0.0, 500, eta=eta, gamma=gamma, trace=True)
    tie = first_near_tie(o["trace"])
    rtol = RTOL_ITER if tie is None else 1e-6
    if tie is not None:
        assert tie_is_late(o["trace"], tie), tie
    for p, g in runs.items():
        assert_iterates_close(g["x"], o["x"], rtol=rtol)
        assert_iterates_close(g["y"], o["y"], rtol=rtol)
    assert np.array_equal(auto["x"], runs[want]["x"]) and np.array_equal(auto["y"], runs[want]["y"])


def test_shared_memory_loop_applies_only_where_it_fits(cuda_device):
    """persistent 3 runs the shared-memory cluster loop on an LP that fits it (every row and
    column at most 128 entries); on one with a 2,000-entry row it chooses as -1 does, with the
    same iterates."""
    small = gen.small_lp(4)
    with lpx.Solver(small, persistent=3) as s:
        s.solve(0.0, 50).result()
        assert lpx.lp_get_info(s.h)[7] == 3.0
    big = gen.miplib_like(6, 3000, 6000, 2000)
    eta = oracle_eta(big)
    with lpx.Solver(big, persistent=3, eta=eta) as s:
        a = s.solve(0.0, 200).result()
        info3 = lpx.lp_get_info(s.h)[7]
    with lpx.Solver(big, persistent=-1, eta=eta) as s:
        b = s.solve(0.0, 200).result()
        info_auto = lpx.lp_get_info(s.h)[7]
    assert info3 == info_auto and info3 != 3.0
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["y"], b["y"])


@pytest.mark.parametrize("seed", range(3))
def test_shared_memory_loop_deterministic_and_reusable(cuda_device, seed):
    """Two solves on one handle of the shared-memory cluster loop give the same bits (its sums
    have a fixed order), and a solve continued over several launches (unroll 7) matches the
    oracle like the one-launch solves do."""
    lp = gen.small_lp(seed)
    with lpx.Solver(lp, persistent=3) as s:
        a = s.solve(0.0, 700).result()
        b = s.solve(0.0, 700).result()
        assert lpx.lp_get_info(s.h)[7] == 3.0
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["y"], b["y"])
    assert a["iters"] == b["iters"] == 700
    compare_fixed(lp, 300, persistent=3, unroll=7)


@pytest.mark.parametrize("shape", [(200, 500, 0.02), (1000, 2000, 0.01), (4000, 4000, 0.001)])
def test_shared_memory_loop_both_orders(cuda_device, shape):
    """The shared-memory cluster loop runs its overlapped order (each CTA's rows and columns in
    one SpMV pass of seven warps: the 200 x 500 and 1000 x 2000 LPs) and its plain order (250
    rows per CTA: the 4000 x 4000 LP); all match the oracle element by element."""
    m, n, dens = shape
    lp = gen.small_lp(7, m, n, dens)
    with lpx.Solver(lp, persistent=3) as s:
        s.solve(0.0, 20).result()
        assert lpx.lp_get_info(s.h)[7] == 3.0
    compare_fixed(lp, 300, persistent=3, unroll=9)


def test_device_inputs_equal_host_inputs(cuda_device):
    import torch
    lp = gen.small_lp(3)
    host = gpu_solve(lp, 0.0, 300)
    d = lambda a, dt: torch.tensor(np.asarray(a), dtype=dt, device="cuda")
    arrs = [d(lp.row_ptr, torch.int64), d(lp.col_idx, torch.int32), d(lp.val, torch.float64)] + \
           [d(getattr(lp, k), torch.float64) for k in ("c", "l_c", "u_c", "l_v", "u_v")]
    h = lpx.lp_create(lp.m, lp.n, lp.nnz, *arrs, where=lpx.LP_DEVICE)
    try:
        lpx.lp_solve(h, 0.0, 300, torch.cuda.current_stream().cuda_stream)
        x = torch.zeros(lp.n, dtype=torch.float64, device="cuda")
        y = torch.zeros(lp.m, dtype=torch.float64, device="cuda")
        st, kkt, it = lpx.lp_get(h, x, y)
    finally:
        lpx.lp_destroy(h)
    assert it == 300
    assert np.array_equal(x.cpu().numpy(), host["x"]) and np.array_equal(y.cpu().numpy(), host["y"])


def test_set_params_changes_the_run(cuda_device):
    lp = gen.small_lp(4)
    eta = oracle_eta(lp)
    with lpx.Solver(lp, eta=eta) as s:
        s.solve(0.0, 200)
        a = s.result()
        s.set_params(gamma=0.5, trace_cap=200)
        s.solve(0.0, 200)
        b = s.result()
        tr = s.trace()
    o = oracle_solve(lp, 0.0, 200, trace=True, eta=eta, gamma=0.5)
    assert not np.array_equal(a["x"], b["x"])
    assert_iterates_close(b["x"], o["x"])
    np.testing.assert_array_equal(tr[:, 2], o["trace"][:, 2])


# --------------------------------------------------------------------------- rescaling

def _rescale_ratio(lp):
    """||c~|| / ||finite (l_c~, u_c~)|| of the oracle's preconditioned data."""
    val, dr, dc = oracle.scale(lp)
    b = np.concatenate([lp.l_c * dr, lp.u_c * dr])
    b = b[np.isfinite(b)]
    beta = np.linalg.norm(b) if np.any(b != 0) else 1.0
    gam = np.linalg.norm(lp.c * dc) if np.any(lp.c != 0) else 1.0
    return gam / beta


@pytest.mark.parametrize("make", [lambda: gen.small_lp(6), lambda: gen.free_and_boxed_mix(2, 60, 90),
                                  lambda: gen.miplib_like(8, 2000, 4000, 1000)])
def test_rescaling_matches_the_oracle(cuda_device, make):
    """The oracle divides objective and bounds explicitly; the GPU starts from the equivalent
    primal weight omega0 ||c~|| / ||b~||.  Same iterates, restarts and epoch steps; the GPU's
    omega is the oracle's times that ratio (the oracle iterates in the rescaled variables)."""
    lp = make()
    eta = oracle_eta(lp)
    iters = 400
    o = oracle_solve(lp, 0.0, iters, trace=True, eta=eta, rescale=1)
    tie = first_near_tie(o["trace"])
    if tie is not None and tie < iters - 1:
        iters = tie + 1
        o = oracle_solve(lp, 0.0, iters, trace=True, eta=eta, rescale=1)
    g = gpu_solve(lp, 0.0, iters, trace=True, eta=eta, rescale=1)
    np.testing.assert_array_equal(g["trace"][:, 2], o["trace"][:, 2])
    np.testing.assert_array_equal(g["trace"][:, 3], o["trace"][:, 3])
    w = _rescale_ratio(lp)
    r = o["trace"][:, 0]
    w_tol = 1e-13 * float(np.max(r)) / np.maximum(r, 1e-300) + 1e-11
    assert np.all(np.abs(g["trace"][:, 1] - o["trace"][:, 1] * w) <= w_tol * g["trace"][:, 1])
    assert_iterates_close(g["x"], o["x"], rtol=1e-9)
    assert_iterates_close(g["y"], o["y"], rtol=1e-9)


def test_rescaled_solve_to_tolerance(cuda_device):
    lp = gen.small_lp(7)
    eta = oracle_eta(lp)
    g = gpu_solve(lp, 1e-8, 100000, eta=eta, rescale=1)
    o = oracle_solve(lp, 1e-8, 100000, eta=eta, rescale=1, trace=True)
    assert g["status"] == o["status"] == oracle.OPTIMAL
    if first_near_tie(o["trace"]) is None:
        assert g["iters"] == o["iters"]
    assert oracle.kkt(lp, g["x"], g["y"])[3] <= 1e-8


def test_one_call_solve_from_scipy_and_torch_csr(cuda_device):
    """lpx.solve takes a scipy CSR matrix with numpy vectors (host) or a torch sparse CSR tensor
    with CUDA vectors (device); both equal the Solver's result bit for bit."""
    import scipy.sparse as sp
    import torch
    lp = gen.small_lp(3)
    A = sp.csr_matrix((lp.val, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n))
    vecs = [getattr(lp, k) for k in ("c", "l_c", "u_c", "l_v", "u_v")]
    with lpx.Solver(lp) as s:
        ref = s.solve(1e-8, 100000).result()
    host = lpx.solve(A, *vecs, tol=1e-8, max_iter=100000)
    At = torch.sparse_csr_tensor(torch.tensor(lp.row_ptr), torch.tensor(lp.col_idx, dtype=torch.int64),
                                 torch.tensor(lp.val), size=(lp.m, lp.n), device="cuda")
    dev = lpx.solve(At, *[torch.tensor(v, device="cuda") for v in vecs], tol=1e-8, max_iter=100000)
    assert host["status"] == dev["status"] == ref["status"] == oracle.OPTIMAL
    assert host["iters"] == dev["iters"] == ref["iters"]
    assert np.array_equal(host["x"], ref["x"]) and np.array_equal(host["y"], ref["y"])
    assert np.array_equal(dev["x"].cpu().numpy(), ref["x"]) and np.array_equal(dev["y"].cpu().numpy(), ref["y"])
