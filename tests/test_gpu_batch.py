"""Batched solver (include/lp_batch.h) against the FP64 oracle, instance by instance.

Each instance of a batch runs the same method as lp_solve with its own scalar state; the batch
only changes the schedule (one persistent kernel, per-task partial sums added per instance in a
fixed order).  So the single-instance tolerances apply per instance (tests/test_gpu_parity.py):
iterates after a fixed count within 1e-10 * max(1, |oracle|_inf), identical restart decisions,
status and iteration count, cut before the oracle's first near-tie restart decision.
"""
import numpy as np
import pytest

import oracle
import paper_2507_14051_b300 as lpx
from paper_2507_14051_b300 import gen

from .test_gpu_parity import SHARED, assert_iterates_close, first_near_tie, tie_is_late

pytestmark = pytest.mark.gpu


def o_solve(lp, tol, max_iter, trace=False, **params):
    return oracle.solve(lp, tol=tol, max_iter=max_iter, trace=trace,
                        **{k: v for k, v in params.items() if k in SHARED})


def o_eta(lp):
    return o_solve(lp, 0.0, 1)["eta"]


# instances with at most this many nonzeros are small (cluster or single-CTA loop): 0 = all on
# the grid loop, 4000 = some of each, 10**9 = all on the small-instance loops
LOCAL = [0, 4000, 10 ** 9]


def small_batch(seed, count=10, m_min=20, m_max=300, density=0.05):
    return gen.batch_uneven(seed, count=count, m_min=m_min, m_max=m_max, density=density)


def mixed_shapes():
    """Instances of very different shapes: no rows, empty rows and columns, one long row,
    free and one-sided bounds, a tiny bounded LP."""
    rng = np.random.default_rng(7)
    n0 = 23
    no_rows = gen.LP(0, n0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0),
                     rng.standard_normal(n0), np.zeros(0), np.zeros(0), -np.ones(n0), np.ones(n0))
    return [gen.small_lp(2), no_rows, gen.ragged_rows(3, 80, 600), gen.free_and_boxed_mix(1, 40, 70),
            gen.tiny_bounded(4, 6, 9), gen.small_lp(5, m=30, n=40, density=0.2)]


@pytest.mark.parametrize("local", LOCAL)
@pytest.mark.parametrize("iters", [1, 100, 600])
@pytest.mark.parametrize("make", [lambda: small_batch(0), mixed_shapes])
def test_batch_fixed_iterations_match_oracle(cuda_device, make, iters, local):
    check_fixed_iterations(make(), iters, batch_local_nnz=local)


@pytest.mark.parametrize("local", [4000, 10 ** 9])
def test_batch_fixed_iterations_other_gamma(cuda_device, local):
    """gamma = 0.5: the small instances run on the plain-form cluster and single-CTA loops (the
    shared-memory loop runs the reflected form, gamma = 1 only)."""
    check_fixed_iterations(small_batch(3), 300, batch_local_nnz=local, gamma=0.5)


def check_fixed_iterations(lps, iters, **params):
    etas = [o_eta(lp) for lp in lps]
    traces, cut = [], []
    oparams = {k: v for k, v in params.items() if k != "batch_local_nnz"}
    for lp, e in zip(lps, etas):
        o = o_solve(lp, 0.0, iters, trace=True, eta=e, **oparams)
        tie = first_near_tie(o["trace"])
        if tie is not None and tie < iters - 1:  # the harness's floor on a cut comparison
            assert tie + 1 >= 0.9 * iters or tie_is_late(o["trace"], tie), (tie, iters)
        cut.append(iters if tie is None or tie >= iters - 1 else tie + 1)
        traces.append(o)
    with lpx.BatchSolver(lps, eta=etas, **params) as b:
        for T in sorted(set(cut)):
            b.solve(0.0, T)
            summ = b.summary()
            for k, lp in enumerate(lps):
                if cut[k] != T:
                    continue
                o = traces[k] if T == iters else o_solve(lp, 0.0, T, eta=etas[k], **oparams)
                g = b.get(k)
                assert g["status"] == o["status"] == oracle.ITER_LIMIT, k
                assert g["iters"] == o["iters"] == T, k
                assert_iterates_close(g["x"], o["x"])
                assert_iterates_close(g["y"], o["y"])
                np.testing.assert_allclose(g["kkt"], o["kkt"][:4], rtol=1e-8, atol=1e-14)
                assert summ["status"][k] == g["status"] and summ["iters"][k] == T


@pytest.mark.parametrize("local", LOCAL)
@pytest.mark.parametrize("seed", [1, 2])
def test_batch_to_tolerance(cuda_device, seed, local):
    """Every instance stops at its own first check meeting 1e-8 (Section 4), at the oracle's
    iteration unless a restart near-tie came first; the oracle's KKT evaluation of the point
    agrees and the objective is the planted one."""
    lps = small_batch(seed, count=12)
    etas = [o_eta(lp) for lp in lps]
    with lpx.BatchSolver(lps, eta=etas, batch_local_nnz=local) as b:
        b.solve(1e-8, 200000)
        res = [b.get(k) for k in range(len(lps))]
    for k, (lp, g) in enumerate(zip(lps, res)):
        o = o_solve(lp, 1e-8, 200000, trace=True, eta=etas[k])
        assert g["status"] == o["status"] == oracle.OPTIMAL, k
        tie = first_near_tie(o["trace"])
        if tie is None or tie >= o["iters"] - 1:
            assert g["iters"] == o["iters"], k
        else:  # only a converged-regime tie may move the stopping check, by one period at most
            assert tie_is_late(o["trace"], tie), (k, tie, o["iters"])
            assert abs(g["iters"] - o["iters"]) <= 64, (k, g["iters"], o["iters"])
        kk = oracle.kkt(lp, g["x"], g["y"])
        assert kk[3] <= 1e-8, k
        np.testing.assert_allclose(g["kkt"], kk[:4], rtol=1e-7, atol=1e-13)
        pstar = float(lp.c @ lp.x_star)
        assert abs(kk[4] - pstar) <= 1e-7 * (1 + abs(pstar)), k


@pytest.mark.parametrize("local", [0, 10 ** 9])
def test_batch_matches_single_instance_solver(cuda_device, local):
    """The batch and lp_solve run the same device functions; only block and task sums are added
    in different orders."""
    lps = small_batch(3, count=8)
    etas = [o_eta(lp) for lp in lps]
    with lpx.BatchSolver(lps, eta=etas, batch_local_nnz=local) as b:
        b.solve(0.0, 300)
        res = [b.get(k) for k in range(len(lps))]
    for lp, e, g in zip(lps, etas, res):
        with lpx.Solver(lp, eta=e) as s:
            s.solve(0.0, 300)
            r = s.result()
        o = o_solve(lp, 0.0, 300, trace=True, eta=e)
        tie = first_near_tie(o["trace"])
        rtol = 1e-10
        if tie is not None:  # a converged-regime tie may part the two sums' orders by about r_tie
            assert tie_is_late(o["trace"], tie), tie
            rtol = 1e-6
        assert_iterates_close(g["x"], r["x"], rtol=rtol)
        assert_iterates_close(g["y"], r["y"], rtol=rtol)


def test_batch_power_iteration_step_sizes(cuda_device):
    lps = small_batch(4, count=6) + [gen.ragged_rows(1, 50, 300)]
    with lpx.BatchSolver(lps) as b:
        b.solve(0.0, 1)
        eta_b = b.summary()["eta"]
    for lp, e in zip(lps, eta_b):
        with lpx.Solver(lp) as s:
            s.solve(0.0, 1)
            e1 = s.result()["eta"]
        # same start vector and stopping rule; the sums differ in order, so the stop may move
        # by a step: agreement to the power iteration's tolerance
        assert abs(e - e1) <= 1e-6 * e1
        assert abs(e - o_eta(lp)) <= 1e-6 * e


@pytest.mark.parametrize("local", LOCAL)
def test_batch_deterministic_and_reusable(cuda_device, local):
    lps = small_batch(5, count=9)
    with lpx.BatchSolver(lps, batch_local_nnz=local) as b:
        b.solve(1e-6, 5000)
        a = [b.get(k) for k in range(len(lps))]
        b.solve(1e-6, 5000)
        c = [b.get(k) for k in range(len(lps))]
    for u, v in zip(a, c):
        assert np.array_equal(u["x"], v["x"]) and np.array_equal(u["y"], v["y"])
        assert u["iters"] == v["iters"] and u["status"] == v["status"]


@pytest.mark.parametrize("local", LOCAL)
def test_batch_statuses_differ_per_instance(cuda_device, local):
    """Instances finish independently: with a tight limit some stop OPTIMAL, others hit it."""
    lps = small_batch(6, count=10)
    with lpx.BatchSolver(lps, batch_local_nnz=local) as b:
        b.solve(1e-6, 400)
        s = b.summary()
    assert set(s["status"].tolist()) <= {oracle.OPTIMAL, oracle.ITER_LIMIT}
    assert np.all((s["iters"] == 400) | (s["status"] == oracle.OPTIMAL))
    assert np.all(s["iters"] <= 400)
    opt = s["status"] == oracle.OPTIMAL
    assert np.all(s["iters"][opt] % 64 == 0)  # OPTIMAL only at check iterations
    assert 0 < opt.sum() < len(lps)


@pytest.mark.parametrize("local", [0, 4000])
@pytest.mark.parametrize("precision", [1, 2])
def test_batch_mixed_precision(cuda_device, precision, local):
    """FP32 stage for every instance, then (precision 1) the FP64 stage: each returned point is
    checked by the oracle's FP64 KKT evaluation."""
    lps = small_batch(7, count=10)
    tol = 1e-8 if precision == 1 else 1e-4
    with lpx.BatchSolver(lps, precision=precision, batch_local_nnz=local) as b:
        b.solve(tol, 200000)
        s = b.summary()
        res = [b.get(k) for k in range(len(lps))]
    for k, (lp, g) in enumerate(zip(lps, res)):
        kk = oracle.kkt(lp, g["x"], g["y"])
        if precision == 1:
            assert g["status"] == oracle.OPTIMAL, k
            assert 0 < s["iters_fp32"][k] <= g["iters"]
            assert kk[3] <= tol
            pstar = float(lp.c @ lp.x_star)
            assert abs(kk[4] - pstar) <= 1e-7 * (1 + abs(pstar)), k
        else:
            assert g["status"] in (oracle.OPTIMAL, lpx.LP_SOLVE_STALLED), k
            assert s["iters_fp32"][k] == g["iters"]
            if g["status"] == oracle.OPTIMAL:
                assert kk[3] <= tol * 1.01


def test_batch_time_loop(cuda_device):
    lps = small_batch(8, count=6)
    with lpx.BatchSolver(lps, precision=1, batch_local_nnz=0) as b:
        ms64, per = b.time_loop(64, fp64=True)
        ms32, _ = b.time_loop(64, fp64=False)
    assert per == 16 and ms64 > 0.0 and ms32 > 0.0


def test_tuner_picks_the_fastest_candidate_and_caches(cuda_device, tmp_path):
    lp = gen.miplib_like(3, 4000, 8000, 2000)
    cache = str(tmp_path / "schedules.txt")
    best, ms = lpx.lp_tune_schedule(lp, cache, timings=True)
    assert best == lpx.TUNE_CANDIDATES[int(np.argmin(ms))]
    assert np.all(ms > 0)
    lines = [ln for ln in open(cache).read().split("\n") if ln.strip()]
    assert len(lines) == 1 and lines[0].endswith(f" {100 * best[0] + best[1]}")
    assert lpx.lp_tune_schedule(lp, cache) == best       # from the cache: no new line
    assert len([ln for ln in open(cache).read().split("\n") if ln.strip()]) == 1


@pytest.mark.parametrize("local", [0, 10 ** 9])
def test_batch_with_per_instance_schedules_matches_oracle(cuda_device, local):
    """Each instance's tile schedule changes only how its rows are split among lanes and tiles."""
    lps = small_batch(9, count=6)
    tiles = [(2, 1), (32, 32), (8, 4), (4, 32), (16, 8), (1, 2)]
    etas = [o_eta(lp) for lp in lps]
    with lpx.BatchSolver(lps, eta=etas, tiles=tiles, batch_local_nnz=local) as b:
        b.solve(0.0, 200)
        res = [b.get(k) for k in range(len(lps))]
    for lp, e, g in zip(lps, etas, res):
        o = o_solve(lp, 0.0, 200, trace=True, eta=e)
        tie = first_near_tie(o["trace"])
        rtol = 1e-10
        if tie is not None:
            assert tie_is_late(o["trace"], tie), tie
            rtol = 1e-6
        assert_iterates_close(g["x"], o["x"], rtol=rtol)
        assert_iterates_close(g["y"], o["y"], rtol=rtol)


def test_batch_schedule_classes(cuda_device):
    """lp_batch_schedule: the grid loop for instances above batch_local_nnz; the small ones on the
    shared-memory cluster loop when all of them fit it, else single CTAs for tiny small instances
    (two row tiles and two column tiles at most per warp of a CTA) and clusters for the others."""
    lps = [gen.small_lp(0, m=30, n=50, density=0.2),        # 297 nonzeros, 1-2 tiles per side
           gen.small_lp(1, m=3000, n=3000, density=0.0005),  # 4,642 nonzeros, ~94 row tiles
           gen.small_lp(2, m=400, n=800, density=0.1)]       # 31,926 nonzeros
    long_row = gen.ragged_rows(3, 80, 600)                  # a row of more than 128 entries
    assert np.max(np.diff(long_row.row_ptr)) > 128
    with lpx.BatchSolver(lps) as b:
        assert b.schedule().tolist() == [3, 3, 0]
        b.solve(1e-6, 20000)
        assert np.all(b.summary()["status"] == oracle.OPTIMAL)
    with lpx.BatchSolver(lps, batch_local_nnz=0) as b:
        assert b.schedule().tolist() == [0, 0, 0]
    with lpx.BatchSolver(lps, batch_local_nnz=10 ** 9) as b:
        assert b.schedule().tolist() == [3, 3, 3]
    with lpx.BatchSolver(lps + [long_row], batch_local_nnz=10 ** 9) as b:
        where = b.schedule().tolist()
        assert where[:3] == [2, 1, 1] and where[3] in (1, 2)
        b.solve(1e-6, 20000)
        assert np.all(b.summary()["status"] == oracle.OPTIMAL)
