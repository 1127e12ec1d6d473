"""Parity at the benchmark workloads' full sizes, in the launch configurations bench.py times.

The oracle cannot run these workloads whole in seconds, so each test checks sampled outputs that
it can compute one by one: a few iterations of the multicommodity LP, sampled instances of the
512-LP batch, sampled instances of the differentiable layer's batch.  Where the oracle's own
power iteration on millions of nonzeros would dominate, both sides use the GPU's step size (the
step size itself is compared with the oracle's at smaller sizes in test_gpu_parity.py and
test_gpu_batch.py); for the layer, the oracle's unrolled map runs on the GPU's recorded
schedule (schedule agreement is tested in test_gpu_diff.py).
"""
import numpy as np
import pytest

import oracle
from oracle import diff as od
import paper_2507_14051_b300 as lpx
from paper_2507_14051_b300 import gen

from .test_gpu_diff import compare_grad, offsets
from .test_gpu_parity import assert_iterates_close, compare_fixed, first_near_tie

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch512():
    return gen.batch_uneven(0, count=512)


@pytest.fixture(scope="module")
def mcf():
    return gen.multicommodity(0)


def test_full_size_multicommodity_iterates(cuda_device, mcf):
    """The multicommodity benchmark LP (m = 1.8M, n = 4.0M, nnz = 12M), default parameters: 200
    iterations against the oracle element by element (three termination checks, at 64, 128 and
    192, and the restarts of the first epochs), with the GPU's step size on both sides."""
    lp = mcf
    with lpx.Solver(lp) as s:
        eta = s.solve(0.0, 1).result()["eta"]
    g, o = compare_fixed(lp, 200, eta=eta)
    assert int(np.sum(o["trace"][:, 2])) >= 5  # restarts compared
    assert o["iters"] >= 193


def test_full_size_multicommodity_fp64_to_1e4(cuda_device, mcf):
    """The plain FP64 solve of the multicommodity LP to 1e-4 (Section 4) with default parameters:
    OPTIMAL, and the oracle's FP64 KKT evaluation of the returned point meets the tolerance and
    agrees with the reported values."""
    with lpx.Solver(mcf) as s:
        r = s.solve(1e-4, 100000).result()
    assert r["status"] == oracle.OPTIMAL and r["iters_fp32"] == 0
    kk = oracle.kkt(mcf, r["x"], r["y"])
    assert kk[3] <= 1e-4
    np.testing.assert_allclose(r["kkt"], kk[:4], rtol=1e-7, atol=1e-13)


def test_full_size_mixed_multicommodity(cuda_device, mcf):
    """The multicommodity LP in mixed precision (FP32 phase, then FP64) to 1e-4: the oracle's
    FP64 KKT evaluation of the returned point meets the tolerance and agrees with the reported
    values."""
    with lpx.Solver(mcf, precision=1) as s:
        r = s.solve(1e-4, 100000).result()
    assert r["status"] == oracle.OPTIMAL and r["iters_fp32"] > 0
    kk = oracle.kkt(mcf, r["x"], r["y"])
    assert kk[3] <= 1e-4
    np.testing.assert_allclose(r["kkt"], kk[:4], rtol=1e-7, atol=1e-13)


def test_full_size_batch_mixed_to_tolerance(cuda_device, batch512):
    """The 512-LP batch in mixed precision to 1e-8: every instance that stops OPTIMAL reports a
    KKT error <= 1e-8, and for sampled instances the oracle's FP64 KKT evaluation of the returned
    point agrees and meets the tolerance."""
    lps = batch512
    with lpx.BatchSolver(lps, precision=1) as b:
        b.solve(1e-8, 100000)
        summ = b.summary()
        opt = np.nonzero(summ["status"] == oracle.OPTIMAL)[0]
        assert len(opt) >= 510
        assert np.all(summ["kkt"][opt, 3] <= 1e-8)
        nnz = np.array([lp.nnz for lp in lps])
        picks = [int(opt[np.argmin(nnz[opt])]), int(opt[len(opt) // 2]), int(opt[np.argmax(nnz[opt])])]
        got = {k: b.get(k) for k in picks}
    for k in picks:
        kk = oracle.kkt(lps[k], got[k]["x"], got[k]["y"])
        assert kk[3] <= 1e-8, k
        np.testing.assert_allclose(got[k]["kkt"], kk[:4], rtol=1e-7, atol=1e-13)


def test_full_size_batch_sampled_instances(cuda_device, batch512):
    """The 512-instance benchmark batch with the default schedule: after 30 iterations, the
    smallest and the largest small instance (the shared-memory cluster loop), a mid-size
    grid-loop one and the largest one equal the oracle's 30 iterations (with the batch's own step
    sizes) element by element."""
    lps = batch512
    T = 30
    with lpx.BatchSolver(lps) as b:
        where = b.schedule()
        b.solve(0.0, T)
        summ = b.summary()
        nnz = np.array([lp.nnz for lp in lps])
        grid = np.nonzero(where == 0)[0]
        small = np.nonzero(where != 0)[0]
        assert np.all(where[small] == 3)
        picks = [int(small[np.argmin(nnz[small])]), int(small[np.argmax(nnz[small])]),
                 int(grid[np.argsort(nnz[grid])[len(grid) // 2]]), int(np.argmax(nnz))]
        got = {k: b.get(k) for k in picks}
    assert np.all(summ["status"] == oracle.ITER_LIMIT) and np.all(summ["iters"] == T)
    compared = 0
    for k in picks:
        o = oracle.solve(lps[k], tol=0.0, max_iter=T, trace=True, eta=float(summ["eta"][k]))
        tie = first_near_tie(o["trace"])
        if tie is not None and tie < T - 1:
            continue
        assert o["status"] == oracle.ITER_LIMIT and o["iters"] == T
        assert_iterates_close(got[k]["x"], o["x"])
        assert_iterates_close(got[k]["y"], o["y"])
        compared += 1
    assert compared >= 3


def test_full_size_layer_sampled_instances(cuda_device):
    """The differentiable layer's benchmark batch (64 LPs of 1000 x 2000, K = 2000, checkpoints
    every 100, the layer's default schedule): for two instances the forward output equals the
    oracle's unrolled map on the GPU's schedule, and sampled gradient entries equal central
    differences of that map where it is affine on the difference interval."""
    import torch
    from paper_2507_14051_b300.diff import UnrolledLPBatch
    K, C = 2000, 100
    lps = [gen.small_lp(k, m=1000, n=2000, density=0.01) for k in range(64)]
    dev = torch.device("cuda")
    cat = lambda name: torch.tensor(np.concatenate([getattr(lp, name) for lp in lps]), device=dev)
    c, lc, uc, lv, uv = (cat(k) for k in ("c", "l_c", "u_c", "l_v", "u_v"))
    rng = np.random.default_rng(0)
    xt = rng.uniform(0.0, 1.0, c.shape[0])
    layer = UnrolledLPBatch(lps, K=K, checkpoint_every=C)
    try:
        cg = c.clone().requires_grad_(True)
        ucg = uc.clone().requires_grad_(True)
        x, y = layer(cg, lc, ucg, lv, uv)
        ((x - torch.tensor(xt, device=dev)) ** 2).sum().backward()
        xs = x.detach().cpu().numpy()
        ys = y.detach().cpu().numpy()
        gc = cg.grad.cpu().numpy()
        guc = ucg.grad.cpu().numpy()
        eta = layer.batch.summary()["eta"]
        picks = [0, 37]
        traces = {k: layer.batch.trace(k, K) for k in picks}
    finally:
        layer.close()
    ox, oy = offsets(lps, "n"), offsets(lps, "m")
    compared = 0
    for k in picks:
        lp, tr = lps[k], traces[k]
        assert tr.shape[0] == K
        xo, yo = od.unrolled(lp, tr, float(eta[k]), K)
        np.testing.assert_allclose(xs[ox[k]:ox[k + 1]], xo, rtol=0, atol=1e-10 * max(1, np.abs(xo).max()))
        np.testing.assert_allclose(ys[oy[k]:oy[k + 1]], yo, rtol=0, atol=1e-10 * max(1, np.abs(yo).max()))
        xtk = xt[ox[k]:ox[k + 1]]
        loss = lambda xx, yy, xtk=xtk: float(np.sum((xx - xtk) ** 2))
        idx = rng.choice(lp.n, size=4, replace=False)
        compared += compare_grad(lp, tr, float(eta[k]), K, loss, "c", idx, gc[ox[k]:ox[k + 1]][idx])
        fin = np.nonzero(np.isfinite(lp.u_c) & (lp.l_c != lp.u_c))[0]
        idx = rng.choice(fin, size=min(4, len(fin)), replace=False)
        compared += compare_grad(lp, tr, float(eta[k]), K, loss, "u_c", idx, guc[oy[k]:oy[k + 1]][idx])
    assert compared >= 4


def test_full_size_miplib_like_to_tolerance(cuda_device):
    """The MIPLIB-shaped benchmark LP solved to 1e-8 with the default parameters (as the
    benchmark's tolerance run does, about a minute): the oracle's FP64 KKT evaluation of the
    returned point meets the tolerance and agrees with the reported values, and the objective is
    the planted optimum's."""
    lp = gen.miplib_like(0)
    with lpx.Solver(lp) as s:
        r = s.solve(1e-8, 3_000_000).result()
    assert r["status"] == oracle.OPTIMAL and r["iters"] % 64 == 0
    kk = oracle.kkt(lp, r["x"], r["y"])
    # the relative gap |pobj - dobj| / (1 + |pobj| + |dobj|) cancels two nearly equal sums of
    # ~10^5 terms; its rounding is absolute, about u times the sum of the terms' magnitudes
    # over the denominator (1e-11 here), not relative to the tiny gap: a point the GPU accepts
    # with a gap just under the tolerance can be evaluated just over it by the oracle
    assert kk[1] <= 1e-8 and kk[2] <= 1e-8 and kk[0] <= 1e-8 + 1e-10
    np.testing.assert_allclose(r["kkt"][0], kk[0], rtol=0, atol=1e-10)
    np.testing.assert_allclose(r["kkt"][1:3], kk[1:3], rtol=1e-7, atol=1e-13)
    # the reported relative KKT error is the largest of the three; when that is the gap it
    # carries the gap's absolute rounding
    assert r["kkt"][3] == max(r["kkt"][:3]) and kk[3] == max(kk[:3])
    assert abs(r["kkt"][3] - kk[3]) <= 1e-10 + 1e-7 * kk[3]
    # the planted optimum p* lies between the objectives up to the residuals weighted by the
    # optimal multipliers (weak duality for a point that violates the constraints by pres and the
    # dual constraints by dres): |pobj - p*| <= |pobj - dobj| + |y*| pres + |x*| dres
    pstar = float(lp.c @ lp.x_star)
    bound = abs(kk[4] - kk[5]) + np.linalg.norm(lp.y_star) * kk[6] + np.linalg.norm(lp.x_star) * kk[7]
    assert abs(kk[4] - pstar) <= bound + 1e-9 * (1 + abs(pstar))
