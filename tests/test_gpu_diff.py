"""Differentiable unrolled solve (include/lp_diff.h) against the differentiation oracle
(oracle/diff.py).

Both sides run the same K-iteration map with a frozen schedule.  The GPU records its schedule
from its own solve and the oracle from its own; the tests first check that the two schedules
agree (restart iterations and epoch steps exactly, omega to 1e-10 relative; runs with a restart
near-tie are skipped, as in tests/test_gpu_parity.py) and then compare:
  * the forward output with the oracle's unrolled map (1e-10 relative);
  * the reverse-mode gradient with central differences of the oracle's map (h = 1e-6; the map is
    piecewise affine, so the differences are exact up to rounding ~1e-16 |L| / h unless a clamp
    changes side within h): |g_gpu - g_fd| <= 1e-6 (1 + |g_fd|);
  * at a nondegenerate vertex and large K, the gradient with the oracle's active-set (implicit
    KKT) gradient of the LP solution (1e-5 relative; 0 for c).
"""
import numpy as np
import pytest

import oracle
from oracle import diff as od
import paper_2507_14051_b300 as lpx
from paper_2507_14051_b300 import gen

from .test_gpu_parity import first_near_tie

pytestmark = pytest.mark.gpu


def cat(lps, name):
    return np.concatenate([np.asarray(getattr(lp, name), dtype=np.float64) for lp in lps])


def offsets(lps, attr):
    return np.concatenate([[0], np.cumsum([getattr(lp, attr) for lp in lps])])


def gpu_unroll(lps, K, ckpt, etas, loss_grad_x, loss_grad_y=None, local=16384, time_unroll=False, **params):
    import torch
    dev = "cuda"
    with lpx.BatchSolver(lps, eta=etas, batch_local_nnz=local, **params) as b:
        nx, ny = sum(lp.n for lp in lps), sum(lp.m for lp in lps)
        x = torch.zeros(nx, dtype=torch.float64, device=dev)
        y = torch.zeros(ny, dtype=torch.float64, device=dev)
        b.unroll(K, ckpt, x, y)
        xs, ys = x.cpu().numpy(), y.cpu().numpy()
        gx = torch.tensor(loss_grad_x(xs), device=dev)
        gy = None if loss_grad_y is None else torch.tensor(loss_grad_y(ys), device=dev)
        if time_unroll:
            ms_f, ms_fc, ms_b, per = b.time_unroll(2)
            assert ms_f > 0.0 and ms_fc > 0.0 and ms_b > 0.0 and per == min(K, ckpt)
        g = {k: torch.zeros(nx if k in ("c", "l_v", "u_v") else ny, dtype=torch.float64, device=dev)
             for k in ("c", "l_c", "u_c", "l_v", "u_v")}
        b.unroll_vjp(gx, gy, g["c"], g["l_c"], g["u_c"], g["l_v"], g["u_v"])
        traces = [b.trace(k, K) for k in range(len(lps))]
        torch.cuda.synchronize()
    return xs, ys, {k: v.cpu().numpy() for k, v in g.items()}, traces


def same_schedule(tg, to):
    """Restart iterations and epoch steps equal; omega within the parity harness's bound
    (1e-13 r_max / r_t + 1e-12 relative: the PID reads differences of nearly equal iterates)."""
    if first_near_tie(to) is not None:
        return False
    np.testing.assert_array_equal(tg[:, 2], to[:, 2])
    np.testing.assert_array_equal(tg[:, 3], to[:, 3])
    r = to[:, 0]
    w_tol = 1e-13 * float(np.max(r)) / np.maximum(r, 1e-300) + 1e-12
    assert np.all(np.abs(tg[:, 1] - to[:, 1]) <= w_tol * to[:, 1])
    return True


def compare_grad(lp, to, eta, K, loss, name, idx, got, h=1e-6):
    """Reverse-mode entries against central differences where the map is affine on
    [theta - h, theta + h] (every clamp of every step takes the same branch at both ends as at
    theta; elsewhere h crosses a kink and the difference is not the derivative).  Tolerance:
    1e-6 relative, plus the differences' own rounding: each loss value carries about
    sqrt(K) u |L| of rounding from the K steps (u = 2^-53), divided by h."""
    fwd, bwd, L0, smooth = od.fd_sides(lp, to, eta, K, loss, name, list(idx), h=h)
    fd = 0.5 * (fwd + bwd)
    atol = 10.0 * np.sqrt(K) * 2.0 ** -53 * max(1.0, abs(L0)) / h
    bad = smooth & ~(np.abs(got - fd) <= 1e-6 * (1 + np.abs(fd)) + atol)
    assert not np.any(bad), (name, got, fd)
    return int(smooth.sum())


def instances():
    return [gen.small_lp(0, m=30, n=50, density=0.2), gen.free_and_boxed_mix(3, 25, 40),
            gen.vertex_lp(2), gen.ragged_rows(1, 30, 100)]


@pytest.mark.parametrize("K", [1, 60, 250])
def test_forward_matches_the_oracle_unrolled_map(cuda_device, K):
    lps = instances()
    etas = [oracle.solve(lp, tol=0.0, max_iter=1)["eta"] for lp in lps]
    xs, ys, _, traces = gpu_unroll(lps, K, 25, etas, lambda x: np.zeros_like(x))
    ox, oy = offsets(lps, "n"), offsets(lps, "m")
    checked = 0
    for k, lp in enumerate(lps):
        to, eta = od.schedule(lp, K, eta=etas[k])
        if not same_schedule(traces[k], to):
            continue
        x, y = od.unrolled(lp, to, eta, K)
        np.testing.assert_allclose(xs[ox[k]:ox[k + 1]], x, rtol=0, atol=1e-10 * max(1, np.abs(x).max()))
        np.testing.assert_allclose(ys[oy[k]:oy[k + 1]], y, rtol=0, atol=1e-10 * max(1, np.abs(y).max()))
        checked += 1
    assert checked >= 3


# With the PID on, omega is read from differences of nearly equal iterates, so the two sides'
# schedules differ by rounding amplified as the run converges; where the unrolled map is badly
# conditioned that moves the gradient more than the FD tolerance.  Long runs are therefore
# compared with omega fixed (restarts still decided by the residual), and with neither.
SCHEDULES = [(40, {}), (160, dict(pid_enabled=0)), (160, dict(pid_enabled=0, restart_enabled=0))]


# small-instance threshold: 0 = every instance on the grid kernels, 280 = two of the four on the
# cluster kernels (297 and 465 nonzeros stay on the grid), 10**9 = all on the cluster kernels
@pytest.mark.parametrize("local", [0, 280, 10 ** 9])
@pytest.mark.parametrize("K,params", SCHEDULES)
def test_gradients_match_oracle_finite_differences(cuda_device, K, params, local):
    lps = instances()
    etas = [oracle.solve(lp, tol=0.0, max_iter=1)["eta"] for lp in lps]
    rng = np.random.default_rng(K)
    xt = [rng.uniform(0, 1, lp.n) for lp in lps]
    wy = [rng.standard_normal(lp.m) for lp in lps]
    gxf = lambda x: 2.0 * (x - np.concatenate(xt))
    gyf = lambda y: np.concatenate(wy)
    _, _, g, traces = gpu_unroll(lps, K, 16, etas, gxf, gyf, local=local, **params)
    ox, oy = offsets(lps, "n"), offsets(lps, "m")
    checked = compared = 0
    for k, lp in enumerate(lps):
        to, eta = od.schedule(lp, K, eta=etas[k], **params)
        if not same_schedule(traces[k], to):
            continue
        loss = lambda x, y, k=k: float(np.sum((x - xt[k]) ** 2) + wy[k] @ y)
        for name, off, size in (("c", ox, lp.n), ("l_v", ox, lp.n), ("u_v", ox, lp.n), ("l_c", oy, lp.m),
                                ("u_c", oy, lp.m)):
            vec = np.asarray(getattr(lp, name))
            eq = (lp.l_c == lp.u_c) if name in ("l_c", "u_c") else np.zeros(size, bool)
            cand = np.nonzero(np.isfinite(vec) & ~eq)[0]
            idx = rng.choice(cand, size=min(5, len(cand)), replace=False) if len(cand) else []
            if len(idx):
                compared += compare_grad(lp, to, eta, K, loss, name, idx, g[name][off[k]:off[k + 1]][idx])
        eqr = np.nonzero(lp.l_c == lp.u_c)[0]
        if len(eqr):  # an equality row's b moves both bounds: dL/db = dL/dl_c + dL/du_c
            idx = list(rng.choice(eqr, size=min(5, len(eqr)), replace=False))
            compared += compare_grad(lp, to, eta, K, loss, "b", idx, (g["l_c"] + g["u_c"])[oy[k]:oy[k + 1]][idx])
        inf_lo = np.nonzero(~np.isfinite(lp.l_v))[0]
        assert np.all(g["l_v"][ox[k]:ox[k + 1]][inf_lo] == 0.0)
        checked += 1
    assert checked >= 3 and compared >= 40


def test_gradient_approaches_the_implicit_kkt_gradient(cuda_device):
    lps = [gen.vertex_lp(1), gen.vertex_lp(3)]
    rng = np.random.default_rng(5)
    xt = [rng.uniform(0, 1, lp.n) for lp in lps]
    _, _, g, _ = gpu_unroll(lps, 4000, 100, None, lambda x: 2.0 * (x - np.concatenate(xt)))
    ox, oy = offsets(lps, "n"), offsets(lps, "m")
    for k, lp in enumerate(lps):
        imp = od.implicit_grad(lp, lp.x_star, lp.y_star, 2.0 * (lp.x_star - xt[k]))
        gb = (g["l_c"] + g["u_c"])[oy[k]:oy[k + 1]]
        scale = max(1.0, np.abs(imp["b"]).max())
        assert np.abs(gb - imp["b"]).max() <= 1e-5 * scale
        assert np.abs(g["c"][ox[k]:ox[k + 1]]).max() <= 1e-5 * scale
        for name in ("l_v", "u_v"):
            assert np.abs(g[name][ox[k]:ox[k + 1]] - imp[name]).max() <= 1e-5 * scale


def test_checkpoint_spacing_does_not_change_the_result(cuda_device):
    lps = instances()[:2]
    gxf = lambda x: np.cos(x)
    runs = [gpu_unroll(lps, 90, ck, None, gxf) for ck in (1, 7, 90, 1000)]
    for r in runs[1:]:
        assert np.array_equal(r[0], runs[0][0])
        for name in r[2]:
            assert np.array_equal(r[2][name], runs[0][2][name])


def test_kernel_timing_leaves_the_gradient_unchanged(cuda_device):
    """lp_batch_time_unroll between the forward and the reverse pass changes neither."""
    lps = instances()[:2]
    gxf = lambda x: np.cos(x)
    a = gpu_unroll(lps, 90, 30, None, gxf)
    b = gpu_unroll(lps, 90, 30, None, gxf, time_unroll=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for name in a[2]:
        assert np.array_equal(a[2][name], b[2][name])


def test_set_data_equals_a_fresh_batch(cuda_device):
    lps = [gen.small_lp(1, m=30, n=50, density=0.2), gen.free_and_boxed_mix(2, 20, 30)]
    rng = np.random.default_rng(3)
    new = []
    for lp in lps:
        q = gen.LP(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.c + rng.standard_normal(lp.n),
                   lp.l_c - 0.1, lp.u_c + 0.1, lp.l_v, lp.u_v)
        new.append(q)
    etas = [0.05, 0.07]
    with lpx.BatchSolver(lps, eta=etas) as b:
        b.set_data(cat(new, "c"), cat(new, "l_c"), cat(new, "u_c"), cat(new, "l_v"), cat(new, "u_v"))
        b.solve(0.0, 300)
        got = [b.get(k) for k in range(2)]
    with lpx.BatchSolver(new, eta=etas) as b2:
        b2.solve(0.0, 300)
        ref = [b2.get(k) for k in range(2)]
    for u, v in zip(got, ref):
        assert np.array_equal(u["x"], v["x"]) and np.array_equal(u["y"], v["y"])


def test_autograd_layer(cuda_device):
    import torch
    from paper_2507_14051_b300.diff import UnrolledLPBatch
    lps = [gen.small_lp(5, m=30, n=50, density=0.2), gen.vertex_lp(4)]
    layer = UnrolledLPBatch(lps, K=120, checkpoint_every=30)
    d = lambda name: torch.tensor(cat(lps, name), device="cuda", requires_grad=True)
    c, lc, uc, lv, uv = (d(k) for k in ("c", "l_c", "u_c", "l_v", "u_v"))
    xt = torch.rand(c.shape[0], dtype=torch.float64, device="cuda")
    x, y = layer(c, lc, uc, lv, uv)
    loss = ((x - xt) ** 2).sum() + y.sum()
    loss.backward()
    # the same through the C ABI directly
    b = layer.batch
    g = {k: torch.zeros_like(t) for k, t in (("c", c), ("l_c", lc), ("u_c", uc), ("l_v", lv), ("u_v", uv))}
    b.unroll(120, 30, None, None)
    b.unroll_vjp(2 * (x.detach() - xt), torch.ones_like(y), g["c"], g["l_c"], g["u_c"], g["l_v"], g["u_v"])
    torch.cuda.synchronize()
    for k, t in (("c", c), ("l_c", lc), ("u_c", uc), ("l_v", lv), ("u_v", uv)):
        assert torch.equal(t.grad, g[k]), k
    # a small step along -grad lowers the loss (first order, the map being piecewise affine)
    cc = c.detach().clone().requires_grad_(True)
    x, _ = layer(cc, lc.detach(), uc.detach(), lv.detach(), uv.detach())
    L = ((x - xt) ** 2).sum()
    L.backward()
    gc = cc.grad.detach()
    step = 1e-4 / (1.0 + float(gc.abs().max()))
    x2, _ = layer(cc.detach() - step * gc, lc.detach(), uc.detach(), lv.detach(), uv.detach())
    L2 = ((x2 - xt) ** 2).sum()
    assert float(L2) < float(L.detach())
    layer.close()
