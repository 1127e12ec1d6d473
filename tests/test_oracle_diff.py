"""Pins of the differentiation oracle (oracle/diff.py) to things other than itself:
  * the unrolled map with the oracle solve's own recorded schedule reproduces that solve;
  * the active-set (implicit KKT) gradient of the LP solution equals central differences of an
    independent LP solver's solution (scipy's HiGHS) under perturbations of b;
  * central differences of the unrolled map approach that implicit gradient as K grows (the
    unrolled derivative converges to the solution's derivative at a nondegenerate vertex), and
    the c-gradient tends to 0 (the vertex does not move with c).
"""
import numpy as np
import pytest
from scipy.optimize import linprog

import oracle
from oracle import diff as od
from paper_2507_14051_b300 import gen


@pytest.mark.parametrize("K", [1, 37, 300])
@pytest.mark.parametrize("make", [lambda: gen.small_lp(0, m=30, n=50, density=0.2),
                                  lambda: gen.free_and_boxed_mix(3, 25, 40)])
def test_unrolled_with_recorded_schedule_reproduces_the_solve(make, K):
    lp = make()
    tr, eta = od.schedule(lp, K)
    x, y = od.unrolled(lp, tr, eta, K)
    o = oracle.solve(lp, tol=0.0, max_iter=K, eta=eta)
    np.testing.assert_allclose(x, o["x"], rtol=0, atol=1e-12 * max(1.0, np.abs(o["x"]).max()))
    np.testing.assert_allclose(y, o["y"], rtol=0, atol=1e-12 * max(1.0, np.abs(o["y"]).max()))


def test_unrolled_without_scaling_is_the_plain_iteration():
    lp = gen.small_lp(2, m=20, n=30, density=0.3)
    kw = dict(ruiz_iters=0, pc_enabled=0)
    tr, eta = od.schedule(lp, 120, **kw)
    x, y = od.unrolled(lp, tr, eta, 120, **kw)
    o = oracle.solve(lp, tol=0.0, max_iter=120, eta=eta, **kw)
    np.testing.assert_allclose(x, o["x"], atol=1e-12)
    np.testing.assert_allclose(y, o["y"], atol=1e-12)


def _loss_and_grad(lp, seed=0):
    xt = np.random.default_rng(seed).uniform(0, 1, lp.n)
    return (lambda x, y: float(np.sum((x - xt) ** 2))), (lambda x: 2.0 * (x - xt))


@pytest.mark.parametrize("seed", [1, 2])
def test_implicit_gradient_matches_highs_differences(seed):
    v = gen.vertex_lp(seed)
    loss, grad = _loss_and_grad(v)
    imp = od.implicit_grad(v, v.x_star, v.y_star, grad(v.x_star))
    A = v.dense()

    def x_of(b):
        r = linprog(v.c, A_eq=A, b_eq=b, bounds=list(zip(v.l_v, v.u_v)), method="highs",
                    options=dict(primal_feasibility_tolerance=1e-10, dual_feasibility_tolerance=1e-10))
        assert r.status == 0
        return r.x

    np.testing.assert_allclose(x_of(v.l_c), v.x_star, atol=1e-8)  # the planted vertex is HiGHS's optimum
    h = 1e-4
    for i in range(v.m):
        bp, bm = v.l_c.copy(), v.l_c.copy()
        bp[i] += h
        bm[i] -= h
        fd = (loss(x_of(bp), None) - loss(x_of(bm), None)) / (2 * h)
        assert abs(fd - imp["b"][i]) <= 1e-7 * (1 + abs(fd)), i
    # moving a variable's bound moves the vertex (entries of variables at a bound)
    N = np.nonzero(np.isclose(v.x_star, 0) | np.isclose(v.x_star, 1))[0][:4]
    for j in N:
        key = "l_v" if np.isclose(v.x_star[j], 0) else "u_v"
        lo, hi = v.l_v.copy(), v.u_v.copy()
        arr = lo if key == "l_v" else hi
        arr[j] += h
        xp = linprog(v.c, A_eq=A, b_eq=v.l_c, bounds=list(zip(lo, hi)), method="highs").x
        arr[j] -= 2 * h
        xm = linprog(v.c, A_eq=A, b_eq=v.l_c, bounds=list(zip(lo, hi)), method="highs").x
        fd = (loss(xp, None) - loss(xm, None)) / (2 * h)
        assert abs(fd - imp[key][j]) <= 1e-6 * (1 + abs(fd)), j
    assert np.all(imp["c"] == 0.0)


def test_unrolled_derivative_approaches_the_implicit_one():
    v = gen.vertex_lp(1)
    loss, grad = _loss_and_grad(v)
    imp = od.implicit_grad(v, v.x_star, v.y_star, grad(v.x_star))
    idx = [0, 7, 13]
    errs = []
    for K in (500, 4000):
        tr, eta = od.schedule(v, K)
        g = od.fd_grad(v, tr, eta, K, loss, "b", idx)
        errs.append(np.abs(g - imp["b"][idx]).max())
    assert errs[1] < 1e-5 * max(1.0, np.abs(imp["b"]).max()) and errs[1] < errs[0]
    tr, eta = od.schedule(v, 4000)
    gc = od.fd_grad(v, tr, eta, 4000, loss, "c", [1, 9, 22])
    assert np.abs(gc).max() < 1e-5


def test_finite_differences_of_an_affine_piece_are_exact():
    """Fixed schedule, no bound active anywhere (bounds far away): the unrolled map is affine in
    c, so central differences with two step sizes agree to rounding."""
    lp = gen.small_lp(4, m=15, n=25, density=0.3)
    lp.l_v = np.full(lp.n, -1e3)
    lp.u_v = np.full(lp.n, 1e3)
    lp.l_c = np.full(lp.m, -1e3)
    lp.u_c = np.full(lp.m, 1e3)
    loss, _ = _loss_and_grad(lp)
    tr, eta = od.schedule(lp, 40)
    lin = lambda x, y: float(np.sum(x))  # linear loss: exactly affine composition
    g1 = od.fd_grad(lp, tr, eta, 40, lin, "c", [0, 5, 9], h=1e-6)
    g2 = od.fd_grad(lp, tr, eta, 40, lin, "c", [0, 5, 9], h=1e-3)
    np.testing.assert_allclose(g1, g2, rtol=1e-6, atol=1e-9)
