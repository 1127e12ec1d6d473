"""Bound/objective rescaling (after the diagonal preconditioning: objective divided by ||c~||_2,
all bounds by the 2-norm of the finite constraint bounds) is a change of variables
x' = x~ / beta, y' = y~ / gamma.  Under it every PDHG step, the P-norm residual (scaled by
1/sqrt(beta gamma)), the restart decisions and the PID error are the same as those of the
unrescaled iteration started from omega0 * gamma / beta: the rescaled solve is the plain solve
with that initial primal weight.  Pinned here on the oracle, whose rescaling is written out
explicitly; the GPU implements the option as that initial weight."""
import numpy as np
import pytest

import oracle
from paper_2507_14051_b300 import gen


def ratio(lp, **kw):
    val, dr, dc = oracle.scale(lp, **kw)
    b = np.concatenate([lp.l_c * dr, lp.u_c * dr])
    b = b[np.isfinite(b)]
    beta = np.linalg.norm(b) if np.any(b != 0) else 1.0
    gam = np.linalg.norm(lp.c * dc) if np.any(lp.c != 0) else 1.0
    return gam / beta, beta, gam


@pytest.mark.parametrize("make", [lambda: gen.small_lp(0), lambda: gen.free_and_boxed_mix(1, 40, 70),
                                  lambda: gen.miplib_like(2, 300, 600, 200)])
def test_rescaled_solve_is_the_plain_solve_with_a_scaled_initial_weight(make):
    lp = make()
    w, beta, gam = ratio(lp)
    a = oracle.solve(lp, tol=0.0, max_iter=400, trace=True, rescale=1)
    b = oracle.solve(lp, tol=0.0, max_iter=400, trace=True, rescale=0, omega0=w)
    np.testing.assert_array_equal(a["trace"][:, 2], b["trace"][:, 2])
    np.testing.assert_allclose(a["trace"][:, 1] * w, b["trace"][:, 1], rtol=1e-9)
    np.testing.assert_allclose(a["trace"][:, 0] * np.sqrt(beta * gam), b["trace"][:, 0], rtol=1e-8,
                               atol=1e-12 * b["trace"][:, 0].max())
    for key in ("x", "y"):
        np.testing.assert_allclose(a[key], b[key], rtol=0, atol=1e-9 * max(1.0, np.abs(b[key]).max()))


def test_rescaled_solve_reaches_the_planted_optimum():
    lp = gen.small_lp(3)
    o = oracle.solve(lp, tol=1e-8, max_iter=100000, rescale=1)
    assert o["status"] == oracle.OPTIMAL
    k = oracle.kkt(lp, o["x"], o["y"])
    assert k[3] <= 1e-8
    assert abs(k[4] - lp.c @ lp.x_star) <= 1e-7 * (1 + abs(lp.c @ lp.x_star))
