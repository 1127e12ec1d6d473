"""Oracle of the differentiable unrolled solve.

TEST INFRASTRUCTURE ONLY: tests and ``bench.py``'s CPU baseline may import it; the CUDA library
never does.  Plain numpy, FP64, natural order, no blocking or fusion.

The map being differentiated is the oracle's own iteration (``orc_solve``: the PDHG step of
Section 2.2, eq. (pdhg), then restart or reflected Halpern update, Section 3) run for K
iterations from zero in the preconditioned variables, with the restart schedule, the epoch
steps and the primal weight taken from a recorded trace instead of being decided.  Its
derivative is checked two ways, neither of which shares code with the CUDA path:
  * ``fd_grad``: central finite differences of ``unrolled`` (the definition of a derivative);
  * ``implicit_grad``: the derivative of the LP solution itself from its active-set KKT system
    (the limit the unrolled derivative approaches at a nondegenerate vertex), itself pinned in
    tests against finite differences of an independent LP solver (scipy's HiGHS).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

import oracle


def schedule(lp, K, **params):
    """The oracle's own trace of a K-iteration solve (tolerance 0) and its step size eta:
    rows (r_t, omega_t, restart flag, k_t)."""
    out = oracle.solve(lp, tol=0.0, max_iter=K, trace=True, **params)
    return out["trace"], out["eta"]


def _scaled(lp, c, l_c, u_c, l_v, u_v, ruiz_iters, pc_enabled, pc_alpha):
    val, dr, dc = oracle.scale(lp, ruiz_iters=ruiz_iters, pc_enabled=pc_enabled, pc_alpha=pc_alpha)
    A = sp.csr_matrix((val, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n))
    return A, dr, dc, c * dc, l_c * dr, u_c * dr, l_v / dc, u_v / dc


def unrolled(lp, trace, eta, K, gamma=1.0, c=None, l_c=None, u_c=None, l_v=None, u_v=None,
             ruiz_iters=10, pc_enabled=1, pc_alpha=1.0, codes=None):
    """zhat after K iterations with the given schedule, in the original variables.  If codes is
    a list, the clamp codes of every step are appended to it (per step: for each column 0
    inside / 1 below l_v / 2 above u_v, then the same for each row against l_c, u_c)."""
    c = lp.c if c is None else c
    l_c = lp.l_c if l_c is None else l_c
    u_c = lp.u_c if u_c is None else u_c
    l_v = lp.l_v if l_v is None else l_v
    u_v = lp.u_v if u_v is None else u_v
    A, dr, dc, cs, lcs, ucs, lvs, uvs = _scaled(lp, c, l_c, u_c, l_v, u_v, ruiz_iters, pc_enabled, pc_alpha)
    x = np.zeros(lp.n)
    y = np.zeros(lp.m)
    x0 = np.zeros(lp.n)
    y0 = np.zeros(lp.m)
    xh, yh = x, y
    for t in range(K):
        omega, restart, k = trace[t, 1], trace[t, 2], trace[t, 3]
        tau, sigma = eta / omega, eta * omega
        # primal step, then the dual step at the extrapolated point (Section 2.2, eq. (pdhg))
        a_ = x - tau * (cs - A.T @ y)
        xh = np.clip(a_, lvs, uvs)
        s = A @ (2.0 * xh - x) - y / sigma
        yh = sigma * (np.clip(s, lcs, ucs) - s)
        if codes is not None:
            codes.append(np.concatenate([(a_ < lvs) * 1 + (a_ > uvs) * 2, (s < lcs) * 1 + (s > ucs) * 2]))
        if restart:
            x, y, x0, y0 = xh, yh, xh, yh
        else:  # reflected Halpern step with the epoch step k (Section 3)
            a, b = (k + 1.0) / (k + 2.0), 1.0 / (k + 2.0)
            x = a * ((1.0 + gamma) * xh - gamma * x) + b * x0
            y = a * ((1.0 + gamma) * yh - gamma * y) + b * y0
    return xh * dc, yh * dr


def fd_grad(lp, trace, eta, K, loss, wrt, idx, h=1e-6, **kw):
    """Central differences of loss(x, y) through ``unrolled`` in the entries idx of the vector
    named wrt ('c', 'l_c', 'u_c', 'l_v', 'u_v'; 'b' moves l_c and u_c together)."""
    base = {k: np.array(getattr(lp, k), dtype=np.float64) for k in ("c", "l_c", "u_c", "l_v", "u_v")}
    out = np.zeros(len(idx))
    for q, i in enumerate(idx):
        vals = []
        for sgn in (1.0, -1.0):
            d = {k: v.copy() for k, v in base.items()}
            for name in (("l_c", "u_c") if wrt == "b" else (wrt,)):
                d[name][i] += sgn * h
            vals.append(loss(*unrolled(lp, trace, eta, K, **d, **kw)))
        out[q] = (vals[0] - vals[1]) / (2.0 * h)
    return out


def fd_sides(lp, trace, eta, K, loss, wrt, idx, h=1e-6, **kw):
    """One-sided differences (forward, backward) of loss through ``unrolled`` in the entries idx
    of wrt, and the unperturbed loss: where the two differences disagree, some clamp of the map
    sits exactly at its kink and the derivative does not exist there.  Also returns, per entry,
    whether every clamp of every step takes the same branch at theta - h, theta and theta + h:
    then the map is affine on that interval and the central difference is its derivative up to
    rounding."""
    base = {k: np.array(getattr(lp, k), dtype=np.float64) for k in ("c", "l_c", "u_c", "l_v", "u_v")}
    c0 = []
    L0 = loss(*unrolled(lp, trace, eta, K, **base, **kw, codes=c0))
    c0 = np.concatenate(c0) if c0 else np.zeros(0)
    fwd, bwd = np.zeros(len(idx)), np.zeros(len(idx))
    same = np.zeros(len(idx), dtype=bool)
    for q, i in enumerate(idx):
        vals, ok = [], True
        for sgn in (1.0, -1.0):
            d = {k: v.copy() for k, v in base.items()}
            for name in (("l_c", "u_c") if wrt == "b" else (wrt,)):
                d[name][i] += sgn * h
            cs = []
            vals.append(loss(*unrolled(lp, trace, eta, K, **d, **kw, codes=cs)))
            ok = ok and np.array_equal(np.concatenate(cs) if cs else np.zeros(0), c0)
        fwd[q] = (vals[0] - L0) / h
        bwd[q] = (L0 - vals[1]) / h
        same[q] = ok
    return fwd, bwd, L0, same


def implicit_grad(lp, x, y, gx, tol=1e-7):
    """dL/d(c, b, l_v, u_v) of the LP solution x*(c, b, bounds) at a nondegenerate optimal
    vertex, for a loss with gradient gx in x.  Active set from (x, y): variables within tol of
    a bound are fixed there (N), the others free (F); rows with |y| > tol are tight (R) on the
    side the sign of y selects.  With |F| = |R| and A_RF nonsingular, x_F solves
    A_RF x_F = b_R - A_RN x_N, so dL/db_R = A_RF^{-T} gx_F, dL/dx_N = gx_N - A_RN^T A_RF^{-T} gx_F,
    and dL/dc = 0 (the vertex does not move under a small change of c)."""
    A = lp.dense()
    lo = np.isclose(x, lp.l_v, atol=tol, rtol=0.0)
    hi = np.isclose(x, lp.u_v, atol=tol, rtol=0.0)
    F = np.nonzero(~lo & ~hi)[0]
    N = np.nonzero(lo | hi)[0]
    R = np.nonzero(np.abs(y) > tol)[0]
    if len(F) != len(R):
        raise ValueError(f"not a nondegenerate vertex: {len(F)} free variables, {len(R)} tight rows")
    ARF = A[np.ix_(R, F)]
    w = np.linalg.solve(ARF.T, gx[F])
    out = {k: np.zeros_like(np.asarray(getattr(lp, k), dtype=np.float64)) for k in ("c", "l_c", "u_c", "l_v", "u_v")}
    out["b"] = np.zeros(lp.m)
    out["b"][R] = w
    lower_side = y[R] > 0
    out["l_c"][R[lower_side]] = w[lower_side]
    out["u_c"][R[~lower_side]] = w[~lower_side]
    gN = gx[N] - A[np.ix_(R, N)].T @ w
    out["l_v"][N[lo[N]]] = gN[lo[N]]
    out["u_v"][N[hi[N] & ~lo[N]]] = gN[hi[N] & ~lo[N]]
    return out
