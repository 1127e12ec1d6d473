"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names the passage of the paper (arXiv 2507.14051) it checks and what pins it:
hand-worked values (tests/golden), closed forms, invariants of the method, brute force on
tiny inputs, and an independent library LP solver (HiGHS through scipy).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2507_14051_b300 import gen

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _num(v):
    if v == "inf":
        return math.inf
    if v == "-inf":
        return -math.inf
    if v == "sqrt5/(1+sqrt5)":
        return math.sqrt(5) / (1 + math.sqrt(5))
    return float(v)


def _lp_from_dense(d):
    A = np.array(d["A"], dtype=float)
    m, n = A.shape
    rows, vals = [], []
    for i in range(m):
        nz = np.nonzero(A[i])[0]
        rows.append(nz)
        vals.append(A[i, nz])
    rp, ci, v = gen._csr_from_rows(m, n, rows, vals)
    f = lambda k: np.array([_num(t) for t in d[k]], dtype=float)
    return gen.LP(m, n, rp, ci, v, f("c"), f("l_c"), f("u_c"), f("l_v"), f("u_v"))


# ------------------------------------------------------------------ PDHG step (Section 2.2)

def test_pdhg_step_hand_worked():
    """Section 2.2 eq. (pdhg): two steps of a 1x1 LP worked by hand."""
    g = _load("pdhg_step_1x1.json")
    lp = _lp_from_dense(g["lp"])
    for st in g["steps"]:
        xp, yp = oracle.pdhg_step(lp, g["eta"], g["omega"], np.array(st["x"]), np.array(st["y"]))
        np.testing.assert_allclose(xp, st["x_plus"], rtol=0, atol=1e-15)
        np.testing.assert_allclose(yp, st["y_plus"], rtol=0, atol=1e-15)


def _printed_dual_step(lp, eta, omega, x, y, xp):
    """The dual line of eq. (pdhg) exactly as printed, with dense numpy products."""
    sigma = eta * omega
    A = lp.dense()
    axbar = A @ (2 * xp - x)
    w = y / sigma - axbar
    proj = np.minimum(np.maximum(w, -lp.u_c), -lp.l_c)  # onto -S = [-u_c, -l_c]
    return y - sigma * axbar - sigma * proj


@pytest.mark.parametrize("seed", range(4))
def test_dual_step_equals_printed_form(seed):
    """The oracle's y+ = sigma (proj_S(s) - s) is the printed dual update of eq. (pdhg)."""
    lp = gen.free_and_boxed_mix(seed, 30, 40)
    rng = np.random.default_rng(100 + seed)
    x, y = rng.standard_normal(lp.n), rng.standard_normal(lp.m)
    eta, omega = 0.3, 1.7
    xp, yp = oracle.pdhg_step(lp, eta, omega, x, y)
    ref = _printed_dual_step(lp, eta, omega, x, y, xp)
    np.testing.assert_allclose(yp, ref, rtol=1e-12, atol=1e-12)
    # primal line as printed (dense)
    A = lp.dense()
    xref = np.clip(x - (eta / omega) * (lp.c - A.T @ y), lp.l_v, lp.u_v)
    np.testing.assert_allclose(xp, xref, rtol=1e-13, atol=1e-13)


def test_pdhg_step_closed_form_A_zero():
    """A = 0: the step decouples into x+ = proj_X(x - tau c) and y+ = sigma(proj_S(-y/sigma) + y/sigma)."""
    rng = np.random.default_rng(7)
    m, n = 5, 6
    rp = np.zeros(m + 1, np.int64)
    lp = gen.LP(m, n, rp, np.zeros(0, np.int32), np.zeros(0), rng.standard_normal(n),
                np.array([-1.0, -np.inf, 0.0, -2.0, -np.inf]), np.array([1.0, 0.5, np.inf, -2.0, np.inf]),
                np.array([-np.inf, 0.0, -1.0, 0.0, -3.0, -np.inf]), np.array([np.inf, np.inf, 1.0, 2.0, -1.0, 0.0]))
    x, y = rng.standard_normal(n), rng.standard_normal(m)
    eta, omega = 0.7, 0.4
    tau, sigma = eta / omega, eta * omega
    xp, yp = oracle.pdhg_step(lp, eta, omega, x, y)
    np.testing.assert_allclose(xp, np.clip(x - tau * lp.c, lp.l_v, lp.u_v), rtol=0, atol=1e-15)
    s = -y / sigma
    np.testing.assert_allclose(yp, sigma * (np.clip(s, lp.l_c, lp.u_c) - s), rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("seed", range(3))
def test_step_lands_in_X_and_Y(seed):
    """x+ in X and y+ in Y (sets of Section 2.1) for every row/column bound pattern."""
    lp = gen.free_and_boxed_mix(seed, 40, 50)
    rng = np.random.default_rng(seed)
    for _ in range(5):
        x, y = 10 * rng.standard_normal(lp.n), 10 * rng.standard_normal(lp.m)
        xp, yp = oracle.pdhg_step(lp, 0.2, 0.5, x, y)
        assert np.all(xp >= lp.l_v) and np.all(xp <= lp.u_v)
        assert np.all(yp[~np.isfinite(lp.l_c)] <= 0.0)  # no finite lower side: y <= 0
        assert np.all(yp[~np.isfinite(lp.u_c)] >= 0.0)  # no finite upper side: y >= 0


# --------------------------------------------------------------------- P-norm, T (Section 2.2)

def _p_inner(lp, eta, omega, a, b):
    """<a, b>_P by polarisation of the oracle's ||.||_P^2."""
    ax, ay = a
    bx, by = b
    plus = oracle.p_norm_sq(lp, eta, omega, ax + bx, ay + by)
    minus = oracle.p_norm_sq(lp, eta, omega, ax - bx, ay - by)
    return 0.25 * (plus - minus)


@pytest.mark.parametrize("seed", range(3))
def test_T_firmly_nonexpansive_in_P(seed):
    """PDHG is a proximal point step in the metric P (Section 2.2), so T is firmly
    nonexpansive there: ||Tz - Tz'||_P^2 <= <Tz - Tz', z - z'>_P, whenever eta ||A|| < 1."""
    lp = gen.free_and_boxed_mix(seed, 25, 35, density=0.2)
    nA = np.linalg.norm(lp.dense(), 2)
    eta = 0.95 / nA
    rng = np.random.default_rng(seed + 50)
    for trial in range(20):
        omega = float(np.exp(rng.uniform(-2, 2)))
        z1 = (rng.standard_normal(lp.n) * 3, rng.standard_normal(lp.m) * 3)
        z2 = (rng.standard_normal(lp.n) * 3, rng.standard_normal(lp.m) * 3)
        t1 = oracle.pdhg_step(lp, eta, omega, *z1)
        t2 = oracle.pdhg_step(lp, eta, omega, *z2)
        dT = (t1[0] - t2[0], t1[1] - t2[1])
        dz = (z1[0] - z2[0], z1[1] - z2[1])
        lhs = oracle.p_norm_sq(lp, eta, omega, *dT)
        rhs = _p_inner(lp, eta, omega, dT, dz)
        assert lhs <= rhs + 1e-10 * (abs(rhs) + 1.0), (trial, lhs, rhs)


def test_P_positive_definite_iff_eta_norm_below_one():
    """P = [[w/eta I, A^T], [A, 1/(eta w) I]] (Section 2.2) is positive definite exactly when
    eta ||A||_2 < 1: checked along the top singular pair of A."""
    lp = gen.small_lp(3, m=20, n=30, density=0.3)
    A = lp.dense()
    U, S, Vt = np.linalg.svd(A)
    u, v = U[:, 0], Vt[0]
    for scale, positive in ((0.99, True), (1.01, False)):
        eta = scale / S[0]
        omega = 1.3
        # minimiser of the quadratic form on span{(v,0), (0,u)}: dx = v * sqrt(omega)^-1, dy = -u sqrt(omega)
        val = oracle.p_norm_sq(lp, eta, omega, v / np.sqrt(omega), -u * np.sqrt(omega))
        assert (val > 0) == positive, (scale, val)


@pytest.mark.parametrize("gamma", [0.0, 0.5, 1.0])
@pytest.mark.parametrize("which", ["small", "miplib"])
def test_halpern_rate_bound(gamma, which):
    """Reflected Halpern without restarts (Section 3): with S = (1+gamma)T - gamma I
    nonexpansive in P, Lieder's bound ||z_k - S z_k|| <= 2||z_0 - z*||/(k+1) gives
    r(z_k) = ||z_k - T z_k||_P <= 2 ||z_0 - z*||_P / ((1+gamma)(k+1)) for the planted z*."""
    lp = gen.small_lp(0) if which == "small" else gen.miplib_like(0, m=400, n=800, lmax=400)
    nA, _ = oracle.power_norm(lp, tol=1e-13, max_iter=100000)
    eta = 0.998 / nA
    out = oracle.solve(lp, tol=0.0, max_iter=1500, trace=True, restart_enabled=0, pid_enabled=0,
                       eta=eta, gamma=gamma, ruiz_iters=0, pc_enabled=0)
    r = out["trace"][:, 0]
    d0 = math.sqrt(oracle.p_norm_sq(lp, eta, 1.0, -lp.x_star, -lp.y_star))
    k = np.arange(len(r))
    assert np.all(r <= 2 * d0 / ((1 + gamma) * (k + 1)) * (1 + 1e-9))
    assert np.all(out["trace"][:, 2] == 0)


# ----------------------------------------------------------------- KKT (Section 4)

def test_kkt_hand_worked():
    g = _load("kkt_hand.json")
    lp = _lp_from_dense(g["lp"])
    for pt in g["points"]:
        k = oracle.kkt(lp, np.array(pt["x"]), np.array(pt["y"]))
        np.testing.assert_allclose(k[:3], [_num(pt["rel_gap"]), _num(pt["rel_pres"]), _num(pt["rel_dres"])],
                                   rtol=1e-15, atol=1e-16)
        assert k[3] == max(k[:3])


@pytest.mark.parametrize("make", [lambda: gen.small_lp(1), lambda: gen.free_and_boxed_mix(2, 60, 80),
                                  lambda: gen.ragged_rows(3, 80, 120), lambda: gen.miplib_like(1, 2000, 4000, 500),
                                  lambda: gen.tiny_bounded(4, 3, 4)])
def test_kkt_zero_at_planted_optimum(make):
    """The generator plants (x*, y*, r*) satisfying the optimality conditions exactly, so all
    three criteria of Section 4 vanish up to rounding."""
    lp = make()
    k = oracle.kkt(lp, lp.x_star, lp.y_star)
    assert k[3] <= 1e-13, k
    # and the dual multiplier of each variable is the planted r*
    rc = lp.c - oracle.spmv_t(lp, lp.y_star)
    np.testing.assert_allclose(rc, lp.r_star, atol=1e-12)


def test_kkt_detects_each_violation():
    """Leaving the planted optimum raises the matching criterion of Section 4."""
    lp = gen.free_and_boxed_mix(2, 40, 60)
    assert oracle.kkt(lp, lp.x_star, lp.y_star)[3] < 1e-13
    y = lp.y_star.copy()
    y[np.argmax((lp.y_star > 0) & (np.diff(lp.row_ptr) > 0))] *= 2.0
    assert oracle.kkt(lp, lp.x_star, y)[3] > 1e-4            # gap or dual residual
    x = lp.x_star.copy()
    x[lp.col_idx[0]] += 5.0
    assert oracle.kkt(lp, x, lp.y_star)[1] > 1e-4            # primal residual
    lower_only = np.isfinite(lp.l_v) & ~np.isfinite(lp.u_v)
    j = int(np.argmax(lower_only))
    c = lp.c.copy()
    c[j] -= 3.0                                              # reduced cost < 0 on an x >= l variable
    bad = gen.LP(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, c, lp.l_c, lp.u_c, lp.l_v, lp.u_v)
    assert oracle.kkt(bad, lp.x_star, lp.y_star)[2] > 1e-4   # dual residual


# ------------------------------------------------------------ restart and PID (Section 3)

def test_restart_decisions_hand_labelled():
    g = _load("restart_decisions.json")
    bs, bn, ba = g["betas"]
    for cs in g["cases"]:
        got = oracle.restart_decide(cs["k"], cs["t"], cs["r"], cs["r0"], cs["r_prev"], bs, bn, ba)
        assert got == cs["restart"], cs


def _frac(v):
    num, _, den = v.partition("/")
    return float(num) / float(den or 1)


def test_restart_trace_hand_worked():
    """Section 3, the restart bookkeeping inside the solve: nine iterations of a 1x1 LP worked by
    hand with exact fractions (tests/golden/restart_trace_1x1.json), spanning two artificial
    restarts.  Each step's PDHG output (x^, y^), residual r_t, primal weight, epoch step k and
    restart flag follow from r0 = r at the epoch's first step, r_prev = the previous step's r,
    the restart point and anchor = the PDHG output z^ (not the pre-step iterate z), and the PID
    update at each restart (K_P = 1 gives omega' = |dy| / |dx|)."""
    g = _load("restart_trace_1x1.json")
    lp = _lp_from_dense(g["lp"])
    prm = dict(g["params"])
    steps = g["steps"]
    T = len(steps)
    out = oracle.solve(lp, tol=0.0, max_iter=T, trace=True, **prm)
    tr = out["trace"]
    assert tr.shape[0] == T
    for st, row in zip(steps, tr):
        assert row[0] == pytest.approx(math.sqrt(_frac(st["r2"])), rel=1e-12), st["t"]
        assert row[1] == pytest.approx(_frac(st["omega"]), rel=1e-12), st["t"]
        assert row[2] == st["restart"], st["t"]
        assert row[3] == st["k"], st["t"]
    for st in steps:  # the solve stopped after t + 1 iterations returns z^_t
        o = oracle.solve(lp, tol=0.0, max_iter=st["t"] + 1, **prm)
        assert o["x"][0] == pytest.approx(_frac(st["xhat"]), rel=1e-12, abs=1e-14), st["t"]
        assert o["y"][0] == pytest.approx(_frac(st["yhat"]), rel=1e-12, abs=1e-14), st["t"]


@pytest.mark.parametrize("seed", range(3))
def test_restart_decisions_follow_the_epoch_definitions(seed):
    """Section 3: at every step with k >= 1 of a long solve, the oracle restarts exactly when the
    (separately pinned) decision rule says so for r0 = the residual of the epoch's first step
    (k = 0) and r_prev = the residual of the step before; after a restart the next step has
    k = 0, otherwise k + 1; the primal weight changes only right after a restart."""
    lp = gen.free_and_boxed_mix(seed, 40, 70) if seed == 2 else gen.small_lp(seed, 60, 140, 0.05)
    out = oracle.solve(lp, tol=0.0, max_iter=4000, trace=True, check_every=10 ** 6)
    tr = out["trace"]
    restarts = 0
    r0 = None
    for t in range(tr.shape[0]):
        r, om, flag, k = tr[t]
        if k == 0:
            r0 = r
            assert flag == 0.0
        else:
            want = oracle.restart_decide(int(k), t, r, r0, tr[t - 1, 0])
            assert bool(flag) == want, (t, r, r0, tr[t - 1, 0], k)
        if t + 1 < tr.shape[0]:
            assert tr[t + 1, 3] == (0.0 if flag else k + 1), t
            if not flag:
                assert tr[t + 1, 1] == om, t
        restarts += int(flag)
    assert restarts >= 5


def test_pid_three_restarts_hand_worked():
    g = _load("pid_three_restarts.json")
    pid = oracle.PID(g["gains"]["k_p"], g["gains"]["k_i"], g["gains"]["k_d"])
    w = g["omega0"]
    for rs in g["restarts"]:
        w = pid.update(w, rs["dx"], rs["dy"])
        assert math.log2(w) == pytest.approx(rs["log2_omega_after"], abs=1e-12)


def test_pid_proportional_only_is_pdlp_smoothing():
    """K_P = theta, K_I = K_D = 0 gives the exponential smoothing of the earlier primal weight
    rule (Section 3, 'cuPDLP ... smoothed using exponential averaging'):
    log w+ = (1 - theta) log w + theta log(|dy| / |dx|)."""
    rng = np.random.default_rng(11)
    for theta in (0.2, 0.5, 0.9):
        pid = oracle.PID(theta, 0.0, 0.0)
        w = 1.0
        for _ in range(10):
            dx, dy = np.exp(rng.uniform(-3, 3, 2))
            want = math.exp((1 - theta) * math.log(w) + theta * math.log(dy / dx))
            w = pid.update(w, dx, dy)
            assert w == pytest.approx(want, rel=1e-13)


def test_pid_skips_degenerate_norms():
    pid = oracle.PID(0.5, 0.1, 0.0)
    assert pid.update(2.0, 0.0, 1.0) == 2.0
    assert pid.update(2.0, 1.0, 0.0) == 2.0
    assert pid.update(2.0, math.inf, 1.0) == 2.0
    assert np.all(pid.state == 0.0)


# ----------------------------------------------------------- stepsize (Section 3)

@pytest.mark.parametrize("make", [lambda: gen.small_lp(0), lambda: gen.ragged_rows(1, 60, 90),
                                  lambda: gen.miplib_like(2, 300, 600, 300)])
def test_power_iteration_matches_lapack_norm(make):
    """||A||_2 by power iteration (Section 3, stepsize) against LAPACK's SVD."""
    lp = make()
    est, it = oracle.power_norm(lp, tol=1e-12, max_iter=200000)
    ref = np.linalg.norm(lp.dense(), 2)
    assert est == pytest.approx(ref, rel=1e-6)
    assert est <= ref * (1 + 1e-12)  # the Rayleigh quotient never overshoots


def test_start_vector_is_splitmix64():
    """Start vector from splitmix64 (published constants), top 53 bits mapped to [-1, 1)."""
    def sm(seed, i):
        M = (1 << 64) - 1
        z = (seed + (i + 1) * 0x9E3779B97F4A7C15) & M
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        z ^= z >> 31
        return (z >> 11) / 2.0 ** 53 * 2.0 - 1.0
    for seed in (0, 1, 12345):
        for i in (0, 1, 2, 1000):
            assert oracle.start_entry(seed, i) == sm(seed, i)
    # first output of the stream seeded with 0 is the published 0xE220A8397B1DCDAF
    assert oracle.start_entry(0, 0) == (0xE220A8397B1DCDAF >> 11) / 2.0 ** 53 * 2.0 - 1.0


# ------------------------------------------------------------ preconditioning

def test_ruiz_equilibrates_rows_and_columns():
    """Many Ruiz passes drive every row and column max-norm of D_r A D_c to 1 (Ruiz 2001)."""
    lp = gen.miplib_like(3, 400, 700, 300)
    val, dr, dc = oracle.scale(lp, ruiz_iters=60, pc_enabled=0)
    rows = np.repeat(np.arange(lp.m), np.diff(lp.row_ptr))
    rmax = np.zeros(lp.m)
    np.maximum.at(rmax, rows, np.abs(val))
    cmax = np.zeros(lp.n)
    np.maximum.at(cmax, lp.col_idx, np.abs(val))
    nzr = np.diff(lp.row_ptr) > 0
    nzc = np.bincount(lp.col_idx, minlength=lp.n) > 0
    assert np.all(np.abs(rmax[nzr] - 1) < 1e-6) and np.all(np.abs(cmax[nzc] - 1) < 1e-6)
    np.testing.assert_allclose(val, dr[rows] * lp.val * dc[lp.col_idx], rtol=1e-12)
    assert np.all(dr[~nzr] == 1.0) and np.all(dc[~nzc] == 1.0)


def test_pock_chambolle_pass():
    """One Pock-Chambolle pass with alpha = 1 (Pock & Chambolle 2011): d_r = 1/sqrt(row l1),
    d_c = 1/sqrt(column l1), both of the unscaled matrix."""
    lp = gen.ragged_rows(5, 50, 70)
    val, dr, dc = oracle.scale(lp, ruiz_iters=0, pc_enabled=1, pc_alpha=1.0)
    A = np.abs(lp.dense())
    r1, c1 = A.sum(1), A.sum(0)
    np.testing.assert_allclose(dr, np.where(r1 > 0, 1 / np.sqrt(np.where(r1 > 0, r1, 1)), 1.0), rtol=1e-14)
    np.testing.assert_allclose(dc, np.where(c1 > 0, 1 / np.sqrt(np.where(c1 > 0, c1, 1)), 1.0), rtol=1e-14)


# -------------------------------------------------------------- full solve

@pytest.mark.parametrize("seed", range(5))
def test_solve_reaches_planted_optimum(seed):
    """Restarted reflected Halpern PDHG (Sections 2.2, 3) from zero (Section 4) reaches
    relative KKT 1e-8 (Section 4) and the planted optimal objective."""
    lp = gen.small_lp(seed)
    out = oracle.solve(lp, tol=1e-8, max_iter=100000, ruiz_iters=10, pc_enabled=1)
    assert out["status"] == oracle.OPTIMAL
    assert out["kkt"][3] <= 1e-8
    pstar = float(lp.c @ lp.x_star)
    assert abs(out["kkt"][4] - pstar) <= 1e-7 * (1 + abs(pstar))
    # the reported KKT is that of the returned point on the original LP
    np.testing.assert_allclose(oracle.kkt(lp, out["x"], out["y"])[:4], out["kkt"][:4], rtol=1e-9, atol=1e-15)


def _vertex_enumeration(lp):
    """min c^T x over the bounded polytope by enumerating all vertices (tiny n)."""
    A = lp.dense()
    G, h = [], []   # G x <= h
    for i in range(lp.m):
        if np.isfinite(lp.u_c[i]):
            G.append(A[i]); h.append(lp.u_c[i])
        if np.isfinite(lp.l_c[i]):
            G.append(-A[i]); h.append(-lp.l_c[i])
    for j in range(lp.n):
        e = np.zeros(lp.n); e[j] = 1.0
        G.append(e); h.append(lp.u_v[j])
        G.append(-e); h.append(-lp.l_v[j])
    G, h = np.array(G), np.array(h)
    best = math.inf
    for S in itertools.combinations(range(len(h)), lp.n):
        M = G[list(S)]
        if abs(np.linalg.det(M)) < 1e-12:
            continue
        x = np.linalg.solve(M, h[list(S)])
        if np.all(G @ x <= h + 1e-9):
            best = min(best, float(lp.c @ x))
    return best


@pytest.mark.parametrize("seed", range(6))
def test_solve_matches_vertex_enumeration(seed):
    lp = gen.tiny_bounded(seed, m=3, n=4)
    ref = _vertex_enumeration(lp)
    out = oracle.solve(lp, tol=1e-10, max_iter=200000, check_every=1)
    assert out["status"] == oracle.OPTIMAL
    assert out["kkt"][4] == pytest.approx(ref, rel=1e-8, abs=1e-8)


def _linprog(lp):
    from scipy.optimize import linprog
    A = lp.dense()
    eq = lp.l_c == lp.u_c
    A_ub, b_ub = [], []
    for i in np.nonzero(~eq)[0]:
        if np.isfinite(lp.u_c[i]):
            A_ub.append(A[i]); b_ub.append(lp.u_c[i])
        if np.isfinite(lp.l_c[i]):
            A_ub.append(-A[i]); b_ub.append(-lp.l_c[i])
    bounds = [(None if not np.isfinite(a) else a, None if not np.isfinite(b) else b) for a, b in zip(lp.l_v, lp.u_v)]
    res = linprog(lp.c, A_ub=np.array(A_ub) if A_ub else None, b_ub=np.array(b_ub) if b_ub else None,
                  A_eq=A[eq] if eq.any() else None, b_eq=lp.l_c[eq] if eq.any() else None,
                  bounds=bounds, method="highs")
    assert res.status == 0
    return res.fun


@pytest.mark.parametrize("make", [lambda: gen.free_and_boxed_mix(0, 60, 90), lambda: gen.ragged_rows(2, 70, 110),
                                  lambda: gen.small_lp(7, m=80, n=160, density=0.05)])
def test_solve_matches_highs(make):
    lp = make()
    ref = _linprog(lp)
    out = oracle.solve(lp, tol=1e-9, max_iter=300000, ruiz_iters=10, pc_enabled=1)
    assert out["status"] == oracle.OPTIMAL
    assert out["kkt"][4] == pytest.approx(ref, rel=1e-7, abs=1e-7)


def test_status_iteration_limit_and_numerical():
    lp = gen.small_lp(0)
    out = oracle.solve(lp, tol=1e-12, max_iter=7)
    assert out["status"] == oracle.ITER_LIMIT and out["iters"] == 7
    assert np.isfinite(out["kkt"][3])  # the last iteration is always a check iteration
    bad = gen.free_and_boxed_mix(0, 30, 40)
    free = int(np.argmax(~np.isfinite(bad.l_v) & ~np.isfinite(bad.u_v)))
    bad.c = bad.c.copy()
    bad.c[free] = 1e308   # |x - xhat|^2 overflows in the first residual
    out = oracle.solve(bad, tol=1e-8, max_iter=100, eta=0.1, ruiz_iters=0, pc_enabled=0)
    assert out["status"] == oracle.NUMERICAL and out["iters"] == 1


def test_check_period_does_not_change_the_trajectory():
    """The termination test (Section 4) only reads the iterates: a coarser check period stops
    at a multiple of the period, never earlier than the per-iteration test, on a point of the
    same trajectory (bitwise)."""
    lp = gen.small_lp(1)
    a = oracle.solve(lp, tol=1e-6, max_iter=100000, check_every=1, eta=0.1)
    b = oracle.solve(lp, tol=1e-6, max_iter=100000, check_every=16, eta=0.1)
    assert a["status"] == b["status"] == oracle.OPTIMAL
    assert b["iters"] % 16 == 0 and b["iters"] >= a["iters"] and b["kkt"][3] <= 1e-6
    same = oracle.solve(lp, tol=0.0, max_iter=b["iters"], check_every=1, eta=0.1)
    assert np.array_equal(same["x"], b["x"]) and np.array_equal(same["y"], b["y"])
