"""Seeded synthetic LP instances (inputs only).

This module draws problem data and nothing else: it holds none of the
solver's arithmetic and imports neither the CUDA library nor the oracle, so
both sides can take their inputs from it.

Every instance is a CSR matrix A (int64 row pointers, int32 column indices,
float64 values) plus c, l_c, u_c, l_v, u_v in the LP form of Section 2.1,
    min c^T x  s.t.  l_c <= A x <= u_c,  l_v <= x <= u_v,
with +-inf for absent bounds.  The ``known_optimum`` construction plants a
primal-dual pair (x*, y*, r*) that satisfies the optimality conditions of the
primal-dual form (Section 2.1) exactly:
  * x* in X, with chosen coordinates at a bound;
  * r* = c - A^T y* in R, nonzero only at active variable bounds, with the
    sign the set R_j requires;
  * y* in Y, nonzero only on rows whose active side is finite, with the sign
    Y_i requires;
so the duality gap c^T x* - dual(y*, r*) is zero.

Workload recipes (sizes and distributions of the workloads the method is
evaluated on; the MIPLIB-2017 relaxations and the large multicommodity class
of Section 4 are not available and are stood in for by these):
  * ``small_lp``        m=200, n=500, 2 % density, N(0,1) entries, x* in
                        [0,1] with 40 % at a bound, y* 50 % nonzero.
  * ``miplib_like``     m=50k, n=100k, nnz~600k, power-law row lengths on
                        [1, 2000], 70 % +-1 entries, the rest +-10^U(-3,3),
                        mixed row types, 30 % of variables without upper bound.
  * ``multicommodity``  node-arc multicommodity flow with joint arc
                        capacities (balanced supplies from a planted flow).
  * ``tiny_bounded``    n, m <= 6 with every bound finite (for brute force).
"""
from __future__ import annotations

import dataclasses
import numpy as np

INF = np.inf


@dataclasses.dataclass
class LP:
    m: int
    n: int
    row_ptr: np.ndarray   # int64[m+1]
    col_idx: np.ndarray   # int32[nnz]
    val: np.ndarray       # float64[nnz]
    c: np.ndarray
    l_c: np.ndarray
    u_c: np.ndarray
    l_v: np.ndarray
    u_v: np.ndarray
    x_star: np.ndarray | None = None
    y_star: np.ndarray | None = None
    r_star: np.ndarray | None = None
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def dense(self) -> np.ndarray:
        """Dense copy of A (small instances only)."""
        A = np.zeros((self.m, self.n))
        for i in range(self.m):
            s, e = self.row_ptr[i], self.row_ptr[i + 1]
            A[i, self.col_idx[s:e]] += self.val[s:e]
        return A

    def scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col_idx, self.row_ptr), shape=(self.m, self.n))


def _csr_from_rows(m: int, n: int, rows: list[np.ndarray], vals: list[np.ndarray]):
    lens = np.array([len(r) for r in rows], dtype=np.int64)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(lens, out=row_ptr[1:])
    col_idx = np.concatenate(rows).astype(np.int32) if rows else np.zeros(0, np.int32)
    val = np.concatenate(vals).astype(np.float64) if vals else np.zeros(0)
    return row_ptr, col_idx, val


def random_csr(rng: np.random.Generator, m: int, n: int, density: float):
    """Bernoulli(density) sparsity, N(0,1) values, columns sorted in each row."""
    rows, vals = [], []
    for _ in range(m):
        mask = rng.random(n) < density
        cols = np.nonzero(mask)[0]
        rows.append(cols)
        vals.append(rng.standard_normal(len(cols)))
    return _csr_from_rows(m, n, rows, vals)


def _matvec(row_ptr, col_idx, val, x):
    """s = A x for the generator's own bookkeeping (planting row bounds)."""
    m = len(row_ptr) - 1
    prod = val * x[col_idx]
    out = np.zeros(m)
    nonempty = row_ptr[:-1] < row_ptr[1:]
    if len(prod):  # segments start at the non-empty rows only (reduceat needs starts < len)
        out[nonempty] = np.add.reduceat(prod, row_ptr[:-1][nonempty])
    return out


def _rmatvec(row_ptr, col_idx, val, y, n):
    rows = np.repeat(np.arange(len(row_ptr) - 1), np.diff(row_ptr))
    return np.bincount(col_idx, weights=val * y[rows], minlength=n).astype(np.float64)


def known_optimum(rng, m, n, row_ptr, col_idx, val, l_v, u_v, *, frac_at_bound=0.4,
                  y_nonzero=0.5, row_type=None, name=""):
    """Plant (x*, y*, r*) and set c, l_c, u_c so that KKT holds exactly.

    row_type (optional, per row): 0 equality, 1 '>=', 2 '<=', 3 ranged,
    restricting which sides of a row may be finite; None lets each row pick.
    """
    l_v = np.asarray(l_v, dtype=np.float64)
    u_v = np.asarray(u_v, dtype=np.float64)
    x = np.empty(n)
    r = np.zeros(n)
    fin_l, fin_u = np.isfinite(l_v), np.isfinite(u_v)
    u = rng.random(n)
    at_lo = (u < frac_at_bound / 2) & fin_l
    at_hi = (u >= frac_at_bound / 2) & (u < frac_at_bound) & fin_u
    # variables with only one finite bound that drew the missing side go to the other one
    at_lo |= (u >= frac_at_bound / 2) & (u < frac_at_bound) & ~fin_u & fin_l
    lo_b = np.where(fin_l, l_v, np.where(fin_u, u_v - 10.0, -5.0))
    hi_b = np.where(fin_u, u_v, lo_b + 10.0)
    t = rng.uniform(0.1, 0.9, n)
    x[:] = lo_b + t * (hi_b - lo_b)
    x[at_lo] = l_v[at_lo]
    x[at_hi] = u_v[at_hi]
    r[at_lo] = rng.uniform(0.1, 1.0, at_lo.sum())
    r[at_hi] = -rng.uniform(0.1, 1.0, at_hi.sum())

    s = _matvec(row_ptr, col_idx, val, x)
    if row_type is None:
        row_type = rng.integers(0, 4, m)
    nz = rng.random(m) < y_nonzero
    sign = np.where(rng.random(m) < 0.5, 1.0, -1.0)
    # sign allowed by the row type: '>=' rows only y >= 0, '<=' rows only y <= 0
    sign = np.where(row_type == 1, 1.0, np.where(row_type == 2, -1.0, sign))
    mag = rng.uniform(0.1, 1.0, m)
    slack = rng.uniform(0.5, 2.0, (m, 2))
    which = rng.integers(0, 3, m)  # for the free choice of the inactive side
    y = np.where(nz, sign * mag, 0.0)
    pos, neg = y > 0, y < 0
    eq, ge, le, rg = row_type == 0, row_type == 1, row_type == 2, row_type == 3
    # equality: l = u = s;  '>=': u = inf, l = s where y > 0 else s - slack;  '<=': mirrored;
    # ranged: the side carrying the multiplier is tight, the other at a slack (both slack if y = 0)
    l_c = np.where(eq, s, np.where(ge, np.where(pos, s, s - slack[:, 0]),
                   np.where(le, -INF, np.where(neg | (y == 0), s - slack[:, 0], s))))
    u_c = np.where(eq, s, np.where(ge, INF, np.where(le, np.where(neg, s, s + slack[:, 1]),
                   np.where(pos | (y == 0), s + slack[:, 1], s))))
    # ranged rows: optional widening to infinity on the side that carries no multiplier
    u_c = np.where(rg & (which == 2) & pos, INF, u_c)
    l_c = np.where(rg & (which == 2) & neg, -INF, l_c)
    c = _rmatvec(row_ptr, col_idx, val, y, n) + r
    return LP(m, n, row_ptr, col_idx, val, c, l_c, u_c, l_v.copy(), u_v.copy(), x, y, r, name)


def small_lp(seed: int, m: int = 200, n: int = 500, density: float = 0.02) -> LP:
    """Small LP: Bernoulli(2 %) N(0,1) matrix, box [0,1] on every variable."""
    rng = np.random.default_rng(seed)
    rp, ci, v = random_csr(rng, m, n, density)
    return known_optimum(rng, m, n, rp, ci, v, np.zeros(n), np.ones(n),
                         frac_at_bound=0.4, y_nonzero=0.5, name=f"small_{m}x{n}_s{seed}")


def tiny_bounded(seed: int, m: int, n: int, density: float = 0.6) -> LP:
    """Tiny LP with every bound finite (bounded feasible region)."""
    rng = np.random.default_rng(seed)
    rp, ci, v = random_csr(rng, m, n, density)
    lv = -rng.uniform(0.5, 2.0, n)
    uv = rng.uniform(0.5, 2.0, n)
    lp = known_optimum(rng, m, n, rp, ci, v, lv, uv, frac_at_bound=0.5, y_nonzero=0.5,
                       row_type=np.full(m, 3), name=f"tiny_{m}x{n}_s{seed}")
    return lp


def power_law_lengths(rng, m: int, lmax: int = 2000, alpha: float = 1.748) -> np.ndarray:
    L = np.arange(1, lmax + 1)
    p = L.astype(np.float64) ** (-alpha)
    p /= p.sum()
    return rng.choice(L, size=m, p=p)


def miplib_like(seed: int = 0, m: int = 50_000, n: int = 100_000, lmax: int = 2000) -> LP:
    """MIPLIB-relaxation-shaped LP (power-law rows, mixed coefficient scales)."""
    rng = np.random.default_rng(seed)
    lens = power_law_lengths(rng, m, min(lmax, n))
    rows, vals = [], []
    for i in range(m):
        cols = np.sort(rng.choice(n, size=int(lens[i]), replace=False))
        L = len(cols)
        unit = rng.random(L) < 0.7
        sgn = np.where(rng.random(L) < 0.5, 1.0, -1.0)
        mag = np.where(unit, 1.0, 10.0 ** rng.uniform(-3.0, 3.0, L))
        rows.append(cols)
        vals.append(sgn * mag)
    rp, ci, v = _csr_from_rows(m, n, rows, vals)
    # row types: 40 % equality, 30 % >=, 20 % <=, 10 % ranged
    row_type = rng.choice(4, size=m, p=[0.4, 0.3, 0.2, 0.1])
    l_v = np.zeros(n)
    u_v = np.where(rng.random(n) < 0.3, INF, rng.uniform(1.0, 10.0, n))
    return known_optimum(rng, m, n, rp, ci, v, l_v, u_v, frac_at_bound=0.4, y_nonzero=0.5,
                         row_type=row_type, name=f"miplib_like_{m}x{n}_s{seed}")


def multicommodity(seed: int = 0, nodes: int = 200_000, arcs: int = 1_000_000, K: int = 4) -> LP:
    """Node-arc multicommodity flow with joint arc capacities.

    Variables x_{a,k} >= 0 (column a*K + k); rows: flow conservation per
    (node, commodity) as equalities (rows k*nodes + v), then one joint capacity
    row per arc, sum_k x_{a,k} <= cap_a.  Supplies come from a planted flow
    (random routes for each commodity inside cap_a / (2K)), so the LP is
    feasible and balanced.  The optimum is not known in closed form.
    """
    rng = np.random.default_rng(seed)
    perm = rng.permutation(nodes)
    tail = np.empty(arcs, dtype=np.int64)
    head = np.empty(arcs, dtype=np.int64)
    tail[:nodes] = perm
    head[:nodes] = np.roll(perm, -1)          # Hamiltonian cycle: strongly connected
    extra = arcs - nodes
    tail[nodes:] = rng.integers(0, nodes, extra)
    off = rng.integers(1, nodes, extra)
    head[nodes:] = (tail[nodes:] + off) % nodes  # no self loops
    cap = rng.uniform(10.0, 1000.0, arcs)
    cost = rng.uniform(1.0, 100.0, arcs)
    n = arcs * K
    m = nodes * K + arcs
    # planted flow: each arc carries a random amount of each commodity within cap/(2K)
    f = rng.uniform(0.0, 1.0, (arcs, K)) * (cap[:, None] / (2.0 * K))
    f *= (rng.random((arcs, K)) < 0.3)
    supply = np.zeros((K, nodes))
    for k in range(K):
        supply[k] = np.bincount(tail, weights=f[:, k], minlength=nodes) - \
            np.bincount(head, weights=f[:, k], minlength=nodes)
    # CSR assembly: conservation row (k, v) has +1 on arcs leaving v, -1 on arcs entering v
    col_arc = np.arange(arcs)
    entries_r, entries_c, entries_v = [], [], []
    for k in range(K):
        entries_r.append(k * nodes + tail); entries_c.append(col_arc * K + k); entries_v.append(np.ones(arcs))
        entries_r.append(k * nodes + head); entries_c.append(col_arc * K + k); entries_v.append(-np.ones(arcs))
    for k in range(K):
        entries_r.append(nodes * K + col_arc); entries_c.append(col_arc * K + k); entries_v.append(np.ones(arcs))
    R = np.concatenate(entries_r)
    C = np.concatenate(entries_c)
    V = np.concatenate(entries_v)
    order = np.lexsort((C, R))
    R, C, V = R[order], C[order], V[order]
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(R, minlength=m), out=row_ptr[1:])
    l_c = np.concatenate([supply.reshape(-1), np.full(arcs, -INF)])
    u_c = np.concatenate([supply.reshape(-1), cap])
    c = np.repeat(cost, K)
    return LP(m, n, row_ptr, C.astype(np.int32), V.astype(np.float64), c, l_c, u_c,
              np.zeros(n), np.full(n, INF), name=f"mcf_{nodes}n_{arcs}a_{K}k_s{seed}")


def free_and_boxed_mix(seed: int, m: int, n: int, density: float = 0.05) -> LP:
    """Known-optimum LP whose variables mix all four bound patterns
    (free, lower only, upper only, boxed), so every branch of the sets R_j
    is exercised."""
    rng = np.random.default_rng(seed)
    rp, ci, v = random_csr(rng, m, n, density)
    kind = rng.integers(0, 4, n)
    l_v = np.where((kind == 1) | (kind == 3), -rng.uniform(0.0, 2.0, n), -INF)
    u_v = np.where((kind == 2) | (kind == 3), rng.uniform(0.0, 2.0, n), INF)
    return known_optimum(rng, m, n, rp, ci, v, l_v, u_v, frac_at_bound=0.5, y_nonzero=0.5,
                         name=f"mixed_{m}x{n}_s{seed}")


def ragged_rows(seed: int, m: int, n: int) -> LP:
    """Adversarial row-length mix: empty rows, length-1 rows, and one long row."""
    rng = np.random.default_rng(seed)
    lens = rng.choice([0, 1, 1, 2, 3, 5, 8, 17, 33, 70], size=m)
    lens[rng.integers(0, m)] = min(n, 2000)
    rows, vals = [], []
    for i in range(m):
        cols = np.sort(rng.choice(n, size=int(lens[i]), replace=False))
        rows.append(cols)
        vals.append(rng.standard_normal(len(cols)))
    rp, ci, v = _csr_from_rows(m, n, rows, vals)
    lv = np.zeros(n)
    uv = np.where(rng.random(n) < 0.5, INF, rng.uniform(1.0, 3.0, n))
    return known_optimum(rng, m, n, rp, ci, v, lv, uv, name=f"ragged_{m}x{n}_s{seed}")


def bernoulli_csr(rng: np.random.Generator, m: int, n: int, density: float):
    """Bernoulli(density) sparsity over the m x n grid, N(0,1) values, sampled by geometric gaps
    between selected positions in row-major order (exact Bernoulli sampling without drawing
    one uniform per grid cell; columns come out sorted in each row)."""
    total = m * n
    if total == 0 or density <= 0.0:
        return np.zeros(m + 1, np.int64), np.zeros(0, np.int32), np.zeros(0)
    parts, cur = [], -1
    while True:
        k = int(total * density * 1.02) + 64
        pos = cur + np.cumsum(rng.geometric(density, size=k))
        parts.append(pos[pos < total])
        if pos[-1] >= total:
            break
        cur = int(pos[-1])
    pos = np.concatenate(parts)
    rows = pos // n
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=m), out=row_ptr[1:])
    col_idx = (pos - rows * n).astype(np.int32)
    val = rng.standard_normal(len(pos))
    return row_ptr, col_idx, val


def batch_sizes(seed: int, count: int = 512, m_min: int = 100, m_max: int = 20_000) -> np.ndarray:
    """Row counts of the uneven batch: m = floor(exp(U(ln m_min, ln m_max)))."""
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(np.log(m_min), np.log(m_max), count))).astype(np.int64)


def batch_uneven(seed: int, count: int = 512, m_min: int = 100, m_max: int = 20_000,
                 density: float = 0.01) -> list[LP]:
    """Batch of independent LPs of uneven size: m log-uniform in [m_min, m_max], n = 2m,
    Bernoulli(density) N(0,1) matrices, box [0, 1] on every variable, planted optima.
    Instance k draws from its own stream (seed, k), so a prefix of the batch does not depend
    on `count`."""
    ms = batch_sizes(seed, count, m_min, m_max)
    out = []
    for k, m in enumerate(ms.tolist()):
        rng = np.random.default_rng([seed, k])
        n = 2 * m
        rp, ci, v = bernoulli_csr(rng, m, n, density)
        out.append(known_optimum(rng, m, n, rp, ci, v, np.zeros(n), np.ones(n),
                                 frac_at_bound=0.4, y_nonzero=0.5, name=f"batch{seed}_{k}_{m}x{n}"))
    return out


def vertex_lp(seed: int, m: int = 20, n: int = 40, density: float = 0.3) -> LP:
    """LP with a unique, nondegenerate optimal vertex: equality rows A x = b, box [0, 1], exactly
    m variables strictly inside the box (their columns A_F form a well-conditioned square block)
    and n - m at a bound with a nonzero reduced cost; every dual multiplier nonzero.  Built for
    derivatives of the solution with respect to b and the bounds (the active-set KKT system)."""
    rng = np.random.default_rng(seed)
    for _ in range(100):
        mask = rng.random((m, n)) < density
        F = rng.permutation(n)[:m]
        mask[np.arange(m), F] = True  # a nonzero "diagonal" in the free block
        A = np.where(mask, rng.standard_normal((m, n)), 0.0)
        if np.linalg.cond(A[:, F]) < 1e3:
            break
    N = np.setdiff1d(np.arange(n), F)
    x = np.empty(n)
    x[F] = rng.uniform(0.2, 0.8, m)
    at_hi = rng.random(len(N)) < 0.5
    x[N] = np.where(at_hi, 1.0, 0.0)
    r = np.zeros(n)
    r[N] = np.where(at_hi, -1.0, 1.0) * rng.uniform(0.5, 1.5, len(N))
    y = np.where(rng.random(m) < 0.5, 1.0, -1.0) * rng.uniform(0.5, 1.5, m)
    b = A @ x
    c = A.T @ y + r
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(mask.sum(axis=1), out=row_ptr[1:])
    rows, cols = np.nonzero(mask)
    return LP(m, n, row_ptr, cols.astype(np.int32), A[rows, cols].astype(np.float64), c, b.copy(), b.copy(),
              np.zeros(n), np.ones(n), x, y, r, name=f"vertex_{m}x{n}_s{seed}")
