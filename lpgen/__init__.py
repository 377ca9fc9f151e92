"""Seeded synthetic LP generators.

This module holds no arithmetic of the PDHG method: it only draws random sparse
LPs whose optimal face is known by construction, in the shapes of the paper's
target class (LPs with many more variables strictly between their bounds than
rows, Section 4.2).  Both the CUDA path and the CPU oracle receive the arrays it
returns; neither is imported here.

Every generator takes an integer seed and uses numpy's PCG64 stream, so one
seed gives one LP on one numpy version.  The seed convention for the named
workloads is ``base_seed + workload_id * 1_000_000 + lp_index``.

An LP is returned as a dict:
  m, n           rows and columns
  row_ptr        int64[m+1]   CSR row pointers of A
  col_idx        int32[nnz]   CSR column indices (sorted within a row)
  val            float64[nnz] CSR values
  b              float64[m]
  c              float64[n]
  lb, ub         float64[n]   bounds, +-inf allowed
  sense          int8[m]      ord('='), ord('<') or ord('>')
  x_star, y_star, z_star      a known optimal triple (when constructed)
  obj_star       c @ x_star (the optimal value, when constructed)
  name           workload name
"""
from __future__ import annotations

import math

import numpy as np

EQ, LE, GE = ord("="), ord("<"), ord(">")

WORKLOAD_SEED_STRIDE = 1_000_000


def workload_seed(base_seed: int, workload_id: int, lp_index: int = 0) -> int:
    return int(base_seed) + int(workload_id) * WORKLOAD_SEED_STRIDE + int(lp_index)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _distinct_rows(rng, col_counts: np.ndarray, m: int):
    """Draw, for every column j, col_counts[j] distinct row indices uniformly
    from [0, m).  Returns (rows, cols) sorted by (col, row)."""
    n = col_counts.shape[0]
    cols = np.repeat(np.arange(n, dtype=np.int64), col_counts)
    rows = rng.integers(0, m, size=cols.shape[0], dtype=np.int64)
    while True:
        key = cols * m + rows
        order = np.argsort(key, kind="stable")
        cols, rows, key = cols[order], rows[order], key[order]
        dup = np.zeros(key.shape[0], dtype=bool)
        dup[1:] = key[1:] == key[:-1]
        ndup = int(dup.sum())
        if ndup == 0:
            return rows, cols
        rows[dup] = rng.integers(0, m, size=ndup, dtype=np.int64)


def _csr_from_coo(m: int, n: int, rows, cols, vals):
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    counts = np.bincount(rows, minlength=m)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, cols.astype(np.int32), vals.astype(np.float64)


def csr_matvec(row_ptr, col_idx, val, x):
    """Plain CSR product used only to build right-hand sides (b = A x*)."""
    m = row_ptr.shape[0] - 1
    rows = np.repeat(np.arange(m), np.diff(row_ptr))
    out = np.zeros(m, dtype=np.float64)
    np.add.at(out, rows, val * x[col_idx])
    return out


def csr_rmatvec(row_ptr, col_idx, val, y, n):
    """Plain CSR transpose product used only to build objectives (c = A^T y*)."""
    m = row_ptr.shape[0] - 1
    rows = np.repeat(np.arange(m), np.diff(row_ptr))
    out = np.zeros(n, dtype=np.float64)
    np.add.at(out, col_idx, val * y[rows])
    return out


def random_face_lp(m: int, n: int, support: int, seed: int, col_nnz=5, name="random_face",
                   col_nnz_range=None):
    """Random sparse LP in canonical form (all '=' rows, x >= 0) with a
    degenerate optimal face of dimension >= support - m.

    Each column j draws col_nnz distinct rows uniformly (or, with
    col_nnz_range=(lo, hi), a count uniform in lo..hi per column), values
    N(0, 1); the matrix is redrawn if a row stays empty.  S is a uniform subset
    of |S| = support columns; x*_S ~ U(0.1, 1), x*_{not S} = 0; y* ~ N(0, 1);
    z*_S = 0, z*_{not S} ~ U(0.1, 1); b = A x*, c = A^T y* + z*.
    """
    rng = _rng(seed)
    while True:
        if col_nnz_range is None:
            counts = np.full(n, min(int(col_nnz), m), dtype=np.int64)
        else:
            lo, hi = col_nnz_range
            counts = rng.integers(lo, hi + 1, size=n, dtype=np.int64)
            counts = np.minimum(counts, m)
        rows, cols = _distinct_rows(rng, counts, m)
        if np.unique(rows).shape[0] == m:
            break
    vals = rng.standard_normal(rows.shape[0])
    row_ptr, col_idx, val = _csr_from_coo(m, n, rows, cols, vals)
    S = np.sort(rng.choice(n, size=support, replace=False))
    x_star = np.zeros(n)
    x_star[S] = rng.uniform(0.1, 1.0, size=support)
    y_star = rng.standard_normal(m)
    z_star = rng.uniform(0.1, 1.0, size=n)
    z_star[S] = 0.0
    b = csr_matvec(row_ptr, col_idx, val, x_star)
    c = csr_rmatvec(row_ptr, col_idx, val, y_star, n) + z_star
    return dict(name=name, m=m, n=n, row_ptr=row_ptr, col_idx=col_idx, val=val, b=b, c=c,
                lb=np.zeros(n), ub=np.full(n, np.inf), sense=np.full(m, EQ, dtype=np.int8),
                x_star=x_star, y_star=y_star, z_star=z_star, obj_star=float(c @ x_star),
                support=S)


def dense_line_lp(m: int, n: int, row_len: int, col_len: int, extra_support: int, seed: int, col_nnz=3):
    """Random-face LP (canonical form, constructed optimum as in random_face_lp)
    whose pattern adds one dense row and one dense column: column 0 gets
    col_len distinct rows and row 0 gets row_len distinct columns, on top of
    col_nnz rows per column.  With row_len and col_len above 4096 both A and
    A^T have a row that the one-CTA-per-row path of the SpMV handles."""
    rng = _rng(seed)
    counts = np.full(n, min(int(col_nnz), m), dtype=np.int64)
    counts[0] = min(int(col_len), m)
    while True:
        rows, cols = _distinct_rows(rng, counts, m)
        if np.unique(rows).shape[0] == m:
            break
    dense_cols = np.sort(rng.choice(n, size=min(int(row_len), n), replace=False))
    have0 = set(cols[rows == 0].tolist())
    add = np.array([j for j in dense_cols if j not in have0], dtype=np.int64)
    rows = np.concatenate([rows, np.zeros(add.shape[0], dtype=np.int64)])
    cols = np.concatenate([cols, add])
    vals = rng.standard_normal(rows.shape[0])
    row_ptr, col_idx, val = _csr_from_coo(m, n, rows, cols, vals)
    support = m + extra_support
    S = np.sort(rng.choice(n, size=support, replace=False))
    x_star = np.zeros(n)
    x_star[S] = rng.uniform(0.1, 1.0, size=support)
    y_star = rng.standard_normal(m)
    z_star = rng.uniform(0.1, 1.0, size=n)
    z_star[S] = 0.0
    b = csr_matvec(row_ptr, col_idx, val, x_star)
    c = csr_rmatvec(row_ptr, col_idx, val, y_star, n) + z_star
    return dict(name=f"dense_line_m{m}_n{n}", m=m, n=n, row_ptr=row_ptr, col_idx=col_idx, val=val, b=b,
                c=c, lb=np.zeros(n), ub=np.full(n, np.inf), sense=np.full(m, EQ, dtype=np.int8),
                x_star=x_star, y_star=y_star, z_star=z_star, obj_star=float(c @ x_star), support=S)


def small_face_lp(seed: int, base_seed: int = 0):
    """200 x 500, 5 nnz per column, |S| = 250 (face dimension >= 50)."""
    return random_face_lp(200, 500, 250, workload_seed(base_seed, 0, seed), 5,
                          name="random_face_m200_n500")


def _power_law_counts(rng, n, kmax, mean, forced_max=True):
    k = np.arange(1, kmax + 1, dtype=np.float64)

    def mean_of(alpha):
        w = k ** (-alpha)
        return float((k * w).sum() / w.sum())

    lo, hi = 1.0, 3.0  # mean_of is decreasing in alpha
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        if mean_of(mid) > mean:
            lo = mid
        else:
            hi = mid
    alpha = 0.5 * (lo + hi)
    p = k ** (-alpha)
    p /= p.sum()
    counts = rng.choice(np.arange(1, kmax + 1), size=n, p=p).astype(np.int64)
    if forced_max:
        counts[rng.integers(0, n)] = kmax
    return counts, alpha


def power_law_lp(m: int, n: int, extra_support: int, seed: int, kmax=2000, mean=8.0,
                 name=None):
    """General-form LP with skewed columns, inequality rows and upper bounds.

    Column nnz follows P(k) ~ k^-alpha on 1..kmax with alpha set by bisection
    so that the mean is `mean`, and one column is forced to kmax.  Rows uniform
    without replacement, values N(0, 1).  Rows [0, m/2) are '=', the rest '<'.
    20% of the columns get u_j ~ U(1, 10) (l = 0 everywhere).  The optimum is
    constructed: |S| = m + extra_support columns strictly inside their bounds
    (x*_S ~ U(0.1, 0.9), z*_S = 0); bounded columns off S sit at u (z* < 0) or
    at 0 (z* > 0) with equal odds; other columns sit at 0 with z* ~ U(0.1, 1).
    '=' rows get y* ~ N(0, 1); half the '<' rows are active (b = (A x*)_i,
    y* = -|N(0, 1)|), half inactive (b = (A x*)_i + U(0.1, 1), y* = 0).
    c = A^T y* + z*.
    """
    rng = _rng(seed)
    counts, alpha = _power_law_counts(rng, n, min(kmax, m), mean)
    while True:
        rows, cols = _distinct_rows(rng, counts, m)
        present = np.zeros(m, dtype=bool)
        present[rows] = True
        if present.all():
            break
        # give every empty row one entry in a random column that lacks it
        empty = np.nonzero(~present)[0]
        extra_cols = rng.integers(0, n, size=empty.shape[0])
        np.add.at(counts, extra_cols, 1)
    vals = rng.standard_normal(rows.shape[0])
    row_ptr, col_idx, val = _csr_from_coo(m, n, rows, cols, vals)

    sense = np.full(m, EQ, dtype=np.int8)
    sense[m // 2:] = LE
    lb = np.zeros(n)
    ub = np.full(n, np.inf)
    bounded = rng.random(n) < 0.2
    ub[bounded] = rng.uniform(1.0, 10.0, size=int(bounded.sum()))

    support = m + extra_support
    S = np.sort(rng.choice(n, size=support, replace=False))
    inS = np.zeros(n, dtype=bool)
    inS[S] = True
    x_star = np.zeros(n)
    z_star = np.zeros(n)
    x_star[S] = rng.uniform(0.1, 0.9, size=support)
    off = ~inS
    at_upper = off & bounded & (rng.random(n) < 0.5)
    at_lower = off & ~at_upper
    x_star[at_upper] = ub[at_upper]
    z_star[at_upper] = -rng.uniform(0.1, 1.0, size=int(at_upper.sum()))
    z_star[at_lower] = rng.uniform(0.1, 1.0, size=int(at_lower.sum()))

    y_star = np.zeros(m)
    y_star[: m // 2] = rng.standard_normal(m // 2)
    ineq = np.arange(m // 2, m)
    active = rng.random(ineq.shape[0]) < 0.5
    ax = csr_matvec(row_ptr, col_idx, val, x_star)
    b = ax.copy()
    y_star[ineq[active]] = -np.abs(rng.standard_normal(int(active.sum())))
    inactive = ineq[~active]
    b[inactive] = ax[inactive] + rng.uniform(0.1, 1.0, size=inactive.shape[0])
    c = csr_rmatvec(row_ptr, col_idx, val, y_star, n) + z_star
    return dict(name=name or f"power_law_m{m}_n{n}", m=m, n=n, row_ptr=row_ptr, col_idx=col_idx,
                val=val, b=b, c=c, lb=lb, ub=ub, sense=sense, x_star=x_star, y_star=y_star,
                z_star=z_star, obj_star=float(c @ x_star), support=S, alpha=alpha)


def large_power_law_lp(seed: int = 0, base_seed: int = 0):
    """100k x 400k, power-law columns (mean 8, max 2000), |S| = m + 5000."""
    return power_law_lp(100_000, 400_000, 5_000, workload_seed(base_seed, 1, seed),
                        name="power_law_m100k_n400k")


def guidance_lp(seed: int, base_seed: int = 0):
    """20k x 80k with the power-law construction, |S| = m + 1000."""
    return power_law_lp(20_000, 80_000, 1_000, workload_seed(base_seed, 4, seed),
                        name="power_law_m20k_n80k")


def transportation_lp(sources: int, sinks: int, seed: int, name=None):
    """Balanced transportation LP.  Column j = i*sinks + k ships from source i
    to sink k: +1 in row i and +1 in row sources + k.  Supplies and demands
    ~ U{1..100}; while the totals differ, one step alternates between
    decrementing a random entry (> 1) on the larger side and incrementing a
    random entry (< 100) on the smaller side.  Costs ~ U{1..10}; x >= 0; all
    rows '='.  The constraint matrix has rank m - 1."""
    rng = _rng(seed)
    s = rng.integers(1, 101, size=sources)
    d = rng.integers(1, 101, size=sinks)
    step = 0
    while s.sum() != d.sum():
        big, small = (s, d) if s.sum() > d.sum() else (d, s)
        if step % 2 == 0:
            cand = np.nonzero(big > 1)[0]
            if cand.shape[0]:
                big[cand[rng.integers(0, cand.shape[0])]] -= 1
        else:
            cand = np.nonzero(small < 100)[0]
            if cand.shape[0]:
                small[cand[rng.integers(0, cand.shape[0])]] += 1
        step += 1
    m = sources + sinks
    n = sources * sinks
    # row i (source): columns i*sinks .. i*sinks+sinks-1 ; row sources+k: columns k, sinks+k, ...
    src_cols = np.arange(n, dtype=np.int64)
    sink_cols = np.arange(n, dtype=np.int64).reshape(sources, sinks).T.reshape(-1)
    col_idx = np.concatenate([src_cols, sink_cols]).astype(np.int32)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    row_ptr[1:sources + 1] = np.arange(1, sources + 1) * sinks
    row_ptr[sources + 1:] = n + np.arange(1, sinks + 1) * sources
    val = np.ones(2 * n)
    b = np.concatenate([s, d]).astype(np.float64)
    c = rng.integers(1, 11, size=n).astype(np.float64)
    return dict(name=name or f"transportation_{sources}x{sinks}", m=m, n=n, row_ptr=row_ptr,
                col_idx=col_idx, val=val, b=b, c=c, lb=np.zeros(n), ub=np.full(n, np.inf),
                sense=np.full(m, EQ, dtype=np.int8), supply=s, demand=d)


def large_transportation_lp(seed: int = 0, base_seed: int = 0):
    """1000 sources x 2000 sinks (m = 3000, n = 2M, nnz = 4M)."""
    return transportation_lp(1000, 2000, workload_seed(base_seed, 2, seed),
                             name="transportation_1000x2000")


def batch_lp(i: int, base_seed: int = 0, m_range=(50, 5000)):
    """LP i of the batch workload: the random-face construction with
    m ~ U{m_range}, n = round(r m), r ~ U(2, 4), column nnz ~ U{3..12},
    |S| = m + ceil(m / 4)."""
    seed = workload_seed(base_seed, 3, i)
    rng = _rng(seed)
    m = int(rng.integers(m_range[0], m_range[1] + 1))
    n = int(round(rng.uniform(2.0, 4.0) * m))
    support = m + int(math.ceil(0.25 * m))
    return random_face_lp(m, n, support, seed + 7919 * WORKLOAD_SEED_STRIDE,
                          col_nnz_range=(3, 12), name=f"batch_{i}")


def batch_lps(count: int = 512, base_seed: int = 0, m_range=(50, 5000)):
    """`count` LPs of the batch workload (batch_lp 0 .. count-1)."""
    return [batch_lp(i, base_seed, m_range) for i in range(count)]


def tiny_face_lp(m: int, n: int, support: int, seed: int, col_nnz=3):
    """Tiny degenerate LP (m <= 6, n <= 12) for brute-force vertex enumeration."""
    return random_face_lp(m, n, support, seed, col_nnz, name=f"tiny_{m}x{n}")


def with_bounds_and_inequalities(lp: dict, seed: int):
    """Variant of a constructed LP that exercises '<', '>' rows and finite
    upper bounds while keeping a known optimum: every third row becomes '<'
    or '>' (active, y* keeps a dual-feasible sign, or inactive with y* = 0 and a
    slack), and 30% of columns get u_j = x*_j + U(0.5, 2) (inactive, z* kept)
    or, when x*_j = 0 and z*_j > 0, are flipped to sit at a finite upper bound
    with z*_j < 0."""
    rng = _rng(seed)
    m, n = lp["m"], lp["n"]
    out = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in lp.items()}
    row_ptr, col_idx, val = out["row_ptr"], out["col_idx"], out["val"]
    y = out["y_star"]
    z = out["z_star"]
    x = out["x_star"]
    sense = out["sense"]
    ub = out["ub"]
    cols = rng.random(n) < 0.3
    flip = cols & (x == 0) & (rng.random(n) < 0.5)
    keep = cols & ~flip
    ub[keep] = x[keep] + rng.uniform(0.5, 2.0, size=int(keep.sum()))
    ub[flip] = rng.uniform(0.2, 1.0, size=int(flip.sum()))
    x[flip] = ub[flip]
    z[flip] = -np.abs(z[flip])
    ax = csr_matvec(row_ptr, col_idx, val, x)
    b = ax.copy()
    for i in range(0, m, 3):
        kind = rng.integers(0, 4)
        if kind == 0:      # active '<': y <= 0
            sense[i] = LE
            y[i] = -abs(y[i])
        elif kind == 1:    # active '>': y >= 0
            sense[i] = GE
            y[i] = abs(y[i])
        elif kind == 2:    # inactive '<'
            sense[i] = LE
            y[i] = 0.0
            b[i] = ax[i] + rng.uniform(0.1, 1.0)
        else:              # inactive '>'
            sense[i] = GE
            y[i] = 0.0
            b[i] = ax[i] - rng.uniform(0.1, 1.0)
    out["b"] = b
    out["c"] = csr_rmatvec(row_ptr, col_idx, val, y, n) + z
    out["obj_star"] = float(out["c"] @ x)
    out["name"] = lp["name"] + "_bounded"
    return out
