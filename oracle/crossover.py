"""Crossover-lite: basis construction and the primal push phase of Section
2.1, as a CPU measurement tool (TEST AND MEASUREMENT INFRASTRUCTURE).

Only the tests and the benchmark use this module; the product has no
crossover (the sequential CPU step stays outside it).  It turns the
corner measure into actual push counts: from a point (x, y, z) it builds a
superbasis and counts the primal and dual superbasics, then runs the primal
push phase, one push per primal superbasic, to a basic solution.  Dense
linear algebra: for LPs with up to a few thousand rows.

The standard form is the user's model with one slack per inequality row:
A_int x - s = b_int, s >= 0 on the internal '>' rows (a '<' row negated),
bounds l <= x <= u.  A column is "off bound" when it is more than tol from
each finite bound (a free column always is), and has a "zero reduced cost"
when |z_j| <= tol (a slack's reduced cost is its row's dual).

Basis construction (Section 2.1: include as many off-bound columns and as
many zero-reduced-cost columns as possible): columns in the priority order
  1. off bound with zero reduced cost,  2. off bound,  3. zero reduced cost,
  4. the rest (slacks first, then structurals),
each added when it is linearly independent of the columns already taken
(Gram-Schmidt residual above 1e-9 of its norm), until m are taken.  Greedy
selection by this order takes a maximal independent subset of each class in
turn, so the off-bound columns left out number |P| - rank(A_P), the least
any basis allows.  Primal superbasics: nonbasic columns off bound; dual
superbasics: basic columns with a nonzero reduced cost.

Primal push (Section 2.1): each primal superbasic j in turn moves toward
its nearer finite bound (a free one toward 0) along the direction that
keeps A x = b with the basic variables adjusting; the ratio test stops it at
its bound or when a basic variable reaches one of its bounds, which then
leaves the basis for j (one pivot).  One push per superbasic.
"""
from __future__ import annotations

import numpy as np

from . import pdhg as P


def standard_form(lp):
    """(A_std, b_std, l_std, u_std, n_struct): the internal form with one
    slack column -e_i per inequality row (dense)."""
    m, n = int(lp["m"]), int(lp["n"])
    A = P.csr_matrix(lp).toarray()
    sense = np.asarray(lp.get("sense", np.full(m, P.EQ)), dtype=np.int64)
    sign = np.where(sense == P.LE, -1.0, 1.0)
    A_int = sign[:, None] * A
    b_int = sign * np.asarray(lp["b"], dtype=np.float64)
    ineq = np.nonzero(sense != P.EQ)[0]
    S = np.zeros((m, len(ineq)))
    S[ineq, np.arange(len(ineq))] = -1.0
    l = np.asarray(lp["lb"], dtype=np.float64) if lp.get("lb") is not None else np.zeros(n)
    u = np.asarray(lp["ub"], dtype=np.float64) if lp.get("ub") is not None else np.full(n, np.inf)
    A_std = np.hstack([A_int, S])
    l_std = np.concatenate([l, np.zeros(len(ineq))])
    u_std = np.concatenate([u, np.full(len(ineq), np.inf)])
    return A_std, b_int, l_std, u_std, n, ineq, sign


def standard_point(lp, x, y, z):
    """The standard-form point of a user (x, y, z): slacks s = A_int x -
    b_int on the inequality rows, and their reduced costs = the internal
    duals of those rows."""
    A_std, b_int, l_std, u_std, n, ineq, sign = standard_form(lp)
    A_int = A_std[:, :n]
    y_int = sign * np.asarray(y, dtype=np.float64)
    s = A_int[ineq] @ x - b_int[ineq]
    return np.concatenate([x, s]), np.concatenate([z, y_int[ineq]])


def classify(xs, zs, l, u, tol):
    """(off_bound, zero_rc) masks of the standard-form columns."""
    dl = np.where(np.isfinite(l), xs - l, np.inf)
    du = np.where(np.isfinite(u), u - xs, np.inf)
    off = (dl > tol) & (du > tol)
    zero = np.abs(zs) <= tol
    return off, zero


def build_superbasis(A, off, zero, n_struct, indep_tol=1e-9):
    """Greedy basis construction in the priority order of the module
    docstring; returns the basic column indices (at most m: fewer when A
    has rank < m)."""
    m, N = A.shape
    idx = np.arange(N)
    slack_first = np.concatenate([idx[n_struct:], idx[:n_struct]])
    rest_mask = ~off & ~zero
    order = np.concatenate([idx[off & zero], idx[off & ~zero], idx[~off & zero],
                            slack_first[rest_mask[slack_first]]])
    Q = np.zeros((m, 0))
    basis = []
    for j in order:
        if len(basis) == m:
            break
        a = A[:, j]
        na = np.linalg.norm(a)
        if na == 0.0:
            continue
        r = a - Q @ (Q.T @ a)
        r = r - Q @ (Q.T @ r)  # a second pass keeps Q orthonormal
        nr = np.linalg.norm(r)
        if nr > indep_tol * na:
            Q = np.hstack([Q, (r / nr)[:, None]])
            basis.append(int(j))
    return basis


def primal_push(A, xs, l, u, basis, off, tol, max_pushes=None):
    """The primal push phase from the superbasis: returns (x, basis,
    pushes, pivots).  x keeps A x unchanged; every nonbasic column ends at a
    bound (or at 0 when free)."""
    x = xs.astype(np.float64).copy()
    B = list(basis)
    inB = np.zeros(A.shape[1], dtype=bool)
    inB[B] = True
    supers = [j for j in np.nonzero(off & ~inB)[0]]
    pushes = pivots = 0
    for j in supers:
        if max_pushes is not None and pushes >= max_pushes:
            break
        if inB[j]:
            continue
        # target: the nearer finite bound (0 for a free column)
        cand = [v for v in (l[j], u[j]) if np.isfinite(v)]
        target = min(cand, key=lambda v: abs(v - x[j])) if cand else 0.0
        step = target - x[j]
        if step == 0.0:
            continue
        AB = A[:, B]
        # basic change per unit move of x_j: AB d = -A_j
        d, *_ = np.linalg.lstsq(AB, -A[:, j], rcond=None)
        d = d * np.sign(step)
        t_max = abs(step)
        leave = -1
        for k, b in enumerate(B):
            if d[k] < -1e-12 and np.isfinite(l[b]):
                t = (x[b] - l[b]) / -d[k]
            elif d[k] > 1e-12 and np.isfinite(u[b]):
                t = (u[b] - x[b]) / d[k]
            else:
                continue
            if t < t_max:
                t_max, leave = max(t, 0.0), k
        x[j] += np.sign(step) * t_max
        x[B] += t_max * d
        pushes += 1
        if leave >= 0:
            out = B[leave]
            # the leaving variable sits at the bound it reached
            x[out] = l[out] if d[leave] < 0 else u[out]
            inB[out] = False
            B[leave] = int(j)
            inB[j] = True
            pivots += 1
        else:
            x[j] = target
    return x, B, pushes, pivots


def crossover_lite(lp, x, y, z, tol=P.METRIC_TOL, push=True, max_pushes=None):
    """Superbasis counts and the primal push phase for a user-space point
    (x, y, z); returns a dict: p, d (off-bound and zero-reduced-cost counts,
    slacks included), the Section 2.1 estimates max(0, p - m) and
    max(0, m - d), the constructed superbasis's primal and dual superbasics,
    and (push=True) the pushes and pivots of the primal push phase and the
    number of columns off bound afterwards."""
    A, b, l, u, n, ineq, sign = standard_form(lp)
    m = A.shape[0]
    xs, zs = standard_point(lp, x, y, z)
    off, zero = classify(xs, zs, l, u, tol)
    basis = build_superbasis(A, off, zero, n)
    inB = np.zeros(A.shape[1], dtype=bool)
    inB[basis] = True
    out = dict(m=m, p=int(off.sum()), d=int(zero.sum()),
               primal_push_est=max(0, int(off.sum()) - m), dual_push_est=max(0, m - int(zero.sum())),
               basis_size=len(basis),
               primal_superbasics=int((off & ~inB).sum()), dual_superbasics=int((inB & ~zero).sum()))
    if push:
        x2, B2, pushes, pivots = primal_push(A, xs, l, u, basis, off, tol, max_pushes)
        off2, _ = classify(x2, zs, l, u, tol)
        inB2 = np.zeros(A.shape[1], dtype=bool)
        inB2[B2] = True
        out.update(primal_pushes=pushes, pivots=pivots, off_bound_after=int(off2.sum()),
                   nonbasic_off_after=int((off2 & ~inB2).sum()),
                   residual_after=float(np.linalg.norm(A @ x2 - b)), x_after=x2[:n])
    return out
