"""Brute-force vertex enumeration for tiny canonical LPs (test helper).

For min c'x s.t. Ax = b, x >= 0 with m <= 6 and n <= 12, every vertex is a
basic feasible solution: a set B of m columns with A_B nonsingular and
x_B = A_B^{-1} b >= 0, x_N = 0 (Section 2.1: basis, basic solution).  All
C(n, m) bases are tried.
"""
import itertools

import numpy as np


def dense(lp):
    A = np.zeros((lp["m"], lp["n"]))
    for i in range(lp["m"]):
        for k in range(lp["row_ptr"][i], lp["row_ptr"][i + 1]):
            A[i, lp["col_idx"][k]] += lp["val"][k]
    return A


def vertices(A, b, feas_tol=1e-12, cond_max=1e10):
    m, n = A.shape
    found = []
    for B in itertools.combinations(range(n), m):
        AB = A[:, B]
        if np.linalg.cond(AB) > cond_max:
            continue
        xB = np.linalg.solve(AB, b)
        if np.all(xB >= -feas_tol):
            x = np.zeros(n)
            x[list(B)] = np.maximum(xB, 0.0)
            found.append((x, B))
    uniq = []
    for x, B in found:
        if not any(np.max(np.abs(x - v)) <= 1e-9 for v, _ in uniq):
            uniq.append((x, B))
    return uniq


def optimal_face_vertices(A, b, c, rel=1e-9):
    vs = vertices(A, b)
    objs = np.array([c @ v for v, _ in vs])
    best = objs.min()
    keep = objs <= best + rel * (1.0 + abs(best))
    return best, [vs[i] for i in np.nonzero(keep)[0]]


def basis_duals(A, c, B):
    """y = A_B^{-T} c_B and z = c - A'y of a basis (Section 2.1)."""
    AB = A[:, list(B)]
    y = np.linalg.solve(AB.T, c[list(B)])
    return y, c - A.T @ y
