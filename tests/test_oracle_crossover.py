"""Pins of the crossover-lite measurement tool (oracle/crossover.py): the
superbasis's primal superbasics are the fewest any basis allows (brute
force over every column subset of tiny LPs), the constructed optimum of the
200 x 500 face LP has exactly |S| - m = 50 of them, a vertex has none, and
the primal push phase keeps A x = b and the objective, takes one push per
superbasic and ends with every nonbasic column at a bound.  CPU only."""
import itertools

import numpy as np
import pytest

import lpgen
import oracle
from oracle import crossover as X
from tests import vertex_enum as ve


def test_constructed_optimum_has_s_minus_m_superbasics():
    lp = lpgen.small_face_lp(0)
    r = X.crossover_lite(lp, lp["x_star"], lp["y_star"], lp["z_star"])
    assert r["p"] == 250 and r["primal_push_est"] == 50
    assert r["primal_superbasics"] == 50 and r["dual_superbasics"] == 0
    assert r["primal_pushes"] == 50 and r["nonbasic_off_after"] == 0 and r["off_bound_after"] <= lp["m"]
    A = ve.dense(lp)
    assert np.max(np.abs(A @ r["x_after"] - lp["b"])) <= 1e-9
    assert abs(lp["c"] @ r["x_after"] - lp["obj_star"]) <= 1e-9 * (1 + abs(lp["obj_star"]))
    assert np.all(r["x_after"] >= -1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4])
def test_superbasics_are_the_fewest_any_basis_allows(seed):
    # a random point on a random 4 x 10 system: the greedy superbasis leaves
    # out exactly min over all bases B of |P minus B| off-bound columns
    rng = np.random.default_rng(seed)
    m, n = 4, 10
    lp = lpgen.tiny_face_lp(m, n, 4, seed=seed)
    A = ve.dense(lp)
    x = np.where(rng.random(n) < 0.6, rng.uniform(0.2, 1.0, n), 0.0)
    z = np.where(x > 0, 0.0, rng.uniform(0.1, 1.0, n))
    lp = dict(lp, b=A @ x)
    r = X.crossover_lite(lp, x, np.zeros(m), z, push=False)
    off = x > 1e-6
    best = n
    for B in itertools.combinations(range(n), m):
        if np.linalg.matrix_rank(A[:, B]) < m:
            continue
        best = min(best, int(off.sum() - off[list(B)].sum()))
    assert r["primal_superbasics"] == best
    assert r["basis_size"] == m


@pytest.mark.parametrize("seed", [101, 7])
def test_a_vertex_has_no_superbasics(seed):
    lp = lpgen.tiny_face_lp(5, 11, 7, seed=seed)
    A = ve.dense(lp)
    best, verts = ve.optimal_face_vertices(A, lp["b"], lp["c"])
    x, B = verts[0]
    y, z = ve.basis_duals(A, lp["c"], B)
    r = X.crossover_lite(lp, x, y, z)
    assert r["primal_superbasics"] == 0 and r["primal_pushes"] == 0
    assert r["dual_superbasics"] == 0 and r["dual_push_est"] == 0


def test_general_form_push_phase():
    # inequality rows (slack columns) and finite upper bounds: at the
    # constructed optimum every push keeps A_int x - s = b_int and the
    # objective, and ends with the nonbasic columns at a bound
    lp = lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(3), 3)
    r = X.crossover_lite(lp, lp["x_star"], lp["y_star"], lp["z_star"])
    assert r["primal_pushes"] == r["primal_superbasics"] >= r["primal_push_est"]
    assert r["nonbasic_off_after"] == 0 and r["residual_after"] <= 1e-9
    assert abs(lp["c"] @ r["x_after"] - lp["obj_star"]) <= 1e-9 * (1 + abs(lp["obj_star"]))
    xa = r["x_after"]
    assert np.all(xa >= lp["lb"] - 1e-9) and np.all(xa <= lp["ub"] + 1e-9)


@pytest.mark.parametrize("alg", ["averaged", "halpern"])
def test_corner_push_removes_the_pushes(alg):
    # the synthetic analogue of Figure 2: crossover-lite needs |S| - m pushes
    # from the phase-1 point; from Algorithm 1's result none with the Halpern
    # loop (its corner phase returns a projected point, T(z)), while the
    # averaged loop's returned average keeps columns a little off the bounds
    # its reduced costs ask for, which the push phase still has to move
    lp = lpgen.small_face_lp(0)
    r1 = oracle.solve(lp, dict(algorithm=alg))
    x1, y1, z1 = oracle.unscale(r1["model"], r1["x_hat"], r1["y_hat"])
    before = X.crossover_lite(lp, x1, y1, z1)
    rc = oracle.corner_phase(r1, dict(obj_seed=1))
    xc, _, _ = oracle.unscale(r1["model"], rc["x_hat"], rc["y_hat"])
    after = X.crossover_lite(lp, xc, y1, z1)
    assert before["primal_pushes"] == 50
    if alg == "halpern":
        assert after["primal_pushes"] == 0
    else:
        assert after["primal_pushes"] < before["primal_pushes"]
