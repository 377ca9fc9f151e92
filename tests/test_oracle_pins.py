"""Pins of the CPU oracle to facts outside itself (no GPU).

Each test checks the oracle against something the paper or the mathematics
fixes: published generator outputs, closed forms, textbook invariants,
brute-force vertex enumeration, optima known by construction, scipy's HiGHS,
and the optimality conditions of Section 2.
"""
import math
import os

import numpy as np
import pytest
import scipy.optimize
import scipy.sparse as sp

import lpgen
import oracle
from tests import vertex_enum as ve

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden_ints(name):
    vals, seed = [], None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("seed"):
                seed = int(line.split()[1])
            else:
                vals.append(int(line))
    return seed, vals


# --------------------------------------------------------------------------
# Random objective of Algorithm 1
# --------------------------------------------------------------------------

def test_splitmix64_matches_published_vector():
    seed, expect = _read_golden_ints("splitmix64_seed1234567.txt")
    got = [int(v) for v in oracle.splitmix64(seed, len(expect))]
    assert got == expect


def test_uniform_is_53bit_in_unit_interval():
    u = oracle.splitmix64_uniform(7, 100_000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all(u * 2.0 ** 53 == np.floor(u * 2.0 ** 53))
    assert abs(u.mean() - 0.5) < 5e-3 and abs(u.var() - 1.0 / 12) < 2e-3
    # counter-based: element j depends only on (seed, j)
    assert np.array_equal(oracle.splitmix64_uniform(7, 10), u[:10])


# --------------------------------------------------------------------------
# Projections (Section 2: bounds handled implicitly)
# --------------------------------------------------------------------------

def test_projections_special_cases():
    inf = np.inf
    l = np.array([0.0, -inf, -1.0, -inf, 2.0])
    u = np.array([inf, 3.0, 1.0, inf, 2.0])
    x = np.array([-5.0, 7.0, 0.25, 11.0, 9.0])
    assert np.array_equal(oracle.project_box(x, l, u), [0.0, 3.0, 0.25, 11.0, 2.0])
    lam = np.array([-2.0, 2.0, -0.5, 4.0, -3.0])
    # only l finite -> z >= 0; only u finite -> z <= 0; both -> lam; free -> 0
    assert np.array_equal(oracle.project_dual_cone(lam, l, u), [0.0, 0.0, -0.5, 0.0, -3.0])
    r = oracle.primal_residual(np.array([1.0, 1.0]), np.array([3.0, 3.0]), np.array([False, True]))
    assert np.array_equal(r, [-2.0, 0.0])


# --------------------------------------------------------------------------
# Scaling and step size
# --------------------------------------------------------------------------

def test_ruiz_equilibrates_rows_and_columns():
    # Ruiz (2001): the infinity-norm equilibration converges to row and column
    # maxima of 1, the log-deviation shrinking about 2x per pass.
    lp = lpgen.small_face_lp(3)
    A = oracle.pdhg.csr_matrix(lp)

    def deviation(passes):
        Dr, Dc = oracle.ruiz_pock_chambolle(A, passes, pock_chambolle=False)
        S = abs(sp.diags(Dr) @ A @ sp.diags(Dc))
        rows = S.max(axis=1).toarray().ravel()
        cols = S.max(axis=0).toarray().ravel()
        return max(np.max(np.abs(np.log(rows))), np.max(np.abs(np.log(cols))))

    d0, d10, d20 = deviation(0), deviation(10), deviation(20)
    assert d10 <= 5e-3 and d10 <= d0 * 2.0 ** -6
    assert d20 <= d10 * 2.0 ** -6


def test_pock_chambolle_norm_bound():
    # Pock & Chambolle (2011), Lemma 2 with alpha = 1: the scaled matrix has
    # spectral norm <= 1, whatever the input matrix.
    rng = np.random.default_rng(5)
    for trial in range(4):
        A = sp.random(40, 90, density=0.1, random_state=trial, data_rvs=rng.standard_normal).tocsr()
        A = A + sp.eye(40, 90)  # no empty rows
        Dr, Dc = oracle.ruiz_pock_chambolle(A.tocsr(), 10)
        Ah = (sp.diags(Dr) @ A @ sp.diags(Dc)).toarray()
        s = np.linalg.svd(Ah, compute_uv=False)[0]
        assert s <= 1.0 + 1e-12
        assert s > 0.3


def test_empty_row_and_column_keep_unit_scale():
    A = sp.csr_matrix(np.array([[2.0, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 8.0]]))
    Dr, Dc = oracle.ruiz_pock_chambolle(A, 10)
    assert Dr[1] == 1.0 and Dc[1] == 1.0


def test_power_iteration_against_svd():
    lp = lpgen.small_face_lp(1)
    model = oracle.Model(lp)
    s_pi = oracle.power_iteration(model.Ahat, model.AhatT, 100)
    sv = np.linalg.svd(model.Ahat.toarray(), compute_uv=False)
    # power iteration converges like (s2/s1)^(2k); the bound below is that rate
    rate = (sv[1] / sv[0]) ** 200
    assert abs(s_pi - sv[0]) / sv[0] <= max(1e-12, 2 * rate) + 1e-6
    # exact on a diagonal matrix with a spectral gap
    D = sp.diags([3.0, 2.0, 1.0]).tocsr()
    assert abs(oracle.power_iteration(D, D.T.tocsr(), 100) - 3.0) < 1e-14


# --------------------------------------------------------------------------
# The PDHG map: closed form of the 1x1 affine recurrence
# --------------------------------------------------------------------------

def test_pdhg_step_matches_closed_form_1x1():
    # min c x s.t. a x = b, -10 <= x <= 10 with a = 1: scaling is the identity,
    # the solution (x*, y*) = (b, c) is interior, so the PDHG map is affine:
    #   e_x' = e_x + tau a e_y,  e_y' = e_y - sigma a (e_x + 2 tau a e_y)
    # and the k-th error is M^k e_0 (computed from M's eigen-decomposition).
    b, c = 0.7, 0.3
    lp = dict(m=1, n=1, row_ptr=np.array([0, 1]), col_idx=np.array([0], dtype=np.int32),
              val=np.array([1.0]), b=np.array([b]), c=np.array([c]),
              lb=np.array([-10.0]), ub=np.array([10.0]), sense=np.array([oracle.EQ], dtype=np.int8))
    model, p, sigma_max, eta = oracle.setup(lp)
    assert model.Dr[0] == 1.0 and model.Dc[0] == 1.0 and sigma_max == 1.0
    s = oracle.State(model, np.array([0.0]), np.array([0.0]), eta, oracle.initial_omega(model))
    tau, sig = s.tau, s.sigma
    M = np.array([[1.0, tau], [-sig, 1.0 - 2.0 * sig * tau]])
    w, V = np.linalg.eig(M)
    e0 = np.array([0.0 - b, 0.0 - c])
    xs = [s.x[0]]
    for k in range(1, 6):
        oracle.pdhg_step(model, s)
        ek = (V @ np.diag(w ** k) @ np.linalg.solve(V, e0)).real
        assert abs(s.x[0] - (b + ek[0])) < 1e-13
        assert abs(s.y[0] - (c + ek[1])) < 1e-13
        xs.append(s.x[0])
    # uniform average of the iterates since the (initial) restart
    xa, _ = s.average()
    assert abs(xa[0] - np.mean(xs[1:])) < 1e-15


def test_projection_active_in_step():
    # x must stay in [l, u] every iteration (Section 2 implicit bounds)
    lp = lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(2), 11)
    model, p, _, eta = oracle.setup(lp)
    s = oracle.State(model, oracle.project_box(np.zeros(model.n), model.lhat, model.uhat),
                     np.zeros(model.m), eta, oracle.initial_omega(model))
    for _ in range(50):
        oracle.pdhg_step(model, s)
        assert np.all(s.x >= model.lhat) and np.all(s.x <= model.uhat)
        assert np.all(s.y[model.ge] >= 0.0)


# --------------------------------------------------------------------------
# KKT quantities against Section 2's definitions in user space (dense)
# --------------------------------------------------------------------------

def _user_space_kkt(lp, x, y):
    A = ve.dense(lp)
    b, c = lp["b"], lp["c"]
    sense = lp["sense"]
    Ax = A @ x
    rp = b - Ax
    rp[sense == oracle.LE] = np.minimum(rp[sense == oracle.LE], 0.0)   # Ax <= b violated when b - Ax < 0
    rp[sense == oracle.GE] = np.maximum(rp[sense == oracle.GE], 0.0)   # Ax >= b violated when b - Ax > 0
    lam = c - A.T @ y
    lf, uf = np.isfinite(lp["lb"]), np.isfinite(lp["ub"])
    z = np.where(lf & uf, lam, np.where(lf, np.maximum(lam, 0), np.where(uf, np.minimum(lam, 0), 0.0)))
    rd = lam - z
    pobj = c @ x
    dobj = b @ y + np.sum(np.where(lf, lp["lb"], 0) * np.maximum(z, 0)) \
        - np.sum(np.where(uf, lp["ub"], 0) * np.maximum(-z, 0))
    return np.linalg.norm(rp), np.linalg.norm(rd), pobj, dobj, z


@pytest.mark.parametrize("bounded", [False, True])
def test_evaluate_matches_user_space_definitions(bounded):
    lp = lpgen.small_face_lp(4)
    if bounded:
        lp = lpgen.with_bounds_and_inequalities(lp, 4)
    model = oracle.Model(lp)
    rng = np.random.default_rng(0)
    xh = oracle.project_box(rng.standard_normal(model.n), model.lhat, model.uhat)
    yh = rng.standard_normal(model.m)
    yh[model.ge] = np.abs(yh[model.ge])
    ev = oracle.evaluate(model, xh, yh, 1.0)
    x, y, z = oracle.unscale(model, xh, yh)
    rP, rD, pobj, dobj, z_ref = _user_space_kkt(lp, x, y)
    assert abs(ev["rP2"] - rP) <= 1e-10 * (1 + rP)
    assert abs(ev["rD2"] - rD) <= 1e-10 * (1 + rD)
    assert abs(ev["pobj"] - pobj) <= 1e-10 * (1 + abs(pobj))
    assert abs(ev["dobj"] - dobj) <= 1e-10 * (1 + abs(dobj))
    assert np.allclose(z, z_ref, rtol=1e-10, atol=1e-12)
    # at the constructed optimum every residual and the gap vanish (Section 2)
    xs = lp["x_star"] / model.Dc
    ys = model.sign * lp["y_star"] / model.Dr
    ev = oracle.evaluate(model, xs, ys, 1.0)
    assert ev["rel_kkt"] < 1e-12


# --------------------------------------------------------------------------
# Convergence to the exact optimum (Section 2 termination, eps_rel = 1e-6)
# --------------------------------------------------------------------------

def _assert_optimal(lp, res, obj_star):
    assert res["status"] == oracle.OPTIMAL
    ev = res["eval"]
    assert ev["rel_kkt"] <= 1e-6
    x, y, z = oracle.unscale(res["model"], res["x_hat"], res["y_hat"])
    rP, rD, pobj, dobj, _ = _user_space_kkt(lp, x, y)
    nb, nc = np.linalg.norm(lp["b"]), np.linalg.norm(lp["c"])
    assert rP <= 1e-6 * (1 + nb) * (1 + 1e-9)
    assert rD <= 1e-6 * (1 + nc) * (1 + 1e-9)
    assert abs(pobj - dobj) <= 1e-6 * (1 + abs(pobj) + abs(dobj)) * (1 + 1e-9)
    # bounds hold up to the rounding of the unscaling product x = D_c x_hat
    assert np.all(x >= lp["lb"] - 1e-12 * np.abs(lp["lb"]))
    assert np.all(x <= lp["ub"] + 1e-12 * np.abs(lp["ub"]))
    # the objective agrees with the known optimum to the tolerance's order
    assert abs(pobj - obj_star) <= 2e-5 * (1 + abs(obj_star))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_converges_to_constructed_optimum(seed):
    lp = lpgen.small_face_lp(seed)
    res = oracle.solve(lp)
    _assert_optimal(lp, res, lp["obj_star"])


@pytest.mark.parametrize("seed", [0, 1])
def test_converges_with_bounds_and_inequalities(seed):
    lp = lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(10 + seed), seed)
    res = oracle.solve(lp)
    _assert_optimal(lp, res, lp["obj_star"])


def test_converges_power_law_general_form():
    lp = lpgen.power_law_lp(1500, 6000, 200, seed=77, kmax=300)
    res = oracle.solve(lp)
    _assert_optimal(lp, res, lp["obj_star"])


def _highs(lp):
    A = oracle.pdhg.csr_matrix(lp)
    sense = lp["sense"]
    eq, le, ge = sense == oracle.EQ, sense == oracle.LE, sense == oracle.GE
    A_ub = sp.vstack([A[le], -A[ge]]).tocsr()
    b_ub = np.concatenate([lp["b"][le], -lp["b"][ge]])
    bounds = list(zip(lp["lb"], [None if not np.isfinite(u) else u for u in lp["ub"]]))
    r = scipy.optimize.linprog(lp["c"], A_ub=A_ub if A_ub.shape[0] else None,
                               b_ub=b_ub if A_ub.shape[0] else None,
                               A_eq=A[eq], b_eq=lp["b"][eq], bounds=bounds, method="highs")
    assert r.status == 0
    return r.fun


def test_transportation_matches_highs():
    lp = lpgen.transportation_lp(12, 25, seed=3)
    res = oracle.solve(lp)
    assert res["status"] == oracle.OPTIMAL
    assert abs(res["eval"]["pobj"] - _highs(lp)) <= 2e-5 * (1 + abs(_highs(lp)))


def test_bounded_variant_matches_highs():
    lp = lpgen.with_bounds_and_inequalities(lpgen.random_face_lp(30, 70, 40, seed=9), 9)
    res = oracle.solve(lp)
    assert res["status"] == oracle.OPTIMAL
    f = _highs(lp)
    assert abs(res["eval"]["pobj"] - f) <= 2e-5 * (1 + abs(f))
    assert abs(f - lp["obj_star"]) <= 1e-7 * (1 + abs(f))


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_tiny_lp_matches_brute_force(seed):
    lp = lpgen.tiny_face_lp(5, 11, 7, seed=100 + seed)
    A = ve.dense(lp)
    best, face = ve.optimal_face_vertices(A, lp["b"], lp["c"])
    assert abs(best - lp["obj_star"]) <= 1e-9 * (1 + abs(best))
    res = oracle.solve(lp, dict(eps_rel=1e-9))
    assert res["status"] == oracle.OPTIMAL
    assert abs(res["eval"]["pobj"] - best) <= 1e-7 * (1 + abs(best))


# --------------------------------------------------------------------------
# Restart mechanics (reading: cuPDLP.jl-style), invariants only
# --------------------------------------------------------------------------

def test_restarts_only_at_checks_and_omega_update():
    lp = lpgen.small_face_lp(5)
    model, p, _, eta = oracle.setup(lp)
    s = oracle.State(model, oracle.project_box(np.zeros(model.n), model.lhat, model.uhat),
                     np.zeros(model.m), eta, oracle.initial_omega(model))
    for _ in range(63):
        oracle.pdhg_step(model, s)
    assert s.restarts == 0 and s.t == 63
    oracle.pdhg_step(model, s)
    xa, ya = s.average()
    ev_c = oracle.evaluate(model, s.x, s.y, s.omega)
    ev_a = oracle.evaluate(model, xa, ya, s.omega)
    x_r, y_r, w0 = s.x_r.copy(), s.y_r.copy(), s.omega
    # the first check always restarts: t = k >= 0.36 k
    assert oracle.restart_check(model, s, p, ev_c, ev_a)
    cand_avg = ev_a["kkt"] <= ev_c["kkt"]
    xc = xa if cand_avg else None
    if cand_avg:
        assert np.array_equal(s.x, xc)
    dx = np.linalg.norm(s.x - x_r)
    dy = np.linalg.norm(s.y - y_r)
    # exp(0.5 ln(dy/dx) + 0.5 ln w) is the geometric mean sqrt(w dy/dx)
    assert abs(s.omega - math.sqrt(w0 * dy / dx)) <= 1e-12 * s.omega
    assert s.t == 0 and s.restarts == 1 and s.kkt_prev == math.inf


# --------------------------------------------------------------------------
# Metrics (Sections 2.1 and 4.2)
# --------------------------------------------------------------------------

def test_metrics_at_constructed_optimum():
    lp = lpgen.small_face_lp(0)
    model = oracle.Model(lp)
    met = oracle.corner_metrics(model, lp["x_star"], lp["y_star"], lp["z_star"])
    # |S| = 250 variables strictly positive with zero reduced cost, m = 200
    assert met["off_bound_p"] == 250 and met["zero_rc_d"] == 250 and met["candidates"] == 250
    assert met["corner_measure"] == 50 and met["primal_push_est"] == 50
    assert met["dual_push_est"] == 0 and met["should_corner"] == 0


def test_metrics_at_a_vertex_are_zero():
    lp = lpgen.tiny_face_lp(5, 11, 7, seed=101)
    A = ve.dense(lp)
    best, face = ve.optimal_face_vertices(A, lp["b"], lp["c"])
    v, B = face[0]
    y, z = ve.basis_duals(A, lp["c"], B)
    met = oracle.corner_metrics(oracle.Model(lp), v, y, z)
    assert met["corner_measure"] == 0 and met["primal_push_est"] == 0
    assert met["zero_rc_d"] >= lp["m"] and met["dual_push_est"] == 0


def test_metrics_count_inequality_slacks():
    # one '<' row inactive at x (slack 1 > 1e-6) with y = 0: a slack candidate
    lp = dict(m=2, n=2, row_ptr=np.array([0, 2, 4]), col_idx=np.array([0, 1, 0, 1], dtype=np.int32),
              val=np.array([1.0, 1.0, 1.0, -1.0]), b=np.array([3.0, 0.0]), c=np.array([1.0, 1.0]),
              lb=np.zeros(2), ub=np.full(2, np.inf), sense=np.array([oracle.LE, oracle.EQ], dtype=np.int8))
    model = oracle.Model(lp)
    x = np.array([1.0, 1.0])
    met = oracle.corner_metrics(model, x, np.array([0.0, 0.5]), np.array([0.0, 0.0]))
    assert met["off_bound_p"] == 3 and met["zero_rc_d"] == 3 and met["candidates"] == 3
    assert met["corner_measure"] == 1


def test_should_corner_threshold():
    # candidates >= max(2m, 100000): build a model with m = 1 and 100000 free candidates
    n = 100_000
    lp = dict(m=1, n=n, row_ptr=np.array([0, 1]), col_idx=np.array([0], dtype=np.int32),
              val=np.array([1.0]), b=np.array([1.0]), c=np.zeros(n), lb=np.zeros(n),
              ub=np.full(n, np.inf), sense=np.array([oracle.EQ], dtype=np.int8))
    model = oracle.Model(lp, ruiz_iters=0)
    x = np.full(n, 1.0)
    assert oracle.corner_metrics(model, x, np.zeros(1), np.zeros(n))["should_corner"] == 1
    x[0] = 0.0
    assert oracle.corner_metrics(model, x, np.zeros(1), np.zeros(n))["should_corner"] == 0


# --------------------------------------------------------------------------
# Algorithm 1 and the Section 3.1 stopping rule
# --------------------------------------------------------------------------

def test_corner_face_invariants_and_stop_rule():
    lp = lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(6), 6)
    r1 = oracle.solve(lp)
    assert r1["status"] == oracle.OPTIMAL
    x1, y1, z1 = oracle.unscale(r1["model"], r1["x_hat"], r1["y_hat"])
    rc = oracle.corner_phase(r1, dict(obj_seed=3))
    assert rc["status"] == oracle.CORNER_DONE
    assert rc["iters"] >= 100 and rc["iters"] % 64 == 0
    model = r1["model"]
    xc = model.Dc * rc["x_hat"]
    up = z1 > 1e-6
    lo = z1 < -1e-6
    # Algorithm 1: ub_j <- x_j where z_j > eps_abs, lb_j <- x_j where z_j < -eps_abs
    assert np.all(xc[up] <= x1[up] * (1 + 1e-12) + 1e-15)
    assert np.all(xc[lo] >= x1[lo] * (1 - 1e-12) - 1e-15)
    assert np.all(xc >= lp["lb"] - 1e-12) and np.all(xc <= lp["ub"] * (1 + 1e-12))
    # the corner model's rows: inequality rows with |y_i| > eps_abs became '='
    cm = rc["corner_model"]
    to_eq = model.ge & (np.abs(y1) > 1e-6)
    assert np.array_equal(cm.ge, model.ge & ~to_eq)
    # the objective is the published SplitMix64 uniform draw, scaled like c
    assert np.array_equal(cm.c_cur, oracle.splitmix64_uniform(3, model.n))
    # Section 3.1: the primal residual on the corner model meets the original
    # tolerance, recomputed here in user space with the new senses
    A = ve.dense(lp)
    Axc = A @ xc
    sense_c = np.where(to_eq, oracle.EQ, lp["sense"])
    rp = lp["b"] - Axc
    rp[sense_c == oracle.LE] = np.minimum(rp[sense_c == oracle.LE], 0)
    rp[sense_c == oracle.GE] = np.maximum(rp[sense_c == oracle.GE], 0)
    assert np.linalg.norm(rp) <= 1e-6 * (1 + np.linalg.norm(lp["b"])) * (1 + 1e-9)
    # the returned duals are the phase-1 duals (Algorithm 1, last step)
    assert np.array_equal(rc["y_hat"], r1["y_hat"])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_corner_reaches_the_random_objective_vertex(seed):
    # run to full convergence (test flag), the corner phase returns the vertex
    # of the optimal face that minimises the random objective
    lp = lpgen.tiny_face_lp(5, 11, 7, seed=200 + seed)
    A = ve.dense(lp)
    best, face = ve.optimal_face_vertices(A, lp["b"], lp["c"])
    r1 = oracle.solve(lp, dict(eps_rel=1e-10))
    assert r1["status"] == oracle.OPTIMAL
    rc = oracle.corner_phase(r1, dict(obj_seed=seed, stop_rule="kkt", eps_rel=1e-10,
                                      max_iters=400_000))
    assert rc["status"] == oracle.CORNER_DONE
    cobj = oracle.splitmix64_uniform(seed, lp["n"])
    vals = [cobj @ v for v, _ in face]
    v_best = face[int(np.argmin(vals))][0]
    xc = r1["model"].Dc * rc["x_hat"]
    assert np.max(np.abs(xc - v_best)) <= 1e-4
    met = oracle.corner_metrics(r1["model"], xc, *oracle.unscale(r1["model"], r1["x_hat"], r1["y_hat"])[1:])
    assert met["primal_push_est"] == 0


def test_corner_row_rule_option_keeps_inactive_rows():
    # row_rule = 1 (an option, not the paper's rule): of the rows Section 3
    # turns into equalities, those whose slack at the phase-1 point exceeds
    # their dual stay inequalities, and the corner phase still regains the
    # tolerance
    lp = lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(6), 6)
    r1 = oracle.solve(lp)
    model = r1["model"]
    x1, y1, _ = oracle.unscale(model, r1["x_hat"], r1["y_hat"])
    cm0, _ = oracle.corner_model(model, r1["x_hat"], r1["y_hat"], dict(oracle.CORNER_DEFAULTS))
    cm1, _ = oracle.corner_model(model, r1["x_hat"], r1["y_hat"], dict(oracle.CORNER_DEFAULTS, row_rule=1))
    eq0 = model.ge & ~cm0.ge
    eq1 = model.ge & ~cm1.ge
    assert np.all(eq1 <= eq0)
    slack = model.A_int @ x1 - model.b_int
    assert np.array_equal(eq1, eq0 & (slack <= np.abs(y1)))
    rc = oracle.corner_phase(r1, dict(obj_seed=3, row_rule=1))
    assert rc["status"] == oracle.CORNER_DONE
