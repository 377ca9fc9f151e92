"""Pins of the Halpern loop of the oracle (oracle.halpern) to facts outside it.

- the PDHG map is firmly nonexpansive in the metric M the module states
  (with the other sign of the cross term it is not);
- the constructed optimum is a fixed point of the map;
- Halpern's anchored iteration keeps the tight rate bound
  ||z_k - T z_k||_M <= 2 ||z_0 - z*||_M / ((1 + rho)(k + 1)) (Lieder 2021) when
  it never restarts;
- with T = 0 the iterates have a closed form that fixes the weights and the
  reflection;
- the PID weight reduces to the ratio |dy| / |dx| with gains (1, 0, 0) and
  settles on a constant ratio from either side;
- full solves reach constructed optima, HiGHS and brute-force vertices, and
  the corner phase reaches the random-objective vertex (Algorithm 1).
"""
import math

import numpy as np
import pytest

import lpgen
import oracle
from oracle import halpern as H
from oracle import pdhg as P
from tests import vertex_enum as ve
from tests.test_oracle_pins import _assert_optimal, _highs

HP = dict(algorithm="halpern")


def _scaled(lp):
    model, p, sigma_max, eta = P.setup(lp)
    omega = P.initial_omega(model)
    return model, eta / omega, eta * omega, eta, omega


def _optimum_hat(model, lp):
    """The constructed optimum in scaled space: x_hat = x / D_c, y_hat = sign y / D_r."""
    return lp["x_star"] / model.Dc, model.sign * lp["y_star"] / model.Dr


def test_map_is_firmly_nonexpansive_in_the_metric():
    lp = lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(6), 6)
    model, tau, sigma, _, _ = _scaled(lp)
    rng = np.random.default_rng(0)

    def excess(sign):
        def n2(dx, dy):
            return dx @ dx / tau + dy @ dy / sigma + sign * 2.0 * dy @ (model.Ahat @ dx)
        worst = -np.inf
        for _ in range(100):
            s = rng.uniform(0.1, 10.0)
            x1, y1 = rng.standard_normal(model.n) * s, rng.standard_normal(model.m) * s
            x2 = x1 + rng.standard_normal(model.n) * rng.uniform(0.01, 1.0)
            y2 = y1 + rng.standard_normal(model.m) * rng.uniform(0.01, 1.0)
            a1, b1 = H.pdhg_map(model, x1, y1, tau, sigma)
            a2, b2 = H.pdhg_map(model, x2, y2, tau, sigma)
            lhs = n2(a1 - a2, b1 - b2) + n2((x1 - a1) - (x2 - a2), (y1 - b1) - (y2 - b2))
            rhs = n2(x1 - x2, y1 - y2)
            assert rhs > 0.0
            worst = max(worst, (lhs - rhs) / rhs)
        return worst

    assert excess(1.0) <= 1e-12
    # the metric's cross-term sign matters: with the other sign the map is not
    # firmly nonexpansive
    assert excess(-1.0) > 1e-2
    # and the module's metric is the + one
    dx, dy = rng.standard_normal(model.n), rng.standard_normal(model.m)
    assert H.metric_norm2(model, dx, dy, tau, sigma) == pytest.approx(
        dx @ dx / tau + dy @ dy / sigma + 2.0 * dy @ (model.Ahat @ dx), rel=1e-13)


def test_constructed_optimum_is_a_fixed_point():
    for seed in (0, 1):
        lp = lpgen.small_face_lp(seed)
        model, tau, sigma, _, _ = _scaled(lp)
        xs, ys = _optimum_hat(model, lp)
        xp, yp = H.pdhg_map(model, xs, ys, tau, sigma)
        assert np.max(np.abs(xp - xs)) <= 1e-13 * (1 + np.max(np.abs(xs)))
        assert np.max(np.abs(yp - ys)) <= 1e-12 * (1 + np.max(np.abs(ys)))
        assert H.fixed_point_residual(model, xs, ys, xp, yp, tau, sigma) <= 1e-12


@pytest.mark.parametrize("rho", [0.0, 0.5, 1.0])
def test_halpern_rate_bound_without_restarts(rho):
    lp = lpgen.small_face_lp(0)
    model, tau, sigma, eta, omega = _scaled(lp)
    xs, ys = _optimum_hat(model, lp)
    s = H.HState(model, P.project_box(np.zeros(model.n), model.lhat, model.uhat),
                 np.zeros(model.m), eta, omega)
    d0 = math.sqrt(H.metric_norm2(model, s.x - xs, s.y - ys, tau, sigma))
    for k in range(1500):
        xp, yp = H.pdhg_map(model, s.x, s.y, tau, sigma)
        r = H.fixed_point_residual(model, s.x, s.y, xp, yp, tau, sigma)
        assert r <= 2.0 * d0 / ((1.0 + rho) * (k + 1)) * (1 + 1e-9)
        H.halpern_step(model, s, rho)


def test_weights_and_reflection_closed_form():
    # T = 0 (zp = 0): rho = 0 gives z_k = z_0 / (k + 1); rho = 1 (S = -I)
    # gives z_k = z_0 / (k + 1) for even k and 0 for odd k
    z0 = np.array([3.0, -2.0, 0.5])
    for rho in (0.0, 1.0):
        z = z0.copy()
        for k in range(1, 40):
            z = H.halpern_update(z, np.zeros(3), z0, k - 1, rho)
            want = z0 / (k + 1) if (rho == 0.0 or k % 2 == 0) else np.zeros(3)
            assert np.allclose(z, want, rtol=1e-14, atol=1e-15)


def test_pid_weight():
    # gains (1, 0, 0): the weight becomes the ratio of the anchor movements
    om, integ, e = H.pid_update(3.0, 0.5, 2.0, 0.0, 0.0, 1.0, 0.0, 0.0)
    assert om == pytest.approx(4.0, rel=1e-14)
    # zero gains or a vanishing movement leave it unchanged
    assert H.pid_update(3.0, 0.5, 2.0, 0.0, 0.0, 0.0, 0.0, 0.0)[0] == pytest.approx(3.0, rel=1e-14)
    assert H.pid_update(3.0, 1e-11, 2.0, 0.7, 0.1, 0.99, 0.01, 0.0) == (3.0, 0.7, 0.1)
    # the default gains settle on a constant ratio from above and from below
    # (the integral term decays like 0.99^n)
    for start in (1e-3, 1e3):
        om, integ, e = start, 0.0, 0.0
        for _ in range(3000):
            om, integ, e = H.pid_update(om, 2.0, 5.0, integ, e, 0.99, 0.01, 0.0)
        assert om == pytest.approx(2.5, rel=1e-6)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_halpern_converges_to_constructed_optimum(seed):
    lp = lpgen.small_face_lp(seed)
    res = oracle.solve(lp, HP)
    _assert_optimal(lp, res, lp["obj_star"])


def test_halpern_converges_with_bounds_and_inequalities():
    lp = lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(10), 0)
    res = oracle.solve(lp, HP)
    _assert_optimal(lp, res, lp["obj_star"])


def test_halpern_converges_power_law_general_form():
    lp = lpgen.power_law_lp(1500, 6000, 200, seed=77, kmax=300)
    res = oracle.solve(lp, HP)
    _assert_optimal(lp, res, lp["obj_star"])


def test_halpern_transportation_matches_highs():
    lp = lpgen.transportation_lp(12, 25, seed=3)
    res = oracle.solve(lp, HP)
    assert res["status"] == oracle.OPTIMAL
    f = _highs(lp)
    assert abs(res["eval"]["pobj"] - f) <= 2e-5 * (1 + abs(f))


@pytest.mark.parametrize("seed", [0, 1])
def test_halpern_tiny_lp_matches_brute_force(seed):
    lp = lpgen.tiny_face_lp(5, 11, 7, seed=100 + seed)
    best, _ = ve.optimal_face_vertices(ve.dense(lp), lp["b"], lp["c"])
    res = oracle.solve(lp, dict(HP, eps_rel=1e-9))
    assert res["status"] == oracle.OPTIMAL
    assert abs(res["eval"]["pobj"] - best) <= 1e-7 * (1 + abs(best))


def test_halpern_restarts_at_checks_from_the_output():
    lp = lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(6), 6)
    p = H._params(HP)
    model, _, _, eta, omega = _scaled(lp)
    s = H.HState(model, P.project_box(np.zeros(model.n), model.lhat, model.uhat),
                 np.zeros(model.m), eta, omega)
    # the anchor residual is that of the start point
    xp, yp = H.pdhg_map(model, s.x, s.y, s.tau, s.sigma)
    assert s.r0 == H.fixed_point_residual(model, s.x, s.y, xp, yp, s.tau, s.sigma)
    restarts = 0
    for _ in range(64 * 40):
        x_pre, y_pre = H.halpern_step(model, s, p["reflection"])
        if s.k % p["check_period"]:
            continue
        r = H.fixed_point_residual(model, x_pre, y_pre, s.xp, s.yp, s.tau, s.sigma)
        if H.restart_due(r, s.r0, s.r_prev, s.t, s.k, p):
            xp, yp = s.xp.copy(), s.yp.copy()
            H.apply_restart(model, s, p, r)
            restarts += 1
            # the new anchor and iterate are the PDHG output of the check
            assert np.array_equal(s.x0, xp) and np.array_equal(s.y, yp) and s.t == 0 and s.r0 == r
            assert np.all(s.x0 >= model.lhat) and np.all(s.x0 <= model.uhat)
            assert np.all(s.y0[model.ge] >= 0.0)
        else:
            s.r_prev = r
    assert restarts >= 3


@pytest.mark.parametrize("seed", [0, 1])
def test_halpern_corner_reaches_the_random_objective_vertex(seed):
    lp = lpgen.tiny_face_lp(5, 11, 7, seed=200 + seed)
    _, face = ve.optimal_face_vertices(ve.dense(lp), lp["b"], lp["c"])
    r1 = oracle.solve(lp, dict(HP, eps_rel=1e-10))
    assert r1["status"] == oracle.OPTIMAL
    rc = oracle.corner_phase(r1, dict(obj_seed=seed, stop_rule="kkt", eps_rel=1e-10, max_iters=400_000))
    assert rc["status"] == oracle.CORNER_DONE
    cobj = oracle.splitmix64_uniform(seed, lp["n"])
    v_best = face[int(np.argmin([cobj @ v for v, _ in face]))][0]
    assert np.max(np.abs(r1["model"].Dc * rc["x_hat"] - v_best)) <= 1e-4


def test_halpern_corner_primal_rule():
    lp = lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(6), 6)
    r1 = oracle.solve(lp, HP)
    rc = oracle.corner_phase(r1, dict(obj_seed=3))
    assert rc["status"] == oracle.CORNER_DONE and rc["iters"] % 64 == 0 and rc["iters"] >= 100
    model = r1["model"]
    x1, y1, z1 = oracle.unscale(model, r1["x_hat"], r1["y_hat"])
    xc = model.Dc * rc["x_hat"]
    A = ve.dense(lp)
    to_eq = model.ge & (np.abs(y1) > 1e-6)
    sense_c = np.where(to_eq, oracle.EQ, lp["sense"])
    rp = lp["b"] - A @ xc
    rp[sense_c == oracle.LE] = np.minimum(rp[sense_c == oracle.LE], 0)
    rp[sense_c == oracle.GE] = np.maximum(rp[sense_c == oracle.GE], 0)
    assert np.linalg.norm(rp) <= 1e-6 * (1 + np.linalg.norm(lp["b"])) * (1 + 1e-9)
    up, lo = z1 > 1e-6, z1 < -1e-6
    assert np.all(xc[up] <= x1[up] * (1 + 1e-12) + 1e-15)
    assert np.all(xc[lo] >= x1[lo] * (1 - 1e-12) - 1e-15)
    assert np.array_equal(rc["y_hat"], r1["y_hat"])


def test_corner_phase_is_scale_equivariant_with_the_objective_weight():
    # omega_rule 0 starts omega at ||c_hat'|| / ||b_hat||, proportional to the
    # objective's scale; scaling c, y and omega together leaves every x
    # iterate unchanged, and the Halpern loop's restart test and PID weight are
    # homogeneous in that scaling, so obj_scale changes nothing but rounding
    lp = lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(3), 3)
    r1 = oracle.solve(lp, HP)
    runs = [oracle.corner_phase(r1, dict(obj_seed=11, obj_scale=sc)) for sc in (1.0, 1e-3, 1e-6)]
    for rc in runs[1:]:
        assert rc["iters"] == runs[0]["iters"] and rc["restarts"] == runs[0]["restarts"]
        assert np.max(np.abs(rc["x_hat"] - runs[0]["x_hat"])) <= 1e-9 * (1 + np.max(np.abs(runs[0]["x_hat"])))


@pytest.mark.parametrize("alg", ["averaged", "halpern"])
def test_corner_omega_rule_keeps_the_phase1_weight(alg):
    lp = lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(3), 3)
    r1 = oracle.solve(lp, dict(algorithm=alg))
    # one step, stopped at its limit before any restart: omega is the start value
    kept = oracle.corner_phase(r1, dict(obj_seed=11, obj_scale=1e-4, omega_rule=1, max_iters=1))
    fresh = oracle.corner_phase(r1, dict(obj_seed=11, obj_scale=1e-4, omega_rule=0, max_iters=1))
    assert kept["state"].omega == r1["state"].omega
    assert fresh["state"].omega == oracle.initial_omega(fresh["corner_model"])
    assert fresh["state"].omega != kept["state"].omega


def test_halpern_guided_corner_with_an_empty_hold_is_the_plain_corner():
    lp = lpgen.small_face_lp(8)
    r = oracle.solve(lp, HP)
    cp = dict(obj_seed=2)
    plain = oracle.corner_phase(r, cp)
    g = oracle.corner_phase(r, cp, hold=np.zeros(lp["n"], dtype=bool))
    assert g["iters"] == plain["iters"] and g["status"] == plain["status"]
    assert np.array_equal(g["x_hat"], plain["x_hat"]) and g["info"]["held"] == 0


def test_halpern_held_columns_end_at_their_bound():
    # the held columns' T(z) is projected onto l_hat = u_hat = the bound, so
    # the returned point holds them exactly there (the reflected iterate itself
    # may sit an ulp off)
    from oracle import guide
    lp = lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(9), 9)
    r = oracle.solve(lp, HP)
    model = r["model"]
    cp = dict(obj_seed=4)
    elig = guide.eligible(r, dict(oracle.CORNER_DEFAULTS, **cp))
    x1 = model.Dc * r["x_hat"]
    dist = np.where(elig, np.minimum(x1 - model.l, model.u - x1), np.inf)
    hold = np.zeros(lp["n"], dtype=bool)
    hold[np.argsort(dist)[:5]] = True
    g = oracle.corner_phase(r, cp, hold=hold)
    held = g["info"]["held_mask"]
    assert held.sum() == hold.sum() > 0
    nb = P.nearest_bound(r["x_hat"], model.lhat, model.uhat)
    assert np.array_equal(g["state"].xp[held], nb[held])
    if g["status"] == oracle.CORNER_DONE:
        assert np.array_equal(g["x_hat"][held], nb[held])
