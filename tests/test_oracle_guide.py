"""Pins of the guidance oracle (oracle/mlp.py, oracle/guide.py) to facts
outside itself: central finite differences, Adam's closed form under a
constant gradient (Kingma & Ba 2015, Algorithm 1), the restart history the
phase-1 state itself recorded, brute-force vertex enumeration of the held
face, and the constructed optima's at-bound pattern.
"""
import numpy as np
import pytest

import lpgen
import oracle
from oracle import guide, mlp
from tests import vertex_enum as ve


def _rand_weights(seed):
    w = mlp.init_weights(seed)
    rng = np.random.default_rng(seed + 100)
    for k in ("b1", "b2"):
        w[k] = rng.standard_normal(w[k].shape) * 0.1
    w["b3"] = np.asarray(0.2)
    return w


# --------------------------------------------------------------------------
# MLP: finite differences, special cases, Adam
# --------------------------------------------------------------------------

def test_mlp_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((40, mlp.IN))
    y = (rng.random(40) < 0.4).astype(float)
    w = _rand_weights(3)
    g = mlp.gradients(w, X, y)
    h = 1e-6
    for k in w:
        fd = np.zeros_like(np.asarray(w[k], dtype=float))
        flat = fd.reshape(-1)
        for idx in range(flat.size):
            wp = {kk: np.array(vv, dtype=float, copy=True) for kk, vv in w.items()}
            wm = {kk: np.array(vv, dtype=float, copy=True) for kk, vv in w.items()}
            wp[k].reshape(-1)[idx] += h
            wm[k].reshape(-1)[idx] -= h
            flat[idx] = (mlp.loss_of(wp, X, y) - mlp.loss_of(wm, X, y)) / (2 * h)
        rel = np.linalg.norm(fd - g[k]) / max(np.linalg.norm(fd), 1e-300)
        assert rel <= 1e-6, (k, rel)


def test_mlp_zero_network_is_half_and_ln2():
    w = {k: np.zeros_like(v) for k, v in mlp.init_weights(0).items()}
    X = np.random.default_rng(2).standard_normal((10, mlp.IN))
    y = np.array([1, 0, 1, 1, 0, 0, 1, 0, 1, 1], dtype=float)
    p, _ = mlp.forward(w, X)
    assert np.all(p == 0.5)
    assert abs(mlp.bce(p, y) - np.log(2.0)) <= 1e-15
    g = mlp.gradients(w, X, y)
    assert abs(float(g["b3"]) - np.mean(0.5 - y)) <= 1e-15
    for k in ("W1", "b1", "W2", "b2", "w3"):
        assert np.all(g[k] == 0.0)


def test_mlp_single_path_closed_form():
    # one active unit per layer: o = w3_0 * relu(W2_00 * relu(W1_0 . x + b1_0) + b2_0) + b3
    w = {k: np.zeros_like(v) for k, v in mlp.init_weights(0).items()}
    w["W1"][0, 3] = 2.0
    w["b1"][0] = -0.5
    w["W2"][0, 0] = 1.5
    w["b2"][0] = 0.25
    w["w3"][0] = -3.0
    w["b3"] = np.asarray(0.1)
    X = np.zeros((3, mlp.IN))
    X[:, 3] = [1.0, 0.1, -2.0]
    h1 = np.maximum(2.0 * X[:, 3] - 0.5, 0.0)
    h2 = np.maximum(1.5 * h1 + 0.25, 0.0)
    o = -3.0 * h2 + 0.1
    p, _ = mlp.forward(w, X)
    assert np.allclose(p, 1.0 / (1.0 + np.exp(-o)), rtol=0, atol=1e-15)


def test_adam_constant_gradient_closed_form():
    # with a constant gradient g the bias-corrected moments are exactly g and
    # g^2, so every step moves by -lr * g / (|g| + eps)
    w = {"a": np.array([1.0, -2.0, 0.5]), "b": np.asarray(3.0)}
    g = {"a": np.array([0.3, -4.0, 1e-3]), "b": np.asarray(-0.7)}
    st = {}
    lr, eps = 0.01, 1e-8
    for _ in range(5):
        w = mlp.adam_step(w, g, st, lr=lr, eps=eps)
    step = -lr * g["a"] / (np.abs(g["a"]) + eps)
    assert np.allclose(w["a"], np.array([1.0, -2.0, 0.5]) + 5 * step, rtol=0, atol=1e-12)
    assert abs(float(w["b"]) - (3.0 + 5 * lr * 0.7 / (0.7 + eps))) <= 1e-12


# --------------------------------------------------------------------------
# History ring and features
# --------------------------------------------------------------------------

def test_history_is_the_restart_sequence():
    lp = lpgen.small_face_lp(3)
    r = oracle.solve(lp)
    s = r["state"]
    assert s.restarts >= 1
    X, Z = guide.history(s)
    # newest entry = the last restart point; its z = proj(c_hat - A_hat' y_r)
    assert np.array_equal(X[:, 0], s.x_r)
    model = r["model"]
    z_r = oracle.project_dual_cone(model.chat - model.AhatT @ s.y_r, model.lhat, model.uhat)
    assert np.allclose(Z[:, 0], z_r, rtol=0, atol=1e-14)
    if s.restarts < 7:
        # padded with the oldest entry: the start point, with y = 0
        k = s.restarts
        x0 = oracle.project_box(np.zeros(model.n), model.lhat, model.uhat)
        assert np.array_equal(X[:, k], x0)
        assert np.all(X[:, k:] == X[:, [k]])
        assert np.array_equal(Z[:, k], oracle.project_dual_cone(model.chat, model.lhat, model.uhat))


def test_history_pads_with_the_oldest_of_the_last_eight():
    lp = lpgen.small_face_lp(0)
    r = oracle.solve(lp, dict(eps_rel=1e-9))
    s = r["state"]
    assert s.restarts >= 8
    X, _ = guide.history(s)
    assert len(s.ring) == 8
    # no padding once the ring is full: 8 distinct restart points
    assert all(not np.array_equal(X[:, i], X[:, i + 1]) for i in range(7))


def test_features_groups_have_unit_rms_and_layout():
    lp = lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(5), 5)
    r = oracle.solve(lp)
    cp = dict(obj_seed=7)
    F, elig = guide.features(r, cp)
    assert F.shape == (lp["n"], 18)
    for cols in ([0], [1], list(range(2, 10)), list(range(10, 18))):
        assert abs(np.sqrt(np.mean(F[:, cols] ** 2)) - 1.0) <= 1e-12
    model = r["model"]
    cm, _ = oracle.corner_model(model, r["x_hat"], r["y_hat"], dict(oracle.CORNER_DEFAULTS, **cp))
    # column 0 is proportional to the corner objective, column 1 to ||A_hat_j||
    ratio = F[:, 0] / cm.chat
    assert np.allclose(ratio, ratio[0], rtol=1e-12)
    dense = ve.dense(dict(m=model.m, n=model.n, row_ptr=model.Ahat.indptr,
                          col_idx=model.Ahat.indices, val=model.Ahat.data))
    cn = np.linalg.norm(dense, axis=0)
    nz = cn > 0
    assert np.allclose(F[nz, 1] / cn[nz], F[nz, 1][0] / cn[nz][0], rtol=1e-12)


def test_eligible_excludes_fixed_and_free_columns():
    lp = lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(6), 6)
    r = oracle.solve(lp)
    cp = dict(oracle.CORNER_DEFAULTS)
    _, info = oracle.corner_model(r["model"], r["x_hat"], r["y_hat"], cp)
    elig = guide.eligible(r, cp)
    assert not np.any(elig & info["fixed"])
    assert np.all(elig | info["fixed"])  # every column here has l = 0 finite
    # a free column is never eligible
    nb = oracle.pdhg.nearest_bound(np.array([0.3, 2.0, 5.0, 1.0]),
                                   np.array([-np.inf, 0.0, 0.0, -np.inf]),
                                   np.array([np.inf, 3.0, 6.0, 4.0]))
    assert np.isnan(nb[0]) and nb[1] == 3.0 and nb[2] == 6.0 and nb[3] == 4.0


def test_labels_at_the_constructed_optimum():
    lp = lpgen.small_face_lp(7)
    model = oracle.Model(lp)
    x_hat = lp["x_star"] / model.Dc
    lab = guide.labels(model, x_hat, x_hat)
    # off S the constructed x* is 0 (at its nearest bound), on S it lies in
    # [0.1, 1], away from the only finite bound
    assert np.array_equal(guide.labels(model, x_hat, np.zeros(lp["n"])), lab)
    on_s = lp["x_star"] > 0
    assert np.array_equal(lab, ~on_s)
    assert int(lab.sum()) == lp["n"] - int(on_s.sum())


def test_labels_use_the_bound_nearest_to_the_phase1_point():
    # a column at its upper bound is labelled 1 only when the phase-1 point
    # was nearer to that bound
    lp = lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(7), 7)
    model = oracle.Model(lp)
    j = int(np.nonzero(np.isfinite(lp["ub"]))[0][0])
    x = np.zeros(lp["n"])
    x[j] = lp["ub"][j]
    x_hat = x / model.Dc
    near_u = np.zeros(lp["n"])
    near_u[j] = 0.9 * lp["ub"][j] / model.Dc[j]
    near_l = np.zeros(lp["n"])
    near_l[j] = 0.1 * lp["ub"][j] / model.Dc[j]
    assert guide.labels(model, x_hat, near_u)[j]
    assert not guide.labels(model, x_hat, near_l)[j]


# --------------------------------------------------------------------------
# Guided corner phase
# --------------------------------------------------------------------------

def test_guided_with_empty_hold_is_the_plain_corner():
    lp = lpgen.small_face_lp(8)
    r = oracle.solve(lp)
    cp = dict(obj_seed=2)
    plain = oracle.corner_phase(r, cp)
    g = oracle.corner_phase(r, cp, hold=np.zeros(lp["n"], dtype=bool))
    assert g["iters"] == plain["iters"] and g["status"] == plain["status"]
    assert np.array_equal(g["x_hat"], plain["x_hat"])
    assert g["info"]["held"] == 0


def test_held_columns_stay_at_their_bound():
    lp = lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(9), 9)
    r = oracle.solve(lp)
    model = r["model"]
    cp = dict(obj_seed=4)
    elig = guide.eligible(r, dict(oracle.CORNER_DEFAULTS, **cp))
    x1 = model.Dc * r["x_hat"]
    # hold the five eligible columns nearest to a bound at the phase-1 point
    dist = np.where(elig, np.minimum(x1 - model.l, model.u - x1), np.inf)
    hold = np.zeros(lp["n"], dtype=bool)
    hold[np.argsort(dist)[:5]] = True
    g = oracle.corner_phase(r, cp, hold=hold)
    held = g["info"]["held_mask"]
    assert held.sum() == hold.sum() > 0
    nb = oracle.pdhg.nearest_bound(r["x_hat"], model.lhat, model.uhat)
    s = g["state"]
    assert np.array_equal(s.x[held], nb[held])
    assert np.array_equal(g["x_hat"][held], nb[held]) or g["status"] == oracle.CORNER_LIMIT


@pytest.mark.parametrize("seed", [0, 1])
def test_guided_corner_reaches_the_held_face_vertex(seed):
    # hold one column of the optimal face at 0: the corner phase, run to full
    # convergence, returns the c'-argmin vertex of the optimal face with that
    # column at 0 (brute force over bases)
    lp = lpgen.tiny_face_lp(5, 11, 7, seed=300 + seed)
    A = ve.dense(lp)
    best, face = ve.optimal_face_vertices(A, lp["b"], lp["c"])
    r1 = oracle.solve(lp, dict(eps_rel=1e-10))
    assert r1["status"] == oracle.OPTIMAL
    cobj = oracle.splitmix64_uniform(seed, lp["n"])
    # a column positive at some face vertex and zero at another
    pos = np.array([v for v, _ in face])
    cand = [j for j in range(lp["n"]) if pos[:, j].max() > 1e-6 and pos[:, j].min() <= 1e-9]
    assert cand, "tiny face without a column to hold"
    j = cand[0]
    hold = np.zeros(lp["n"], dtype=bool)
    hold[j] = True
    cp = dict(obj_seed=seed, stop_rule="kkt", eps_rel=1e-10, max_iters=400_000)
    rc = oracle.corner_phase(r1, cp, hold=hold)
    assert rc["status"] == oracle.CORNER_DONE
    sub = [v for v, _ in face if v[j] <= 1e-9]
    v_best = sub[int(np.argmin([cobj @ v for v in sub]))]
    xc = r1["model"].Dc * rc["x_hat"]
    assert np.max(np.abs(xc - v_best)) <= 1e-4


def test_fallback_when_the_hold_breaks_feasibility():
    # holding every column of S at 0 leaves b = A x unreachable: the guided run
    # regresses, and the plain corner phase is returned
    lp = lpgen.small_face_lp(10)
    r = oracle.solve(lp)
    cp = dict(obj_seed=1, max_iters=4096)
    hold = lp["x_star"] > 0
    out = guide.guided_corner_phase(r, hold, cp)
    assert out["fell_back"]
    plain = oracle.corner_phase(r, cp)
    assert np.array_equal(out["result"]["x_hat"], plain["x_hat"])
    # a hold that changes nothing never falls back
    out2 = guide.guided_corner_phase(r, np.zeros(lp["n"], dtype=bool), cp)
    assert not out2["fell_back"] or out2["guided"]["status"] == oracle.CORNER_LIMIT
