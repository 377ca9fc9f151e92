"""Pins of the oracle's dual corner push (oracle.pdhg.dual_corner_model /
dual_corner_phase, oracle.halpern.dual_corner_phase) against facts outside
the oracle: the model follows its definition (complementary slackness with
the phase-1 x), brute-force enumeration of the dual optimal face's vertices
on tiny LPs with a non-unique dual (the phase, run to full convergence,
returns the vertex that maximises the random b'), the count of zero reduced
costs at such a vertex (at least m), and the special case of a unique dual
(nothing moves).  CPU only."""
import itertools

import numpy as np
import pytest

import lpgen
import oracle
from tests import vertex_enum as ve

ALGS = ["averaged", "halpern"]


def _phase1(lp, alg, eps=1e-10):
    return oracle.solve(lp, dict(algorithm=alg, eps_rel=eps))


def test_dual_corner_model_follows_its_definition():
    lp = lpgen.with_bounds_and_inequalities(lpgen.random_face_lp(200, 500, 150, seed=3), 3)
    r1 = _phase1(lp, "averaged", 1e-9)
    model = r1["model"]
    cp = dict(oracle.CORNER_DEFAULTS, obj_seed=9, obj_scale=0.5)
    dm, info = oracle.dual_corner_model(model, r1["x_hat"], r1["y_hat"], cp)
    x, y, z = oracle.unscale(model, r1["x_hat"], r1["y_hat"])
    eps = cp["eps_abs"]
    # a bound stays unless x is off it: the distance exceeds eps_abs and the
    # part of z that bound allows (complementary slackness read at x)
    at_l = np.isfinite(model.l) & ~((x - model.l > eps) & (x - model.l > np.maximum(z, 0)))
    at_u = np.isfinite(model.u) & ~((model.u - x > eps) & (model.u - x > np.maximum(-z, 0)))
    assert np.array_equal(np.isfinite(dm.l), at_l) and np.array_equal(dm.l[at_l], model.l[at_l])
    assert np.array_equal(np.isfinite(dm.u), at_u) and np.array_equal(dm.u[at_u], model.u[at_u])
    # the constructed optimum: columns of S free, the others at a bound
    S = np.zeros(lp["n"], bool)
    S[lp["support"]] = True
    assert not np.any(np.isfinite(dm.l[S]) | np.isfinite(dm.u[S]))
    assert np.all(np.isfinite(dm.l[~S]) | np.isfinite(dm.u[~S]))
    # inactive inequality rows (slack above eps_abs and |y| at x) get a dual fixed at 0
    slack = model.A_int @ x - model.b_int
    assert np.array_equal(dm.y_zero, model.ge & (slack > eps) & (slack > np.abs(y)))
    ineq_inactive = (np.asarray(lp["sense"]) != oracle.EQ) & (np.abs(lp["y_star"]) == 0.0) & \
        (np.abs(lp["b"] - ve.dense(lp) @ lp["x_star"]) > 0.05)
    assert np.array_equal(dm.y_zero, ineq_inactive)
    # b' = obj_scale U[0,1) per user row (0 where the dual is fixed), negated on '<' rows, scaled by D_r
    u = 0.5 * oracle.splitmix64_uniform(9, lp["m"])
    want = np.where(dm.y_zero, 0.0, u)
    assert np.array_equal(dm.b_user, want)
    assert np.array_equal(dm.bhat, model.Dr * (model.sign * want))
    assert np.array_equal(dm.chat, model.chat)  # c is unchanged
    assert info["rows_zero"] == int(dm.y_zero.sum())


def _dual_face_vertices(A, c, S):
    """Vertices of {y : A_S' y = c_S, A_N' y <= c_N}: m - |S| more active
    columns K of N with [A_S A_K] nonsingular."""
    m, n = A.shape
    N = [j for j in range(n) if j not in set(S)]
    out = []
    for K in itertools.combinations(N, m - len(S)):
        B = list(S) + list(K)
        AB = A[:, B]
        if np.linalg.cond(AB) > 1e10:
            continue
        y = np.linalg.solve(AB.T, c[B])
        if np.all(A[:, N].T @ y <= c[N] + 1e-9):
            if not any(np.max(np.abs(y - v)) <= 1e-9 for v in out):
                out.append(y)
    return out


@pytest.mark.parametrize("alg", ALGS)
@pytest.mark.parametrize("seed", [1, 4, 8])
def test_dual_corner_reaches_the_random_objective_vertex(alg, seed):
    # 5 x 12 with |S| = 3: the dual optimal face has dimension 2; run to full
    # convergence, the dual corner phase returns the face vertex that
    # maximises b'y (brute force over all bases containing S)
    lp = lpgen.tiny_face_lp(5, 12, 3, seed=seed)
    A = ve.dense(lp)
    S = list(lp["support"])
    verts = _dual_face_vertices(A, lp["c"], S)
    assert len(verts) >= 2  # a non-unique dual
    cp = dict(obj_seed=seed + 100, stop_rule="kkt", eps_rel=1e-11, max_iters=2_000_000)
    bprime = oracle.splitmix64_uniform(cp["obj_seed"], lp["m"])
    vals = [float(bprime @ v) for v in verts]
    best = int(np.argmax(vals))
    srt = sorted(vals)
    if srt[-1] - srt[-2] < 1e-6:
        pytest.skip("two vertices tie for b'")
    r1 = _phase1(lp, alg)
    rd = oracle.dual_corner_phase(r1, cp)
    assert rd["status"] == oracle.CORNER_DONE
    _, y, z = oracle.unscale(r1["model"], rd["x_hat"], rd["y_hat"])
    assert np.max(np.abs(y - verts[best])) <= 1e-6
    # at the vertex m reduced costs vanish: no dual superbasic left
    rep = oracle.kkt_report(r1["model"], rd["x_hat"], rd["y_hat"])
    assert rep["zero_rc_d"] >= lp["m"] and rep["dual_push_est"] == 0
    # the phase keeps phase 1's x
    assert np.array_equal(rd["x_hat"], r1["x_hat"])


@pytest.mark.parametrize("alg", ALGS)
def test_dual_corner_removes_the_dual_superbasics(alg):
    # 200 x 500 with |S| = 150: phase 1 leaves the dual in the relative
    # interior of a 50-dimensional face (d = 150 zero reduced costs, a dual
    # push estimate of 50); the dual corner phase, converged to 1e-9,
    # reaches a vertex (d = m) while staying optimal
    lp = lpgen.random_face_lp(200, 500, 150, seed=3)
    r1 = _phase1(lp, alg, 1e-9)
    rep1 = oracle.kkt_report(r1["model"], r1["x_hat"], r1["y_hat"])
    assert rep1["zero_rc_d"] == 150 and rep1["dual_push_est"] == 50
    rd = oracle.dual_corner_phase(r1, dict(obj_seed=5, stop_rule="kkt", eps_rel=1e-9, max_iters=400_000))
    rep = oracle.kkt_report(r1["model"], rd["x_hat"], rd["y_hat"])
    assert rd["status"] == oracle.CORNER_DONE
    assert rep["zero_rc_d"] == 200 and rep["dual_push_est"] == 0
    assert rep["rel_kkt"] <= 1e-8  # still optimal for the original LP (x from phase 1)
    _, y, _ = oracle.unscale(r1["model"], rd["x_hat"], rd["y_hat"])
    assert abs(rep["dobj"] - lp["obj_star"]) <= 1e-7 * (1 + abs(lp["obj_star"]))


@pytest.mark.parametrize("alg", ALGS)
def test_dual_corner_keeps_a_unique_dual(alg):
    # |S| = m: the dual optimal face is one point, so the push moves nothing
    lp = lpgen.random_face_lp(60, 150, 60, seed=11)
    r1 = _phase1(lp, alg, 1e-10)
    rd = oracle.dual_corner_phase(r1, dict(obj_seed=2, stop_rule="kkt", eps_rel=1e-10, max_iters=400_000))
    _, y1, _ = oracle.unscale(r1["model"], r1["x_hat"], r1["y_hat"])
    _, y, _ = oracle.unscale(r1["model"], rd["x_hat"], rd["y_hat"])
    assert np.max(np.abs(y - y1)) <= 1e-6 * (1 + np.max(np.abs(y1)))
    assert np.max(np.abs(y - lp["y_star"])) <= 1e-6 * (1 + np.max(np.abs(lp["y_star"])))


@pytest.mark.parametrize("alg", ALGS)
def test_dual_corner_fixed_rows_and_limit(alg):
    # rows whose dual is fixed stay at exactly 0; the default stop rule (the
    # dual residual regained) stops at a check after min_iters; a limit keeps
    # the phase-1 dual
    lp = lpgen.with_bounds_and_inequalities(lpgen.random_face_lp(200, 500, 150, seed=3), 3)
    r1 = _phase1(lp, alg, 1e-9)
    rd = oracle.dual_corner_phase(r1, dict(obj_seed=5))
    dm = rd["dual_model"]
    assert dm.y_zero.any() and np.all(rd["y_hat"][dm.y_zero] == 0.0)
    assert rd["status"] == oracle.CORNER_DONE and rd["iters"] >= 100 and rd["iters"] % 64 == 0
    ev = oracle.evaluate(dm, r1["x_hat"] * 0 + rd["state"].x if alg == "averaged" else rd["state"].xp,
                         rd["y_hat"], 1.0)
    assert ev["rD2"] <= 1e-6 * (1 + np.linalg.norm(lp["c"]))
    lim = oracle.dual_corner_phase(r1, dict(obj_seed=5, max_iters=64))
    assert lim["status"] == oracle.CORNER_LIMIT and np.array_equal(lim["y_hat"], r1["y_hat"])


@pytest.mark.parametrize("alg", ALGS)
def test_dual_corner_reads_near_threshold_pairs_by_complementarity(alg):
    # at a 1e-6 phase-1 point an active row can show a slack just above
    # eps_abs (1.4e-6 here) beside a dual of order 1: it keeps its dual, the
    # model's dual stays non-empty, and the phase regains dual feasibility
    lp = lpgen.with_bounds_and_inequalities(lpgen.random_face_lp(200, 500, 150, seed=3), 3)
    r1 = _phase1(lp, alg, 1e-6)
    model = r1["model"]
    x, y, _ = oracle.unscale(model, r1["x_hat"], r1["y_hat"])
    slack = model.A_int @ x - model.b_int
    near = model.ge & (slack > 1e-6) & (slack < 1e-5) & (np.abs(y) > 1e-2)
    assert near.any()
    rd = oracle.dual_corner_phase(r1, dict(obj_seed=5, max_iters=200_000))
    assert not rd["dual_model"].y_zero[near].any()
    assert rd["status"] == oracle.CORNER_DONE
    rep = oracle.kkt_report(model, rd["x_hat"], rd["y_hat"])
    assert rep["rel_d"] <= 1e-6 and rep["rel_kkt"] <= 1e-5
