"""Batched solve (one persistent launch, one CTA per LP) vs the CPU oracle
through the C ABI (needs a GB300).  The batched kernel runs the same
operators as the single-LP path with CTA-level scheduling and reductions, so
the same tolerances apply: FP64 iterates to 1e-10 after 100 iterations, equal
iteration and restart counts on full solves."""
import numpy as np
import pytest

import lpgen
import oracle

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2511_13894_gb300.pdhgc")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _mixed_lps():
    return [
        lpgen.small_face_lp(0),
        lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(3), 3),
        lpgen.tiny_face_lp(5, 11, 7, seed=101),
        lpgen.transportation_lp(30, 70, seed=2),
        lpgen.power_law_lp(1500, 6000, 200, seed=77, kmax=300),
        lpgen.random_face_lp(700, 2100, 875, seed=31, col_nnz_range=(3, 12)),
    ]


def rel_err(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(1.0, float(np.max(np.abs(b)))))


def test_batch_fp64_iterates_after_100_match_oracle():
    lps = _mixed_lps()
    B = P.Batch(lps)
    reps = B.solve(max_iters=100, eps_rel=-1.0)
    for k, lp in enumerate(lps):
        ref = oracle.run_iterations(lp, 100)
        assert reps[k]["status_name"] == "ITER_LIMIT" and reps[k]["iters"] == 100
        assert reps[k]["restarts"] == ref["restarts"]
        xo, yo, _ = oracle.unscale(ref["model"], ref["x_hat"], ref["y_hat"])
        x, y = B.get_solution(k)
        assert rel_err(x, xo) <= 1e-10 and rel_err(y, yo) <= 1e-10, k


def test_batch_fp64_full_solves_match_oracle():
    lps = _mixed_lps()
    B = P.Batch(lps)
    B.set_handoff(0)  # every LP to the end inside the batched kernel
    reps = B.solve()
    for k, lp in enumerate(lps):
        ref = oracle.solve(lp)
        assert reps[k]["status_name"] == "OPTIMAL" and ref["status"] == oracle.OPTIMAL, k
        assert reps[k]["iters"] == ref["iters"] and reps[k]["restarts"] == ref["restarts"], k
        assert reps[k]["rel_kkt"] <= 1e-6
        orep = oracle.kkt_report(ref["model"], ref["x_hat"], ref["y_hat"])
        for key in ("off_bound_p", "zero_rc_d", "candidates", "corner_measure"):
            assert reps[k][key] == orep[key], (k, key)
    # Algorithm 1 on every LP, same counts as the oracle
    creps = B.corner_phase(obj_seed=11)
    for k, lp in enumerate(lps[:3]):
        ref1 = oracle.solve(lp)
        refc = oracle.corner_phase(ref1, dict(obj_seed=11))
        assert creps[k]["status"] == refc["status"] and creps[k]["iters"] == refc["iters"], k
        x, _ = B.get_solution(k, P.CORNER)
        xo, _, _ = oracle.unscale(ref1["model"], refc["x_hat"], refc["y_hat"])
        assert rel_err(x, xo) <= 1e-7, k


def test_batch_fp32_reaches_tolerance_and_schedules_agree():
    lps = _mixed_lps()
    B = P.Batch(lps)
    reps = B.solve(precision=P.FP32_BULK)
    for k, r in enumerate(reps):
        assert r["status_name"] == "OPTIMAL" and r["rel_kkt"] <= 1e-6, (k, r["status_name"], r["rel_kkt"])
    # another schedule (lanes per row, block size) changes only rounding order
    B.set_block(512)
    B.set_lanes(1, 1)
    reps2 = B.solve(precision=P.FP32_BULK)
    for r, r2 in zip(reps, reps2):
        assert r2["status_name"] == "OPTIMAL" and r2["rel_kkt"] <= 1e-6
        assert abs(r2["pobj"] - r["pobj"]) <= 1e-5 * (1 + abs(r["pobj"]))


def test_batch_tail_handoff_matches_oracle():
    # with few LPs left every LP past 128 iterations is handed to the single-LP
    # path: same results as the oracle, flagged as handed off
    lps = _mixed_lps()
    B = P.Batch(lps)
    B.set_handoff(16, 128)
    reps = B.solve()
    handed = [B.handed_off(k) for k in range(len(lps))]
    assert sum(handed) >= 3
    for k, lp in enumerate(lps):
        ref = oracle.solve(lp)
        assert reps[k]["status_name"] == "OPTIMAL", k
        assert reps[k]["iters"] == ref["iters"] and reps[k]["restarts"] == ref["restarts"], k
        xo, yo, _ = oracle.unscale(ref["model"], ref["x_hat"], ref["y_hat"])
        x, y = B.get_solution(k)
        assert rel_err(x, xo) <= 1e-8 and rel_err(y, yo) <= 1e-8, k
    creps = B.corner_phase(obj_seed=11)
    for k, lp in enumerate(lps[:3]):
        ref1 = oracle.solve(lp)
        refc = oracle.corner_phase(ref1, dict(obj_seed=11))
        assert creps[k]["status"] == refc["status"] and creps[k]["iters"] == refc["iters"], k
        x, _ = B.get_solution(k, P.CORNER)
        xo, _, _ = oracle.unscale(ref1["model"], refc["x_hat"], refc["y_hat"])
        assert rel_err(x, xo) <= 1e-7, k


def test_batch_corner_row_rule_matches_the_single_lp_path():
    # the row_rule = 1 option inside the batched kernel equals the single-LP path's
    lps = _mixed_lps()[:3]
    B = P.Batch(lps)
    B.set_handoff(0)
    B.solve()
    creps = B.corner_phase(obj_seed=7, row_rule=1)
    for k, lp in enumerate(lps):
        g = P.lp_from_dict(lp)
        g.solve()
        rc = g.corner_phase(obj_seed=7, row_rule=1)
        assert creps[k]["status"] == rc["status"] and creps[k]["iters"] == rc["iters"], k
        xb, _ = B.get_solution(k, P.CORNER)
        xs, _, _ = g.get_solution(P.CORNER)
        assert rel_err(xb, xs) <= 1e-8, k


# ---------------------------------------------------------------------------
# The Halpern loop in the batched kernel (the same operators and decision as
# the single-LP Halpern path, one CTA per LP)
# ---------------------------------------------------------------------------
HP = dict(algorithm="halpern")


def test_batch_halpern_fp64_iterates_after_100_match_oracle():
    lps = _mixed_lps()
    B = P.Batch(lps)
    reps = B.solve(max_iters=100, eps_rel=-1.0, algorithm=P.HALPERN)
    for k, lp in enumerate(lps):
        ref = oracle.run_iterations(lp, 100, HP)
        assert reps[k]["status_name"] == "ITER_LIMIT" and reps[k]["iters"] == 100 and reps[k]["chosen"] == 2
        assert reps[k]["restarts"] == ref["restarts"], k
        # the returned point is T(z) of the last check
        xo, yo, _ = oracle.unscale(ref["model"], ref["x_hat"], ref["y_hat"])
        x, y = B.get_solution(k)
        assert rel_err(x, xo) <= 1e-10 and rel_err(y, yo) <= 1e-10, k
        assert abs(reps[k]["omega"] - ref["state"].omega) <= 1e-10 * ref["state"].omega, k


def test_batch_halpern_fp64_full_solves_and_corners_match_oracle():
    lps = _mixed_lps()
    B = P.Batch(lps)
    B.set_handoff(0)  # every LP to the end inside the batched kernel
    reps = B.solve(algorithm=P.HALPERN)
    refs = []
    for k, lp in enumerate(lps):
        ref = oracle.solve(lp, HP)
        refs.append(ref)
        assert reps[k]["status_name"] == "OPTIMAL" and ref["status"] == oracle.OPTIMAL, k
        assert reps[k]["iters"] == ref["iters"] and reps[k]["restarts"] == ref["restarts"], k
        assert reps[k]["rel_kkt"] <= 1e-6
        orep = oracle.kkt_report(ref["model"], ref["x_hat"], ref["y_hat"])
        for key in ("off_bound_p", "zero_rc_d", "candidates", "corner_measure"):
            assert reps[k][key] == orep[key], (k, key)
    creps = B.corner_phase(obj_seed=11)
    for k, lp in enumerate(lps[:4]):
        refc = oracle.corner_phase(refs[k], dict(obj_seed=11))
        assert creps[k]["status"] == refc["status"] == oracle.CORNER_DONE, k
        assert creps[k]["iters"] == refc["iters"] and creps[k]["restarts"] == refc["restarts"], k
        x, _ = B.get_solution(k, P.CORNER)
        xo, _, _ = oracle.unscale(refs[k]["model"], refc["x_hat"], refc["y_hat"])
        assert rel_err(x, xo) <= 1e-7, k


def test_batch_halpern_fp32_reaches_tolerance_and_corners():
    lps = _mixed_lps()
    B = P.Batch(lps)
    reps = B.solve(precision=P.FP32_BULK, algorithm=P.HALPERN)
    for k, r in enumerate(reps):
        assert r["status_name"] == "OPTIMAL" and r["rel_kkt"] <= 1e-6 and r["chosen"] == 2, (k, r["status_name"])
        ref = oracle.solve(lps[k], HP)
        assert abs(r["pobj"] - ref["eval"]["pobj"]) <= 1e-5 * (1 + abs(ref["eval"]["pobj"])), k
    creps = B.corner_phase(obj_seed=11)
    for k, r in enumerate(creps):
        assert r["status_name"] == "CORNER_DONE" and r["rel_p"] <= 1e-6 * (1 + 1e-9), (k, r["status_name"])


def test_batch_halpern_single_lp_path_agrees_on_handoff():
    # a handed-off LP finishes on the single-LP Halpern path: same counts
    lps = _mixed_lps()
    B = P.Batch(lps)
    B.set_handoff(16, 128)
    reps = B.solve(algorithm=P.HALPERN)
    assert sum(B.handed_off(k) for k in range(len(lps))) >= 3
    for k, lp in enumerate(lps):
        ref = oracle.solve(lp, HP)
        assert reps[k]["status_name"] == "OPTIMAL", k
        assert reps[k]["iters"] == ref["iters"] and reps[k]["restarts"] == ref["restarts"], k


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_fused_phases_equal_the_two_calls(precision):
    # pdhgc_batch_solve_corner (both phases per LP in one launch) gives the
    # reports and results of pdhgc_batch_solve followed by
    # pdhgc_batch_corner_phase: the per-LP work is the same, only the
    # batch-wide barrier between the phases is gone
    lps = _mixed_lps()
    prec = P.FP64 if precision == "fp64" else P.FP32_BULK
    params = P.default_params(algorithm=P.HALPERN, precision=prec)
    cparams = P.default_corner_params(obj_seed=11)
    B = P.Batch(lps)
    B.set_handoff(0)
    r1 = B.solve(params)
    rc = B.corner_phase(cparams)
    xs = [B.get_solution(k, P.CORNER)[0] for k in range(len(lps))]
    F = P.Batch(lps)
    F.set_handoff(0)
    f1, fc = F.solve_corner(params, cparams)
    for k in range(len(lps)):
        assert (f1[k]["status"], f1[k]["iters"], f1[k]["restarts"]) == (r1[k]["status"], r1[k]["iters"],
                                                                        r1[k]["restarts"]), k
        assert (fc[k]["status"], fc[k]["iters"], fc[k]["restarts"]) == (rc[k]["status"], rc[k]["iters"],
                                                                        rc[k]["restarts"]), k
        assert np.array_equal(F.get_solution(k, P.CORNER)[0], xs[k]), k
    # with handoffs: every LP still ends as the oracle's (FP64) and at a corner
    H = P.Batch(lps)
    H.set_handoff(16, 128)
    h1, hc = H.solve_corner(params, cparams)
    assert sum(H.handed_off(k) or H.handed_off(k, P.CORNER) for k in range(len(lps))) >= 3
    for k, lp in enumerate(lps):
        assert h1[k]["status_name"] == "OPTIMAL" and hc[k]["status_name"] == "CORNER_DONE", k
        if precision == "fp64":
            ref = oracle.solve(lp, HP)
            assert h1[k]["iters"] == ref["iters"], k
