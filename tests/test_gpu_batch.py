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
