"""The dual corner push (pdhgc_dual_corner_phase) of the CUDA path against
the oracle (oracle.pdhg.dual_corner_phase, oracle.halpern.dual_corner_phase)
through the C-ABI (needs a GB300).  The device fixes the dual of an inactive
row by a right-hand side of -1e30 (the projection then returns 0); the
oracle zeroes it explicitly: two independent forms of the same model.
Same bar as the other phases: iterates after 100 steps to 1e-10, equal
iteration and restart counts, statuses and metric counts."""
import numpy as np
import pytest

import lpgen
import oracle
from tests.test_gpu_parity import ITER_TOL, rel_err

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2511_13894_gb300.pdhgc")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _cases():
    return {
        "face_dual_200x500": lambda: lpgen.random_face_lp(200, 500, 150, seed=3),
        "bounded_ineq_dual": lambda: lpgen.with_bounds_and_inequalities(
            lpgen.random_face_lp(200, 500, 150, seed=3), 3),
    }


ALG = {"averaged": P.AVERAGED, "halpern": P.HALPERN}


@pytest.mark.parametrize("alg", list(ALG))
@pytest.mark.parametrize("name", list(_cases()))
def test_dual_corner_iterates_and_counts_match_oracle(alg, name):
    lp = _cases()[name]()
    ref1 = oracle.solve(lp, dict(algorithm=alg, eps_rel=1e-9))
    g = P.lp_from_dict(lp)
    r1 = g.solve(algorithm=ALG[alg], eps_rel=1e-9)
    assert r1["iters"] == ref1["iters"] and r1["restarts"] == ref1["restarts"]
    # 100 dual corner steps (the limit keeps y1; compare the model's iterates)
    refk = oracle.dual_corner_phase(ref1, dict(obj_seed=5, max_iters=100))
    g.dual_corner_phase(obj_seed=5, max_iters=100)
    it = g.get_iterates()
    s = refk["state"]
    assert it["k"] == 100 and it["restarts"] == s.restarts
    assert rel_err(it["x"], s.x) <= ITER_TOL and rel_err(it["y"], s.y) <= ITER_TOL
    # the default rule (dual residual regained): the oracle's iterations,
    # restarts, point and counts
    ref = oracle.dual_corner_phase(ref1, dict(obj_seed=5))
    rep = g.dual_corner_phase(obj_seed=5)
    assert rep["status_name"] == "CORNER_DONE" and ref["status"] == oracle.CORNER_DONE
    assert rep["iters"] == ref["iters"] and rep["restarts"] == ref["restarts"]
    x, y, z = g.get_solution(P.DUAL_CORNER)
    xo, yo, zo = oracle.unscale(ref1["model"], ref["x_hat"], ref["y_hat"])
    assert rel_err(x, xo) <= 1e-8 and rel_err(y, yo) <= 1e-7 and rel_err(z, zo) <= 1e-7
    orep = oracle.kkt_report(ref1["model"], ref["x_hat"], ref["y_hat"])
    for k in ("zero_rc_d", "dual_push_est", "off_bound_p", "candidates"):
        assert rep[k] == orep[k], k
    # the full test at 1e-9: over ~10^4 iterations at that tolerance the
    # rounding order may move a restart by a check, so the runs are compared
    # where the result is unique: both end at the same vertex of the dual
    # optimal face, with m zero reduced costs
    ref = oracle.dual_corner_phase(ref1, dict(obj_seed=5, stop_rule="kkt", eps_rel=1e-9, max_iters=400_000))
    rep = g.dual_corner_phase(obj_seed=5, stop_rule=1, eps_rel=1e-9, max_iters=400_000)
    print(f"{name} {alg}: converged dual corner {rep['iters']} iterations (oracle {ref['iters']})")
    assert rep["status_name"] == "CORNER_DONE" and ref["status"] == oracle.CORNER_DONE
    assert abs(rep["iters"] - ref["iters"]) <= max(640, ref["iters"] // 5)
    _, y, z = g.get_solution(P.DUAL_CORNER)
    _, yo, zo = oracle.unscale(ref1["model"], ref["x_hat"], ref["y_hat"])
    assert rel_err(y, yo) <= 1e-6 and rel_err(z, zo) <= 1e-6
    orep = oracle.kkt_report(ref1["model"], ref["x_hat"], ref["y_hat"])
    assert rep["zero_rc_d"] == orep["zero_rc_d"] >= lp["m"] and rep["dual_push_est"] == 0
    assert g.kkt_report(P.DUAL_CORNER)["zero_rc_d"] == rep["zero_rc_d"]


def test_dual_corner_fp32_bulk_and_limits():
    # FP32 bulk (Halpern loop): the dual corner phase regains dual
    # feasibility (its stop rule) and keeps the fixed duals at 0; the counts
    # are stated beside phase 1's
    lp = _cases()["bounded_ineq_dual"]()
    g = P.lp_from_dict(lp)
    r1 = g.solve(algorithm=P.HALPERN, precision=P.FP32_BULK)
    rep = g.dual_corner_phase(obj_seed=5)
    print(f"FP32 bulk: phase 1 {r1['status_name']} {r1['iters']} (d {r1['zero_rc_d']}), dual corner "
          f"{rep['status_name']} {rep['iters']} (d {rep['zero_rc_d']}, rel_d {rep['rel_d']:.1e})")
    assert r1["status_name"] == "OPTIMAL"
    assert rep["status_name"] == "CORNER_DONE" and rep["precision"] == P.FP32_BULK
    assert rep["rel_d"] <= 1e-6 * (1 + 1e-9) and rep["rel_p"] == r1["rel_p"]
    ref1 = oracle.solve(lp, dict(algorithm="halpern"))
    dm, _ = oracle.dual_corner_model(ref1["model"], ref1["x_hat"], ref1["y_hat"], dict(oracle.CORNER_DEFAULTS))
    _, y, _ = g.get_solution(P.DUAL_CORNER)
    rows_zero = dm.y_zero  # the oracle keeps the user's row order
    assert rows_zero.any() and np.all(y[rows_zero] == 0.0)
    # a limit keeps phase 1's dual
    lim = g.dual_corner_phase(obj_seed=5, max_iters=64)
    assert lim["status_name"] == "CORNER_LIMIT"
    assert np.array_equal(g.get_solution(P.DUAL_CORNER)[1], g.get_solution(P.PHASE1)[1])
    with pytest.raises(P.PdhgcError, match="INVALID_ARG"):
        g.dual_corner_phase(row_rule=1)
    h = P.lp_from_dict(lp)
    with pytest.raises(P.PdhgcError, match="NO_PHASE1"):
        h.dual_corner_phase()
    h.solve(algorithm=P.HALPERN)
    with pytest.raises(P.PdhgcError, match="NO_CORNER"):
        h.get_solution(P.DUAL_CORNER)
