"""The Halpern loop (PDHGC_ALG_HALPERN) of the CUDA path against the oracle's
(oracle.halpern), through the C-ABI (needs a GB300).

Same bar as the averaged loop: iterates after 100 steps to 1e-10 relative
(both sides run the same FP64 steps; they differ in rounding order only, and
the anchored combination z_0 + w (r - z_0) on the device is w r + (1 - w) z_0
in the oracle), equal iteration counts, restarts, statuses and metric counts.
"""
import numpy as np
import pytest

import lpgen
import oracle
from oracle import guide as oguide
from tests.test_gpu_parity import ITER_TOL, _lp_cases, rel_err

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2511_13894_gb300.pdhgc")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

HP = dict(algorithm="halpern")


@pytest.mark.parametrize("name", list(_lp_cases()))
def test_halpern_iterates_after_100_match_oracle(name):
    lp = _lp_cases()[name]()
    ref = oracle.run_iterations(lp, 100, HP)
    s = ref["state"]
    g = P.lp_from_dict(lp)
    rep = g.solve(max_iters=100, eps_rel=-1.0, algorithm=P.HALPERN)
    assert rep["status_name"] == "ITER_LIMIT" and rep["iters"] == 100 and rep["chosen"] == 2
    it = g.get_iterates()
    assert it["k"] == 100 and it["t"] == s.t and it["restarts"] == s.restarts
    assert s.restarts >= 1  # the first check always restarts (t = k)
    assert rel_err(it["x"], s.x) <= ITER_TOL
    assert rel_err(it["y"], s.y) <= ITER_TOL
    # the PDHG output of the last step, which the phase returns
    assert rel_err(it["x_avg"], s.xp) <= ITER_TOL
    assert rel_err(it["y_avg"], s.yp) <= ITER_TOL
    # the primal weight after the PID update(s)
    assert abs(g.get_scaling()["omega"] - s.omega) <= 1e-10 * s.omega


@pytest.mark.parametrize("name", ["face_200x500_s0", "bounded_ineq", "power_law_skewed", "transport_30x70"])
def test_halpern_full_solve_matches_oracle(name):
    lp = _lp_cases()[name]()
    ref = oracle.solve(lp, HP)
    g = P.lp_from_dict(lp)
    rep = g.solve(algorithm=P.HALPERN)
    assert rep["status_name"] == "OPTIMAL" and ref["status"] == oracle.OPTIMAL
    assert rep["iters"] == ref["iters"] and rep["restarts"] == ref["restarts"]
    assert rep["rel_kkt"] <= 1e-6
    x, y, z = g.get_solution()
    xo, yo, zo = oracle.unscale(ref["model"], ref["x_hat"], ref["y_hat"])
    assert rel_err(x, xo) <= 1e-8 and rel_err(y, yo) <= 1e-8 and rel_err(z, zo) <= 1e-8
    orep = oracle.kkt_report(ref["model"], ref["x_hat"], ref["y_hat"])
    for k in ("rP2", "rD2", "pobj", "dobj"):
        assert abs(rep[k] - orep[k]) <= 1e-7 * (1.0 + abs(orep[k])), k
    for k in ("off_bound_p", "zero_rc_d", "candidates", "corner_measure"):
        assert rep[k] == orep[k], k


@pytest.mark.parametrize("name", ["face_200x500_s0", "bounded_ineq"])
@pytest.mark.parametrize("row_rule", [0, 1])
def test_halpern_corner_phase_matches_oracle(name, row_rule):
    lp = _lp_cases()[name]()
    ref1 = oracle.solve(lp, HP)
    refc = oracle.corner_phase(ref1, dict(obj_seed=11, row_rule=row_rule))
    g = P.lp_from_dict(lp)
    g.solve(algorithm=P.HALPERN)
    rep = g.corner_phase(obj_seed=11, row_rule=row_rule)
    assert rep["status_name"] == "CORNER_DONE" and refc["status"] == oracle.CORNER_DONE
    assert rep["iters"] == refc["iters"] and rep["restarts"] == refc["restarts"]
    x, y, z = g.get_solution(P.CORNER)
    xo, yo, zo = oracle.unscale(ref1["model"], refc["x_hat"], refc["y_hat"])
    assert rel_err(x, xo) <= 1e-7
    orep = oracle.kkt_report(ref1["model"], refc["x_hat"], refc["y_hat"])
    for k in ("off_bound_p", "zero_rc_d", "candidates", "corner_measure", "primal_push_est"):
        assert rep[k] == orep[k], k


def test_halpern_corner_limit_keeps_the_phase1_point():
    lp = _lp_cases()["bounded_ineq"]()
    ref1 = oracle.solve(lp, HP)
    refc = oracle.corner_phase(ref1, dict(obj_seed=11, max_iters=128))
    g = P.lp_from_dict(lp)
    g.solve(algorithm=P.HALPERN)
    rep = g.corner_phase(obj_seed=11, max_iters=128)
    assert rep["status_name"] == "CORNER_LIMIT" and refc["status"] == oracle.CORNER_LIMIT
    x1 = g.get_solution(P.PHASE1)[0]
    assert np.array_equal(g.get_solution(P.CORNER)[0], x1)


def test_halpern_edge_shapes():
    one = dict(m=1, n=1, row_ptr=np.array([0, 1]), col_idx=np.array([0], dtype=np.int32), val=np.array([2.0]),
               b=np.array([3.0]), c=np.array([1.0]), lb=np.zeros(1), ub=np.full(1, np.inf),
               sense=np.array([oracle.EQ], dtype=np.int8))
    empty_row = dict(m=3, n=2, row_ptr=np.array([0, 2, 2, 3]), col_idx=np.array([0, 1, 1], dtype=np.int32),
                     val=np.array([1.0, 1.0, 1.0]), b=np.array([1.0, 0.0, 0.25]), c=np.array([1.0, 2.0]),
                     lb=np.zeros(2), ub=np.full(2, np.inf),
                     sense=np.array([oracle.EQ, oracle.EQ, oracle.GE], dtype=np.int8))
    no_nnz = dict(m=1, n=2, row_ptr=np.array([0, 0]), col_idx=np.zeros(0, dtype=np.int32), val=np.zeros(0),
                  b=np.array([0.0]), c=np.array([1.0, -1.0]), lb=np.array([0.0, -1.0]), ub=np.array([5.0, 2.0]),
                  sense=np.array([oracle.EQ], dtype=np.int8))
    for lp in (one, empty_row, no_nnz):
        ref = oracle.run_iterations(lp, 100, HP)
        g = P.lp_from_dict(lp)
        g.solve(max_iters=100, eps_rel=-1.0, algorithm=P.HALPERN)
        it = g.get_iterates()
        s = ref["state"]
        assert rel_err(it["x"], s.x) <= ITER_TOL and rel_err(it["y"], s.y) <= ITER_TOL
        full = oracle.solve(lp, HP)
        rep = P.lp_from_dict(lp).solve(algorithm=P.HALPERN)
        assert rep["status"] == full["status"] and rep["iters"] == full["iters"]


def test_halpern_restart_history_feeds_the_guidance_features():
    # the ring of restart points (T(z) at each restart) matches the oracle's
    lp = lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(5), 5)
    r1 = oracle.solve(lp, HP)
    g = P.lp_from_dict(lp)
    rep = g.solve(algorithm=P.HALPERN)
    assert rep["iters"] == r1["iters"] and rep["restarts"] == r1["restarts"]
    feat, elig = g.guide_features(obj_seed=7)
    F, E = oguide.features(r1, dict(obj_seed=7))
    bits = feat.view(torch.int16).cpu().numpy().view(np.uint16).astype(np.uint32) << 16
    got = bits.view(np.float32).astype(np.float64)[:, :18]
    assert np.all(np.abs(got - F) <= 2.0 ** -7 * np.abs(F) + 1e-30)
    assert np.array_equal(elig.cpu().numpy().astype(bool), E)


def test_halpern_refuses_bad_settings():
    lp = lpgen.small_face_lp(0)
    g = P.lp_from_dict(lp)
    with pytest.raises(P.PdhgcError, match="INVALID_ARG"):
        g.solve(algorithm=P.HALPERN, reflection=1.5)
    with pytest.raises(P.PdhgcError, match="INVALID_ARG"):
        g.solve(algorithm=7)
    B = P.Batch([lpgen.batch_lp(i) for i in range(2)])
    with pytest.raises(P.PdhgcError, match="INVALID_ARG"):
        B.solve(algorithm=P.HALPERN, reflection=-0.5)


def test_halpern_corner_phase_on_skewed_power_law_matches_oracle():
    # 3000 x 12000 with power-law columns up to 2000 nonzeros (warp and SELL
    # segments), '<' rows and upper bounds: the whole corner phase (about
    # 51k iterations) takes the oracle's iterations, restarts and counts
    lp = _lp_cases()["power_law_skewed"]()
    ref1 = oracle.solve(lp, HP)
    refc = oracle.corner_phase(ref1, dict(obj_seed=3))
    g = P.lp_from_dict(lp)
    r1 = g.solve(algorithm=P.HALPERN)
    assert r1["iters"] == ref1["iters"] and r1["restarts"] == ref1["restarts"]
    rep = g.corner_phase(obj_seed=3)
    assert rep["status_name"] == "CORNER_DONE" and refc["status"] == oracle.CORNER_DONE
    assert rep["iters"] == refc["iters"] and rep["restarts"] == refc["restarts"]
    x, _, _ = g.get_solution(P.CORNER)
    xo, _, _ = oracle.unscale(ref1["model"], refc["x_hat"], refc["y_hat"])
    assert rel_err(x, xo) <= 1e-7
    orep = oracle.kkt_report(ref1["model"], refc["x_hat"], refc["y_hat"])
    for k in ("off_bound_p", "zero_rc_d", "candidates", "corner_measure", "primal_push_est"):
        assert rep[k] == orep[k], k


# ---------------------------------------------------------------------------
# The Halpern loop in FP32 bulk: FP32 values and gathers, float-float
# iterates, anchors and row sums, FP64 checks.  No exact pin exists (a
# different rounding of the same map); results are judged by the FP64
# evaluation and by the distance to the FP64 oracle.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["face_200x500_s0", "bounded_ineq", "power_law_skewed", "transport_30x70"])
def test_halpern_fp32_bulk_reaches_the_fp64_tolerance(name):
    lp = _lp_cases()[name]()
    ref = oracle.solve(lp, HP)
    g = P.lp_from_dict(lp)
    rep = g.solve(algorithm=P.HALPERN, precision=P.FP32_BULK)
    print(f"{name}: Halpern FP32 bulk {rep['iters']} iterations, FP64 oracle {ref['iters']}")
    assert rep["status_name"] == "OPTIMAL" and rep["precision"] == P.FP32_BULK and rep["chosen"] == 2
    assert rep["rel_kkt"] <= 1e-6
    pobj = ref["eval"]["pobj"]
    assert abs(rep["pobj"] - pobj) <= 1e-5 * (1.0 + abs(pobj))
    x, _, _ = g.get_solution()
    assert np.all(x >= lp["lb"] - 1e-12 * np.abs(lp["lb"])) and np.all(x <= lp["ub"] + 1e-12 * np.abs(lp["ub"]))


def test_halpern_fp32_bulk_iterate_error_against_the_fp64_oracle():
    # the stated error of the FP32-bulk Halpern iterates z and T(z) against the
    # FP64 oracle at k = 100 and k = 1000 (max-norm, relative): FP32 rounding
    # of the matrix and the gathered vectors (about 6e-8) amplified by the map
    lp = _lp_cases()["power_law_skewed"]()
    for k, bound in ((100, 1e-4), (1000, 1e-2)):
        ref = oracle.run_iterations(lp, k, HP)
        s = ref["state"]
        g = P.lp_from_dict(lp)
        rep = g.solve(max_iters=k, eps_rel=-1.0, algorithm=P.HALPERN, precision=P.FP32_BULK)
        assert rep["iters"] == k
        it = g.get_iterates()
        errs = (rel_err(it["x"], s.x), rel_err(it["y"], s.y), rel_err(it["x_avg"], s.xp),
                rel_err(it["y_avg"], s.yp))
        print(f"Halpern FP32 bulk vs FP64 oracle at k={k}: x {errs[0]:.3e} y {errs[1]:.3e} "
              f"T(z)_x {errs[2]:.3e} T(z)_y {errs[3]:.3e}")
        assert max(errs) <= bound


@pytest.mark.parametrize("name", ["face_200x500_s0", "bounded_ineq", "power_law_skewed"])
def test_halpern_fp32_bulk_corner_phase(name):
    # the corner phase in FP32 bulk reaches Section 3.1's rule (CORNER_DONE);
    # its corner measure is stated beside the FP64 oracle's
    lp = _lp_cases()[name]()
    ref1 = oracle.solve(lp, HP)
    refc = oracle.corner_phase(ref1, dict(obj_seed=3))
    orep = oracle.kkt_report(ref1["model"], refc["x_hat"], refc["y_hat"])
    g = P.lp_from_dict(lp)
    g.solve(algorithm=P.HALPERN, precision=P.FP32_BULK)
    rep = g.corner_phase(obj_seed=3)
    print(f"{name}: FP32 corner {rep['iters']} iterations, measure {rep['corner_measure']}; "
          f"FP64 oracle {refc['iters']}, measure {orep['corner_measure']}")
    assert rep["status_name"] == "CORNER_DONE" and rep["chosen"] == 2
    assert rep["rel_p"] <= 1e-6 * (1 + 1e-9)
    assert rep["corner_measure"] <= orep["corner_measure"] + max(5, lp["m"] // 100)
    x, _, _ = g.get_solution(P.CORNER)
    assert np.all(x >= lp["lb"] - 1e-12 * np.abs(lp["lb"])) and np.all(x <= lp["ub"] + 1e-12 * np.abs(lp["ub"]))


@pytest.mark.parametrize("name", ["power_law_skewed", "dense_lines", "bounded_ineq"])
def test_halpern_primal_layouts_agree(name):
    # the primal pass over the row segments with global gathers (the
    # default) and with the gathered y staged in shared memory: the same
    # iterates up to the summation order, both within 1e-10 of the oracle
    lp = _lp_cases()[name]()
    ref = oracle.run_iterations(lp, 100, HP)
    s = ref["state"]
    its = []
    for chunked in (1, 0):
        g = P.lp_from_dict(lp)
        g.set_primal_layout(chunked)
        rep = g.solve(max_iters=100, eps_rel=-1.0, algorithm=P.HALPERN)
        assert rep["iters"] == 100 and rep["restarts"] == s.restarts
        it = g.get_iterates()
        assert rel_err(it["x"], s.x) <= ITER_TOL and rel_err(it["y"], s.y) <= ITER_TOL
        its.append(it)
    assert rel_err(its[0]["x"], its[1]["x"]) <= 1e-12 and rel_err(its[0]["y"], its[1]["y"]) <= 1e-12
    # FP32 bulk: both layouts reach the tolerance in about the same iterations
    reps = []
    for chunked in (1, 0):
        g = P.lp_from_dict(lp)
        g.set_primal_layout(chunked)
        reps.append(g.solve(algorithm=P.HALPERN, precision=P.FP32_BULK))
    for r in reps:
        assert r["status_name"] == "OPTIMAL" and r["rel_kkt"] <= 1e-6
    assert abs(reps[0]["iters"] - reps[1]["iters"]) <= max(256, reps[1]["iters"] // 10)
    with pytest.raises(P.PdhgcError, match="INVALID_ARG"):
        P._check(P.lib.pdhgc_set_primal_layout(g._h, 2), "pdhgc_set_primal_layout")


def test_halpern_profile_iteration_times_its_kernels():
    lp = lpgen.power_law_lp(3000, 12000, 500, seed=5, kmax=2000)
    g = P.lp_from_dict(lp)
    g.solve(algorithm=P.HALPERN)
    ms = g.profile_iteration(5)
    assert ms[0] > 0.0 and ms[1] > 0.0
    g.solve(algorithm=P.HALPERN, precision=P.FP32_BULK)
    ms = g.profile_iteration(5)
    assert ms[0] > 0.0 and ms[1] > 0.0


@pytest.mark.parametrize("alg", ["averaged", "halpern"])
@pytest.mark.parametrize("scale", [1e-6, 1e-2])
def test_corner_omega_rule_matches_oracle(alg, scale):
    # Section 5's objective-scale setting: the corner phase keeps phase 1's
    # primal weight (omega_rule 1) and the random objective is scaled
    lp = _lp_cases()["bounded_ineq"]()
    ref1 = oracle.solve(lp, dict(algorithm=alg))
    refc = oracle.corner_phase(ref1, dict(obj_seed=11, obj_scale=scale, omega_rule=1))
    g = P.lp_from_dict(lp)
    g.solve(algorithm=P.HALPERN if alg == "halpern" else P.AVERAGED)
    rep = g.corner_phase(obj_seed=11, obj_scale=scale, omega_rule=1)
    assert rep["status_name"] == "CORNER_DONE" and refc["status"] == oracle.CORNER_DONE
    assert rep["iters"] == refc["iters"] and rep["restarts"] == refc["restarts"]
    assert abs(rep["omega"] - refc["state"].omega) <= 1e-9 * refc["state"].omega
    x, y, z = g.get_solution(P.CORNER)
    xo, yo, zo = oracle.unscale(ref1["model"], refc["x_hat"], refc["y_hat"])
    assert rel_err(x, xo) <= 1e-7
    orep = oracle.kkt_report(ref1["model"], refc["x_hat"], refc["y_hat"])
    for k in ("off_bound_p", "zero_rc_d", "candidates", "corner_measure", "primal_push_est"):
        assert rep[k] == orep[k], k
    with pytest.raises(P.PdhgcError, match="INVALID_ARG"):
        g.corner_phase(obj_seed=11, omega_rule=2)


def test_halpern_checkpoint_restore_resumes_at_the_corner_phase():
    # the state carries the parameters (the inner loop among them): a restored
    # handle runs the corner phase in the Halpern loop, bit for bit as the
    # original handle does
    lp = _lp_cases()["bounded_ineq"]()
    g = P.lp_from_dict(lp)
    r1 = g.solve(algorithm=P.HALPERN)
    state = g.get_state()
    c_orig = g.corner_phase(obj_seed=5)
    x_orig, _, _ = g.get_solution(P.CORNER)
    h = P.lp_from_dict(lp)
    h.set_state(state)
    assert h.kkt_report(P.PHASE1)["rel_kkt"] == r1["rel_kkt"]
    c_rest = h.corner_phase(obj_seed=5)
    assert c_rest["iters"] == c_orig["iters"] and c_rest["chosen"] == c_orig["chosen"] == 2
    x_rest, _, _ = h.get_solution(P.CORNER)
    assert np.array_equal(x_rest, x_orig)
