"""CUDA path vs the CPU oracle, through the C-ABI (needs a GB300).

Tolerances: iterates after 100 iterations agree to 1e-10 relative (max-norm
error over max(1, max-norm of the oracle's vector)): both sides run the
same FP64 algorithm and differ only in rounding order (FMA contraction,
row-sum order, 1/t versus division), which stays near 1e-14 after 100
contractive PDHG steps.  Integer results (iteration counts, restarts,
status, metric counts) must be equal.
"""
import numpy as np
import pytest

import lpgen
import oracle

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2511_13894_gb300.pdhgc")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ITER_TOL = 1e-10


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    if b.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


def _lp_cases():
    return {
        "face_200x500_s0": lambda: lpgen.small_face_lp(0),
        "face_200x500_s7": lambda: lpgen.small_face_lp(7),
        "bounded_ineq": lambda: lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(3), 3),
        "power_law_skewed": lambda: lpgen.power_law_lp(3000, 12000, 500, seed=5, kmax=2000),
        "transport_30x70": lambda: lpgen.transportation_lp(30, 70, seed=2),
        "tiny_5x11": lambda: lpgen.tiny_face_lp(5, 11, 7, seed=101),
        # one row of A with 4500 nonzeros and one column with 4150: both
        # matrix passes run their one-CTA-per-row segment
        "dense_lines": lambda: lpgen.dense_line_lp(4200, 12000, 4500, 4150, 400, seed=2, col_nnz=3),
    }


@pytest.mark.parametrize("name", list(_lp_cases()))
def test_iterates_after_100_match_oracle(name):
    lp = _lp_cases()[name]()
    ref = oracle.run_iterations(lp, 100)
    s = ref["state"]
    g = P.lp_from_dict(lp)
    rep = g.solve(max_iters=100, eps_rel=-1.0)
    assert rep["status_name"] == "ITER_LIMIT" and rep["iters"] == 100
    it = g.get_iterates()
    assert it["k"] == 100 and it["t"] == s.t and it["restarts"] == s.restarts
    xa, ya = s.average()
    assert rel_err(it["x"], s.x) <= ITER_TOL
    assert rel_err(it["y"], s.y) <= ITER_TOL
    assert rel_err(it["x_avg"], xa) <= ITER_TOL
    assert rel_err(it["y_avg"], ya) <= ITER_TOL
    sc = g.get_scaling()
    model = ref["model"]
    assert rel_err(sc["Dr"], model.Dr) <= 1e-13
    assert rel_err(sc["Dc"], model.Dc) <= 1e-13
    assert abs(sc["sigma_max"] - ref["sigma_max"]) <= 1e-12 * ref["sigma_max"]
    assert abs(sc["omega"] - s.omega) <= 1e-10 * s.omega


@pytest.mark.parametrize("name", ["face_200x500_s0", "bounded_ineq", "power_law_skewed", "transport_30x70"])
def test_full_solve_matches_oracle(name):
    lp = _lp_cases()[name]()
    ref = oracle.solve(lp)
    g = P.lp_from_dict(lp)
    rep = g.solve()
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
def test_corner_phase_matches_oracle(name):
    lp = _lp_cases()[name]()
    ref1 = oracle.solve(lp)
    refc = oracle.corner_phase(ref1, dict(obj_seed=11))
    g = P.lp_from_dict(lp)
    g.solve()
    rep = g.corner_phase(obj_seed=11)
    assert rep["status_name"] == "CORNER_DONE" and refc["status"] == oracle.CORNER_DONE
    assert rep["iters"] == refc["iters"] and rep["restarts"] == refc["restarts"]
    x, y, z = g.get_solution(P.CORNER)
    xo, yo, zo = oracle.unscale(ref1["model"], refc["x_hat"], refc["y_hat"])
    assert rel_err(x, xo) <= 1e-7
    orep = oracle.kkt_report(ref1["model"], refc["x_hat"], refc["y_hat"])
    for k in ("off_bound_p", "zero_rc_d", "candidates", "corner_measure", "primal_push_est"):
        assert rep[k] == orep[k], k


def test_uniform_objective_is_bitwise_equal():
    for seed, n in [(0, 1), (1234567, 1000), (2**63 + 5, 4099)]:
        got = P.uniform(seed, n).cpu().numpy()
        ref = oracle.splitmix64_uniform(seed, n)
        assert np.array_equal(got, ref)


def test_edge_shapes():
    # 1 x 1; an empty column; an empty row with b = 0; nnz = 0
    one = dict(m=1, n=1, row_ptr=np.array([0, 1]), col_idx=np.array([0], dtype=np.int32), val=np.array([2.0]),
               b=np.array([3.0]), c=np.array([1.0]), lb=np.zeros(1), ub=np.full(1, np.inf),
               sense=np.array([oracle.EQ], dtype=np.int8))
    empty_col = dict(m=2, n=3, row_ptr=np.array([0, 2, 4]), col_idx=np.array([0, 2, 0, 2], dtype=np.int32),
                     val=np.array([1.0, 1.0, 1.0, -1.0]), b=np.array([2.0, 0.0]), c=np.array([1.0, 5.0, 1.0]),
                     lb=np.zeros(3), ub=np.array([np.inf, 4.0, np.inf]),
                     sense=np.array([oracle.EQ, oracle.EQ], dtype=np.int8))
    empty_row = dict(m=3, n=2, row_ptr=np.array([0, 2, 2, 3]), col_idx=np.array([0, 1, 1], dtype=np.int32),
                     val=np.array([1.0, 1.0, 1.0]), b=np.array([1.0, 0.0, 0.25]), c=np.array([1.0, 2.0]),
                     lb=np.zeros(2), ub=np.full(2, np.inf),
                     sense=np.array([oracle.EQ, oracle.EQ, oracle.GE], dtype=np.int8))
    no_nnz = dict(m=1, n=2, row_ptr=np.array([0, 0]), col_idx=np.zeros(0, dtype=np.int32), val=np.zeros(0),
                  b=np.array([0.0]), c=np.array([1.0, -1.0]), lb=np.array([0.0, -1.0]), ub=np.array([5.0, 2.0]),
                  sense=np.array([oracle.EQ], dtype=np.int8))
    for lp in (one, empty_col, empty_row, no_nnz):
        ref = oracle.run_iterations(lp, 100)
        g = P.lp_from_dict(lp)
        g.solve(max_iters=100, eps_rel=-1.0)
        it = g.get_iterates()
        s = ref["state"]
        assert rel_err(it["x"], s.x) <= ITER_TOL and rel_err(it["y"], s.y) <= ITER_TOL
        full = oracle.solve(lp)
        rep = P.lp_from_dict(lp).solve()
        assert rep["status"] == full["status"] and rep["iters"] == full["iters"]


def test_device_inputs_and_errors():
    lp = lpgen.small_face_lp(2)
    g = P.lp_from_dict(lp, device=True)
    rep = g.solve(max_iters=100, eps_rel=-1.0)
    h = P.lp_from_dict(lp)
    rep2 = h.solve(max_iters=100, eps_rel=-1.0)
    assert np.array_equal(g.get_iterates()["x"], h.get_iterates()["x"])  # deterministic
    x_dev, _, _ = g.get_solution(device=True)
    assert x_dev.is_cuda
    with pytest.raises(P.PdhgcError):
        g.corner_phase(stop_rule=7)
    with pytest.raises(P.PdhgcError):
        P.lp_from_dict(lp).corner_phase()  # no phase 1
    bad = dict(lp)
    bad["lb"] = lp["lb"].copy()
    bad["lb"][3] = 5.0
    bad["ub"] = lp["ub"].copy()
    bad["ub"][3] = 1.0
    with pytest.raises(P.PdhgcError) as ei:
        P.lp_from_dict(bad)
    assert ei.value.code == -4
    assert rep["iters"] == rep2["iters"] == 100


def test_iteration_and_time_limits_stop_the_device_loop():
    lp = lpgen.small_face_lp(4)
    g = P.lp_from_dict(lp)
    rep = g.solve(max_iters=130, eps_rel=1e-14)
    assert rep["status_name"] == "ITER_LIMIT" and rep["iters"] == 130
    rep = g.solve(max_iters=10**9, eps_rel=1e-300, time_limit_s=0.05)
    assert rep["status_name"] == "TIME_LIMIT"
    assert rep["seconds"] < 5.0


@pytest.mark.parametrize("name", ["face_200x500_s0", "bounded_ineq", "power_law_skewed"])
def test_kkt_eval_of_a_point_matches_oracle(name):
    # the oracle's phase-1 point, evaluated on the GPU without a handle
    lp = _lp_cases()[name]()
    ref = oracle.solve(lp, dict(max_iters=640))
    model = ref["model"]
    x, y, _ = oracle.unscale(model, ref["x_hat"], ref["y_hat"])
    orep = oracle.kkt_report(model, ref["x_hat"], ref["y_hat"])
    rep = P.kkt_eval(lp, x, y)
    scale = 1.0 + float(np.linalg.norm(lp["b"])) + float(np.linalg.norm(lp["c"]))
    for k in ("rP2", "rD2", "rPinf", "rDinf", "pobj", "dobj", "gap"):
        assert abs(rep[k] - orep[k]) <= 1e-9 * (scale + abs(orep[k])), (k, rep[k], orep[k])
    for k in ("rel_p", "rel_d", "rel_gap"):
        assert abs(rep[k] - orep[k]) <= 1e-9 * (1.0 + abs(orep[k])), k
    for k in ("off_bound_p", "zero_rc_d", "candidates", "corner_measure", "primal_push_est", "dual_push_est"):
        assert rep[k] == orep[k], k
    # the constructed optimum is optimal: every residual and the gap vanish
    rep = P.kkt_eval(lp, lp["x_star"], lp["y_star"])
    assert rep["rel_kkt"] <= 1e-12


@pytest.mark.parametrize("alg", ["averaged", "halpern"])
def test_dense_lines_run_the_cta_segment_and_match_oracle(alg):
    # rows longer than 4096 nonzeros (in A and in A') go to the one-CTA-per-row
    # segment; the full solve takes the oracle's iterations and restarts
    lp = _lp_cases()["dense_lines"]()
    g = P.lp_from_dict(lp)
    lay = g.get_layout()
    assert lay["A"]["nb_cta"] >= 1 and lay["AT"]["nb_cta"] >= 1, lay
    ref = oracle.solve(lp, dict(algorithm=alg))
    rep = g.solve(algorithm=P.HALPERN if alg == "halpern" else P.AVERAGED)
    assert rep["status_name"] == "OPTIMAL" and ref["status"] == oracle.OPTIMAL
    assert rep["iters"] == ref["iters"] and rep["restarts"] == ref["restarts"]
    x, y, z = g.get_solution()
    xo, yo, zo = oracle.unscale(ref["model"], ref["x_hat"], ref["y_hat"])
    assert rel_err(x, xo) <= 1e-8 and rel_err(y, yo) <= 1e-8
    orep = oracle.kkt_report(ref["model"], ref["x_hat"], ref["y_hat"])
    for k in ("off_bound_p", "zero_rc_d", "candidates", "corner_measure"):
        assert rep[k] == orep[k], k
    # FP32 bulk through the same segments.  In the averaged loop the FP32
    # map's fixed point is the optimum of the LP with FP32-rounded scaled
    # coefficients: on the 4500-entry row that rounding (2^-24 relative per
    # value) leaves an FP64 relative primal residual of about 2e-6, so its
    # stated bound here is 1e-5.  The Halpern loop's FP32 kernels gather and
    # multiply only differences from the anchor, with c - A'y_0 and b - A x_0
    # formed in FP64 at each anchor: its fixed point is the FP64 LP's, and
    # it meets 1e-6 in the FP64 loop's iterations.
    r32 = g.solve(algorithm=P.HALPERN if alg == "halpern" else P.AVERAGED, precision=P.FP32_BULK,
                  max_iters=200_000)
    print(f"dense lines, {alg} FP32 bulk: {r32['status_name']} after {r32['iters']} iterations, "
          f"rel_p {r32['rel_p']:.2e} rel_d {r32['rel_d']:.2e} rel_gap {r32['rel_gap']:.2e}")
    if alg == "halpern":
        assert r32["status_name"] == "OPTIMAL" and r32["rel_kkt"] <= 1e-6
        assert abs(r32["iters"] - ref["iters"]) <= max(640, ref["iters"] // 10)
    else:
        assert r32["rel_kkt"] <= 1e-5
    assert abs(r32["pobj"] - orep["pobj"]) <= 1e-5 * (1.0 + abs(orep["pobj"]))


# ---------------------------------------------------------------------------
# FP32 bulk (FP32 matrix and iterates, float-float row sums, FP64 KKT)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["face_200x500_s0", "bounded_ineq", "power_law_skewed", "transport_30x70"])
def test_fp32_bulk_reaches_the_fp64_tolerance(name):
    # no exact pin: the FP32 iteration is a different rounding of the same
    # map; its result is judged by the FP64 KKT numbers and by the distance
    # to the FP64 oracle's optimum
    lp = _lp_cases()[name]()
    g = P.lp_from_dict(lp)
    rep = g.solve(precision=P.FP32_BULK)
    assert rep["status_name"] == "OPTIMAL", rep
    assert rep["precision"] == P.FP32_BULK
    assert rep["rel_kkt"] <= 1e-6
    full = oracle.solve(lp)
    assert abs(rep["pobj"] - full["eval"]["pobj"]) <= 1e-5 * (1.0 + abs(full["eval"]["pobj"]))
    x, _, _ = g.get_solution()
    assert np.all(x >= lp["lb"] - 1e-12 * np.abs(lp["lb"])) and np.all(x <= lp["ub"] + 1e-12 * np.abs(lp["ub"]))


def test_fp32_bulk_iterate_error_against_the_fp64_oracle():
    # the stated error of the FP32-bulk iterates against the FP64 oracle:
    # at k = 100 the max-norm relative error stays at the level of FP32
    # rounding of the inputs (about 1e-7) amplified by the iteration
    lp = lpgen.power_law_lp(3000, 12000, 500, seed=5, kmax=2000)
    for k, bound in ((100, 1e-4), (1000, 1e-2)):
        ref = oracle.run_iterations(lp, k)
        s = ref["state"]
        g = P.lp_from_dict(lp)
        g.solve(max_iters=k, eps_rel=-1.0, precision=P.FP32_BULK)
        it = g.get_iterates()
        ex, ey = rel_err(it["x"], s.x), rel_err(it["y"], s.y)
        print(f"FP32 bulk vs FP64 oracle at k={k}: x {ex:.3e}, y {ey:.3e}")
        assert ex <= bound and ey <= bound


def test_fp32_bulk_corner_phase():
    lp = _lp_cases()["face_200x500_s0"]()
    g = P.lp_from_dict(lp)
    g.solve(precision=P.FP32_BULK)
    rep = g.corner_phase(obj_seed=11)
    assert rep["status_name"] == "CORNER_DONE"
    assert rep["rel_p"] <= 1e-6 * (1 + 1e-9)


def test_fp32_bulk_converges_where_small_steps_underflow():
    # LP 199 of the 512-LP batch: its primal weight falls to ~1e-3, so the dual
    # step sigma * r drops below an FP32 unit of y; the float-float iterates
    # keep those steps (plain FP32 iterates stalled at rel-KKT 1e-1 here)
    lp = lpgen.batch_lp(199)
    g = P.lp_from_dict(lp)
    r64 = g.solve()
    r32 = g.solve(precision=P.FP32_BULK, max_iters=200_000)
    assert r64["status_name"] == "OPTIMAL"
    assert r32["status_name"] == "OPTIMAL" and r32["rel_kkt"] <= 1e-6, (r32["status_name"], r32["rel_kkt"])
    assert abs(r32["pobj"] - r64["pobj"]) <= 1e-5 * (1 + abs(r64["pobj"]))


def test_corner_row_rule_option_matches_oracle():
    # the option that keeps rows inactive at the phase-1 point as inequalities
    lp = _lp_cases()["bounded_ineq"]()
    ref1 = oracle.solve(lp)
    refc = oracle.corner_phase(ref1, dict(obj_seed=11, row_rule=1))
    g = P.lp_from_dict(lp)
    g.solve()
    rep = g.corner_phase(obj_seed=11, row_rule=1)
    assert rep["status"] == refc["status"] and rep["iters"] == refc["iters"]
    x, _, _ = g.get_solution(P.CORNER)
    xo, _, _ = oracle.unscale(ref1["model"], refc["x_hat"], refc["y_hat"])
    assert rel_err(x, xo) <= 1e-7


def test_checkpoint_restore_resumes_at_the_corner_phase():
    lp = _lp_cases()["bounded_ineq"]()
    g = P.lp_from_dict(lp)
    r1 = g.solve()
    state = g.get_state()
    c_orig = g.corner_phase(obj_seed=5)
    x_orig, _, _ = g.get_solution(P.CORNER)
    h = P.lp_from_dict(lp)
    h.set_state(state)
    assert h.kkt_report(P.PHASE1)["rel_kkt"] == r1["rel_kkt"]
    x1a, y1a, _ = g.get_solution(P.PHASE1)
    x1b, y1b, _ = h.get_solution(P.PHASE1)
    assert np.array_equal(x1a, x1b) and np.array_equal(y1a, y1b)
    c_rest = h.corner_phase(obj_seed=5)
    assert c_rest["iters"] == c_orig["iters"]
    x_rest, _, _ = h.get_solution(P.CORNER)
    assert np.array_equal(x_rest, x_orig)
    # a state of another LP is refused
    other = P.lp_from_dict(lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(4), 4))
    with pytest.raises(P.PdhgcError) as e:
        other.set_state(state)
    assert e.value.code == -1


def test_checkpoint_restore_fp32_bulk():
    lp = _lp_cases()["power_law_skewed"]()
    g = P.lp_from_dict(lp)
    g.solve(precision=P.FP32_BULK)
    state = g.get_state()
    c_orig = g.corner_phase(obj_seed=2, max_iters=20000)
    h = P.lp_from_dict(lp)
    h.set_state(state)
    c_rest = h.corner_phase(obj_seed=2, max_iters=20000)
    assert c_rest["iters"] == c_orig["iters"] and c_rest["status"] == c_orig["status"]
    xa, _, _ = g.get_solution(P.CORNER)
    xb, _, _ = h.get_solution(P.CORNER)
    assert np.array_equal(xa, xb)


def test_gather_probe_reports_a_plausible_rate():
    ms = P.probe_gather(100_000, 3_206_827, 8, reps=5)
    rate = 3_206_827 / (ms * 1e-3)
    assert 1e9 < rate < 1e13
    with pytest.raises(P.PdhgcError):
        P.probe_gather(0, 10, 8)
