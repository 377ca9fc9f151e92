"""The two loop drivers (pdhgc_set_launch_mode) make the same decisions: a
phase run as plain stream launches, one body at a time with the done flag
read back by the host, gives bitwise the results of the conditional-WHILE
graph, in both inner loops and both precisions, and counts the same kernel
launches (needs a GB300)."""
import numpy as np
import pytest

import lpgen

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2511_13894_gb300.pdhgc")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _run(lp, mode, algorithm, precision):
    g = P.lp_from_dict(lp)
    g.set_launch_mode(mode)
    l0 = g.kernel_launches()
    r1 = g.solve(algorithm=algorithm, precision=precision)
    rc = g.corner_phase(obj_seed=3)
    x1, y1, _ = g.get_solution(P.PHASE1)
    xc, yc, _ = g.get_solution(P.CORNER)
    launches = g.kernel_launches() - l0
    g.close()
    return r1, rc, (x1, y1, xc, yc), launches


@pytest.mark.parametrize("algorithm", ["halpern", "averaged"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_stream_mode_equals_graph_mode(algorithm, precision):
    lp = lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(3), 3)
    alg = P.HALPERN if algorithm == "halpern" else P.AVERAGED
    prec = P.FP64 if precision == "fp64" else P.FP32_BULK
    g1, gc, gv, gl = _run(lp, P.LAUNCH_GRAPH, alg, prec)
    s1, sc, sv, sl = _run(lp, P.LAUNCH_STREAM, alg, prec)
    for a, b in ((g1, s1), (gc, sc)):
        assert a["status_name"] == b["status_name"]
        assert a["iters"] == b["iters"] and a["restarts"] == b["restarts"]
        assert a["corner_measure"] == b["corner_measure"]
    assert g1["status_name"] == "OPTIMAL" and gc["status_name"] == "CORNER_DONE"
    for a, b in zip(gv, sv):
        assert np.array_equal(a, b)
    assert gl == sl > 0


def test_bad_launch_mode_is_refused():
    g = P.lp_from_dict(lpgen.small_face_lp(0))
    with pytest.raises(P.PdhgcError, match="INVALID_ARG"):
        g.set_launch_mode(2)
    g.close()
