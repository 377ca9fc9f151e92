"""Actual push counts of the CUDA path's results (needs a GB300): the
crossover-lite measurement tool (oracle/crossover.py, on the CPU) takes the
GPU phase-1, corner and dual corner results and counts the primal pushes and
the dual superbasics a crossover would start from: the synthetic analogue of
the paper's Figure 2 (primal pushes after / before the corner push), and its
dual counterpart for the dual corner push."""
import numpy as np
import pytest

import lpgen
from oracle import crossover as X

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2511_13894_gb300.pdhgc")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_corner_push_removes_the_primal_pushes(precision):
    lp = lpgen.small_face_lp(0)   # |S| = m + 50: 50 primal superbasics at the optimum
    g = P.lp_from_dict(lp)
    prec = P.FP64 if precision == "fp64" else P.FP32_BULK
    g.solve(algorithm=P.HALPERN, precision=prec)
    x1, y1, z1 = g.get_solution(P.PHASE1)
    before = X.crossover_lite(lp, x1, y1, z1)
    g.corner_phase(obj_seed=1)
    xc, _, _ = g.get_solution(P.CORNER)
    after = X.crossover_lite(lp, xc, y1, z1)
    print(f"{precision}: primal pushes {before['primal_pushes']} -> {after['primal_pushes']} "
          f"(estimates {before['primal_push_est']} -> {after['primal_push_est']})")
    assert before["primal_pushes"] == 50 and after["primal_pushes"] == 0


def test_dual_corner_push_removes_the_dual_superbasics():
    lp = lpgen.random_face_lp(200, 500, 150, seed=3)   # a 50-dimensional dual optimal face
    g = P.lp_from_dict(lp)
    g.solve(algorithm=P.HALPERN, eps_rel=1e-9)
    x1, y1, z1 = g.get_solution(P.PHASE1)
    before = X.crossover_lite(lp, x1, y1, z1, push=False)
    g.dual_corner_phase(obj_seed=5, stop_rule=1, eps_rel=1e-9, max_iters=400_000)
    xd, yd, zd = g.get_solution(P.DUAL_CORNER)
    after = X.crossover_lite(lp, xd, yd, zd, push=False)
    print(f"dual superbasics {before['dual_superbasics']} -> {after['dual_superbasics']} "
          f"(estimates {before['dual_push_est']} -> {after['dual_push_est']})")
    assert before["dual_push_est"] == 50 and before["dual_superbasics"] == 50
    assert after["dual_push_est"] == 0 and after["dual_superbasics"] == 0
    assert np.array_equal(xd, x1)
