"""The benchmark's headline workload is the recipe the design notes state
(no GPU): power_law_m100k_n400k with nnz 3,206,827, alpha 1.855 for mean 8,
one column of 2000, half the rows '<', about 20% of the columns bounded,
|S| = m + 5000, and a constructed optimum that satisfies its own
optimality conditions (primal feasible, complementary, dual feasible)."""
import numpy as np
import pytest

import bench
import lpgen

EQ, LE = ord("="), ord("<")


@pytest.fixture(scope="module")
def lp():
    return bench.WORKLOADS["power_law_m100k_n400k"]()


def test_shape_and_structure(lp):
    m, n = lp["m"], lp["n"]
    assert (m, n, int(lp["row_ptr"][-1])) == (100_000, 400_000, 3_206_827)
    assert abs(lp["alpha"] - 1.855) < 5e-4
    col_counts = np.bincount(lp["col_idx"], minlength=n)
    assert col_counts.max() == 2000 and col_counts.min() >= 1
    assert abs(col_counts.mean() - 8.0) < 0.05
    assert np.all(np.diff(lp["row_ptr"]) >= 1)  # no empty row
    assert np.all(lp["sense"][: m // 2] == EQ) and np.all(lp["sense"][m // 2:] == LE)
    bounded = np.isfinite(lp["ub"])
    assert abs(bounded.mean() - 0.2) < 0.005
    assert np.all((lp["ub"][bounded] >= 1.0) & (lp["ub"][bounded] <= 10.0)) and np.all(lp["lb"] == 0.0)
    assert len(lp["support"]) == m + 5000


def test_constructed_optimum_is_optimal(lp):
    m, n = lp["m"], lp["n"]
    x, y, z = lp["x_star"], lp["y_star"], lp["z_star"]
    ax = lpgen.csr_matvec(lp["row_ptr"], lp["col_idx"], lp["val"], x)
    eq = lp["sense"] == EQ
    # primal feasibility: '=' rows exact, '<' rows a x <= b, bounds
    assert np.max(np.abs(ax[eq] - lp["b"][eq])) <= 1e-9 * (1 + np.max(np.abs(lp["b"])))
    slack = lp["b"][~eq] - ax[~eq]
    assert np.all(slack >= -1e-9)
    assert np.all(x >= lp["lb"]) and np.all(x <= lp["ub"])
    # dual feasibility and complementarity: c - A'y = z, z_j = 0 off both
    # bounds, z >= 0 at 0, z <= 0 at u; y <= 0 on '<' rows, 0 where slack > 0
    rc = lp["c"] - lpgen.csr_rmatvec(lp["row_ptr"], lp["col_idx"], lp["val"], y, n)
    assert np.max(np.abs(rc - z)) <= 1e-9 * (1 + np.max(np.abs(lp["c"])))
    inside = (x > lp["lb"]) & (x < lp["ub"])
    assert np.all(z[inside] == 0.0)
    assert np.all(z[(x == 0.0) & ~inside] > 0.0) and np.all(z[(x == lp["ub"]) & ~inside] < 0.0)
    assert np.all(y[~eq] <= 0.0) and np.all(y[~eq][slack > 1e-9] == 0.0)
    # strong duality: c'x = b'y + sum u_j z_j over columns at their upper bound
    at_u = (x == lp["ub"]) & np.isfinite(lp["ub"])
    dual = lp["b"] @ y + lp["ub"][at_u] @ z[at_u]
    assert abs(lp["obj_star"] - dual) <= 1e-7 * (1 + abs(dual))
