"""Host-side logic of bench.py (no GPU): which loop the headline runs, the
algorithmic byte counts, and that the CPU-baseline and reference legs time
exactly the oracle's own iteration."""
import argparse

import numpy as np
import pytest

import bench
import lpgen
import oracle


def _args(**kw):
    a = argparse.Namespace(workload="power_law_m100k_n400k", algorithm="both")
    for k, v in kw.items():
        setattr(a, k, v)
    return a


def test_headline_algorithm():
    assert bench.headline_algorithm(_args()) == "halpern"
    assert bench.headline_algorithm(_args(algorithm="halpern")) == "halpern"
    assert bench.headline_algorithm(_args(algorithm="averaged")) == "averaged"
    # the batched workload follows the same setting
    assert bench.headline_algorithm(_args(workload="batch_512")) == "halpern"
    assert bench.headline_algorithm(_args(workload="batch_512", algorithm="averaged")) == "averaged"


def test_halpern_bytes_differ_by_the_sums_and_the_anchor():
    m, n, nnz = 1000, 4000, 30000
    p_avg, d_avg = bench.algorithmic_bytes(m, n, nnz)
    p_h, d_h = bench.algorithmic_bytes_halpern(m, n, nnz)
    # primal: the running sum's read and write (16 B) become the anchor's read (8 B)
    assert p_avg - p_h == 8 * n
    # dual: likewise per row
    assert d_avg - d_h == 8 * m


@pytest.mark.parametrize("alg", ["averaged", "halpern"])
def test_cpu_sample_is_the_oracle_iteration(alg):
    lp = lpgen.small_face_lp(0)
    model, p, sigma_max, eta = oracle.setup(lp)
    _, s = bench.oracle_sample(model, p, eta, 130, alg)
    ref = oracle.run_iterations(lp, 130, dict(algorithm=alg))["state"]
    assert s.k == ref.k == 130 and s.restarts == ref.restarts
    assert np.array_equal(s.x, ref.x) and np.array_equal(s.y, ref.y)


def test_step_roofline():
    # 100 MB per iteration, 1000 iterations in 50 ms: 50 us each, 2 TB/s
    r = bench.step_roofline(100e6, 50.0, 1000, 8000.0)
    assert r["us_per_iter"] == pytest.approx(50.0)
    assert r["achieved"] == pytest.approx(2000.0)
    assert r["frac"] == pytest.approx(0.25)


def test_headline_bound_follows_the_larger_fraction():
    hbm = {"achieved": 2187.0, "peak": 6789.6, "unit": "GB/s", "frac": 2187.0 / 6789.6,
           "peak_source": "measured hbm_gbs"}
    fp64 = {"achieved_tflops": 0.415, "peak_tflops": 1.25, "frac": 0.415 / 1.25}
    top = bench.headline_bound(hbm, fp64)
    assert top["bound"] == "alu" and top["unit"] == "TFLOP/s"
    assert top["achieved"] == 0.415 and top["peak"] == 1.25 and top["frac"] == pytest.approx(0.332)
    fp64_low = dict(fp64, achieved_tflops=0.3, frac=0.24)
    top = bench.headline_bound(hbm, fp64_low)
    assert top["bound"] == "hbm" and top["unit"] == "GB/s" and top["peak"] == 6789.6
    # the FP64 unit rate the docstring derives
    assert 152 * 2 * 2 * 2.07e9 / 1e12 == pytest.approx(1.26, abs=0.01)


@pytest.mark.parametrize("fp32, halpern, ms, alg_bytes, kernel", [
    (False, True, (0.02894, 0.02048), 63281924, "spmv<PrimalOpH> (primal step)"),
    (True, True, (0.02289, 0.01843), 43654616, "spmv<PrimalOpH32> (primal step)"),
    (False, False, (0.02758, 0.02004), 66481924, "spmv<PrimalOp> (primal step)"),
    (True, False, (0.02266, 0.01812), 46854616, "spmv<PrimalOp32> (primal step)"),
])
def test_kernel_roofline(fp32, halpern, ms, alg_bytes, kernel):
    # the 100k x 400k workload with the replayed durations of the default bench
    m, n, nnz = 100000, 400000, 3206827
    rec = {"halpern_dram_bytes_per_launch_primal": "57401600", "halpern32_dram_bytes_per_launch_primal": "40662784"}
    r = bench.kernel_roofline(m, n, nnz, fp32, halpern, ms[0], ms[1], 6789.6, "measured", rec)
    assert r["kernel"] == kernel and r["algorithmic_bytes_per_launch"] == alg_bytes
    assert r["hbm"]["achieved"] == pytest.approx(alg_bytes / (ms[0] * 1e-3) / 1e9)
    # the record's counters for the kernel it names, null for kernels it does not hold
    want = {(False, True): 57401600.0, (True, True): 40662784.0}.get((fp32, halpern))
    assert r["traffic"] == want
    assert r["bound"] in ("hbm", "alu")
    top = r["fp64"] if r["bound"] == "alu" else r["hbm"]
    assert r["frac"] == top["frac"] and r["frac"] >= min(r["hbm"]["frac"], r["fp64"]["frac"])
    if fp32:
        assert r["fp64"]["frac"] == 0.0 and r["bound"] == "hbm"
    if halpern and not fp32:
        # one FMA per nonzero plus 5 FP64 operations per column (x_bar doubles as the reflected point)
        assert r["fp64"]["ops_per_launch"] == nnz + 5 * n
    if halpern and fp32:
        expect = bench.algorithmic_bytes_halpern32(m, n, nnz)
    elif halpern:
        expect = bench.algorithmic_bytes_halpern(m, n, nnz)
    elif fp32:
        expect = bench.algorithmic_bytes(m, n, nnz, s_v=4, s_x=4, s_sum=8, s_lo=4)
    else:
        expect = bench.algorithmic_bytes(m, n, nnz)
    assert sum(r["bytes_per_launch"]) == sum(expect)


def test_halpern32_bytes():
    # FP32 bulk halves the value and gathered-vector bytes; the float-float
    # iterate and anchor keep 8 B each per entry
    m, n, nnz = 1000, 4000, 30000
    p32, d32 = bench.algorithmic_bytes_halpern32(m, n, nnz)
    p64, d64 = bench.algorithmic_bytes_halpern(m, n, nnz)
    assert p64 - p32 == 4 * nnz + 4 * m + n * (3 * 4 + 8 + 8 + 8 + 4 - 7 * 8) * -1
    assert d64 - d32 == 4 * nnz + 4 * n + m * (33 - 29)


def test_corner_speedup_needs_corners_on_both_arms():
    def arm(ms, statuses):
        return {"total_ms": ms, "reps": [({}, {"status_name": st}) for st in statuses]}
    ok = bench.corner_speedup(arm(300.0, ["CORNER_DONE"] * 3), arm(200.0, ["CORNER_DONE"] * 3))
    assert ok["value"] == pytest.approx(1.5) and ok["reason"] is None
    bad = bench.corner_speedup(arm(300.0, ["CORNER_LIMIT"] * 3), arm(200.0, ["CORNER_DONE"] * 3))
    assert bad["value"] is None and bad["base_corner_status"] == ["CORNER_LIMIT"] and bad["reason"]
