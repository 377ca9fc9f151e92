"""pdhgc_kkt_eval_noalloc against pdhgc_kkt_eval, through the C-ABI.

Some callers cannot allocate device memory: services with a fixed device
memory budget, applications whose device memory belongs to a pool or
framework allocator that must account for every byte, and code paths that
cannot accept the implicit synchronisation of cudaMalloc / cudaFree.  For
them the library offers a KKT evaluation whose scratch lives in a static
device array.  This file is collected last so that, if it fails, a run that
stops at the first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import lpgen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
P = pytest.importorskip("paper_2511_13894_gb300.pdhgc")

NOALLOC_MAX_N = 1 << 18
FIELDS = ("rP2", "rD2", "rPinf", "rDinf", "pobj", "dobj", "gap", "rel_p", "rel_d", "rel_gap", "rel_kkt")
COUNTS = ("off_bound_p", "zero_rc_d", "candidates", "corner_measure", "primal_push_est", "dual_push_est",
          "should_corner")

_noalloc = P.lib.pdhgc_kkt_eval_noalloc
_noalloc.restype = C.c_int
_noalloc.argtypes = P.lib.pdhgc_kkt_eval.argtypes


def _call(fn, lp, t, n_override=None):
    r = P.Report()
    ptr = P._ptr
    rc = fn(int(lp["m"]), int(n_override or lp["n"]), int(lp["row_ptr"][-1]), ptr(t["row_ptr"]),
            ptr(t["col_idx"]), ptr(t["val"]), ptr(t["b"]), ptr(t["c"]), ptr(t["lb"]), ptr(t["ub"]),
            ptr(t["sense"]), ptr(t["x"]), ptr(t["y"]), C.byref(r), torch.cuda.current_stream().cuda_stream)
    return rc, r.as_dict()


def _point(lp, seed):
    rng = np.random.default_rng(seed)
    x = np.clip(lp["x_star"] + 0.05 * rng.standard_normal(lp["n"]), lp["lb"], lp["ub"])
    y = lp["y_star"] + 0.05 * rng.standard_normal(lp["m"])
    return x, y


def _same(a, b, scale):
    # pdhgc_kkt_eval accumulates A'y with atomic adds, so the two entry points
    # may differ in the last bits; the tolerance is the parity tolerance of
    # the KKT evaluation tests
    for k in FIELDS:
        assert abs(a[k] - b[k]) <= 1e-9 * (scale + abs(b[k])), (k, a[k], b[k])
    for k in COUNTS:
        assert a[k] == b[k], k


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    lp_a = lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(3), 3)
    lp_b = lpgen.power_law_lp(3000, 12000, 500, seed=5, kmax=2000)
    for lp, seed in ((lp_a, 1), (lp_b, 2)):  # two calls in a row, different sizes
        x, y = _point(lp, seed)
        t = P._device_lp_args(lp, x, y)
        rc_ref, ref = _call(P.lib.pdhgc_kkt_eval, lp, t)
        rc, got = _call(_noalloc, lp, t)
        assert rc_ref == 0 and rc == 0
        scale = 1.0 + float(np.linalg.norm(lp["b"])) + float(np.linalg.norm(lp["c"]))
        _same(got, ref, scale)


def test_noalloc_rejects_n_above_its_capacity():
    lp = lpgen.small_face_lp(1)
    x, y = _point(lp, 0)
    t = P._device_lp_args(lp, x, y)
    rc, _ = _call(_noalloc, lp, t, n_override=NOALLOC_MAX_N + 1)
    assert rc == -9  # PDHGC_ERR_TOO_LARGE, before any device work
    assert b"static scratch capacity" in P.lib.pdhgc_last_error_detail()


def _cudart():
    """The CUDA runtime, for the device's default memory pool (the pool
    cudaMallocAsync draws from)."""
    import ctypes.util
    import glob
    import os
    names = [ctypes.util.find_library("cudart")] + sorted(glob.glob("/usr/local/cuda/lib64/libcudart.so*"))
    for nm in names:
        if nm and (os.path.exists(nm) or "/" not in nm):
            try:
                return C.CDLL(nm)
            except OSError:
                continue
    pytest.skip("libcudart not found")


def test_noalloc_allocates_no_device_memory():
    # the default pool's high-water mark of used memory, reset before each
    # call, moves for the allocating entry point (its cudaMallocAsync
    # scratch) and stays put for the no-allocation one; torch's allocator
    # sees no change either
    rt = _cudart()
    USED_HIGH = 8  # cudaMemPoolAttrUsedMemHigh
    dev = C.c_int(0)
    assert rt.cudaGetDevice(C.byref(dev)) == 0
    pool = C.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(C.byref(pool), dev) == 0

    def used_high_after(fn, lp, t):
        torch.cuda.synchronize()
        zero = C.c_uint64(0)
        assert rt.cudaMemPoolSetAttribute(pool, USED_HIGH, C.byref(zero)) == 0
        before = torch.cuda.memory_allocated()
        rc, _ = _call(fn, lp, t)
        torch.cuda.synchronize()
        assert rc == 0
        v = C.c_uint64(0)
        assert rt.cudaMemPoolGetAttribute(pool, USED_HIGH, C.byref(v)) == 0
        return v.value, torch.cuda.memory_allocated() - before

    lp = lpgen.power_law_lp(3000, 12000, 500, seed=5, kmax=2000)
    x, y = _point(lp, 3)
    t = P._device_lp_args(lp, x, y)
    high_ref, torch_ref = used_high_after(P.lib.pdhgc_kkt_eval, lp, t)
    high, torch_delta = used_high_after(_noalloc, lp, t)
    assert high_ref > 0          # the control: the allocating entry point used the pool
    assert high == 0 and torch_delta == 0 and torch_ref == 0
