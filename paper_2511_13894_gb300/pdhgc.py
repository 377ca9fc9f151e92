"""Python binding of libpdhgc (include/pdhgc.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels; this module
converts arrays to pointers, fills the C parameter structs and turns
reports into dicts.  PyTorch supplies device memory and the CUDA stream.
There is no CPU fallback: importing this module raises if the compiled
library is missing, and every call raises PdhgcError on a non-zero return.

Function names follow the C entry points without the `pdhgc_` prefix
(`lp_create`, `solve`, `corner_phase`, `kkt_report`, `get_solution`, ...);
the raw ctypes functions are available as `lib.pdhgc_*`.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpdhgc.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it first (python -m paper_2511_13894_gb300.build); "
        "there is no CPU fallback")

lib = C.CDLL(LIB_PATH)

# ---- constants (include/pdhgc.h) -------------------------------------------
OK = 0
ERR_NAMES = {-1: "INVALID_ARG", -2: "INVALID_CSR", -3: "NONFINITE", -4: "BOUNDS", -5: "CUDA", -6: "OOM",
             -7: "NO_PHASE1", -8: "NO_CORNER", -9: "TOO_LARGE", -10: "DEVICE", -11: "BUFFER", -12: "IO"}
STATUS_NAMES = {0: "NONE", 1: "OPTIMAL", 2: "ITER_LIMIT", 3: "TIME_LIMIT", 4: "NUMERICAL",
                5: "CORNER_DONE", 6: "CORNER_LIMIT", 7: "GUIDE_FALLBACK"}
GUIDE_FEATURES, GUIDE_FEAT_STRIDE, GUIDE_PARAMS = 18, 32, 5441
FP64, FP32_BULK = 0, 1
PHASE1, CORNER, DUAL_CORNER = 0, 1, 2
AVERAGED, HALPERN = 0, 1  # pdhgc_params.algorithm (PDHGC_ALG_*)
LAUNCH_GRAPH, LAUNCH_STREAM = 0, 1  # pdhgc_set_launch_mode


class PdhgcError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        detail = lib.pdhgc_last_error_detail().decode(errors="replace")
        super().__init__(f"{where}: {ERR_NAMES.get(code, code)} "
                         f"({lib.pdhgc_strerror(code).decode()}): {detail}")


class Params(C.Structure):
    _fields_ = [("eps_rel", C.c_double), ("max_iters", C.c_int64), ("time_limit_s", C.c_double),
                ("check_period", C.c_int32), ("beta_suff", C.c_double), ("beta_nec", C.c_double),
                ("beta_art", C.c_double), ("theta", C.c_double), ("eta_factor", C.c_double),
                ("ruiz_iters", C.c_int32), ("power_iters", C.c_int32), ("precision", C.c_int32),
                ("algorithm", C.c_int32), ("reflection", C.c_double), ("pid_kp", C.c_double),
                ("pid_ki", C.c_double), ("pid_kd", C.c_double)]


class CornerParams(C.Structure):
    _fields_ = [("eps_abs", C.c_double), ("eps_rel", C.c_double), ("min_iters", C.c_int64),
                ("max_iters", C.c_int64), ("time_limit_s", C.c_double), ("obj_seed", C.c_uint64),
                ("obj_scale", C.c_double), ("stop_rule", C.c_int32), ("row_rule", C.c_int32),
                ("omega_rule", C.c_int32), ("reserved", C.c_int32)]


class Report(C.Structure):
    _fields_ = [("status", C.c_int32), ("chosen", C.c_int32), ("iters", C.c_int64), ("restarts", C.c_int64),
                ("rP2", C.c_double), ("rD2", C.c_double), ("rPinf", C.c_double), ("rDinf", C.c_double),
                ("pobj", C.c_double), ("dobj", C.c_double), ("gap", C.c_double),
                ("rel_p", C.c_double), ("rel_d", C.c_double), ("rel_gap", C.c_double), ("rel_kkt", C.c_double),
                ("off_bound_p", C.c_int64), ("zero_rc_d", C.c_int64), ("candidates", C.c_int64),
                ("corner_measure", C.c_int64), ("primal_push_est", C.c_int64), ("dual_push_est", C.c_int64),
                ("should_corner", C.c_int32), ("precision", C.c_int32), ("seconds", C.c_double),
                ("omega", C.c_double), ("eta", C.c_double), ("sigma_max", C.c_double)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["status_name"] = STATUS_NAMES.get(self.status, str(self.status))
        return d


class GuideParams(C.Structure):
    _fields_ = [("threshold", C.c_double), ("guided_max_iters", C.c_int64), ("fallback", C.c_int32),
                ("reserved", C.c_int32)]


class GuideReport(C.Structure):
    _fields_ = [("status", C.c_int32), ("fell_back", C.c_int32), ("eligible", C.c_int64), ("held", C.c_int64),
                ("guided_iters", C.c_int64), ("guided_seconds", C.c_double), ("guided_rel_kkt", C.c_double),
                ("guided_corner_measure", C.c_int64), ("infer_seconds", C.c_double)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["status_name"] = STATUS_NAMES.get(self.status, str(self.status))
        return d


_vp = C.c_void_p
_sig = {
    "pdhgc_default_params": (None, [C.POINTER(Params)]),
    "pdhgc_default_corner_params": (None, [C.POINTER(CornerParams)]),
    "pdhgc_lp_create": (C.c_int, [C.POINTER(_vp), C.c_int32, C.c_int32, C.c_int64, _vp, _vp, _vp, _vp, _vp,
                                  _vp, _vp, _vp, C.c_int, _vp]),
    "pdhgc_solve": (C.c_int, [_vp, C.POINTER(Params), C.POINTER(Report)]),
    "pdhgc_corner_phase": (C.c_int, [_vp, C.POINTER(CornerParams), C.POINTER(Report)]),
    "pdhgc_dual_corner_phase": (C.c_int, [_vp, C.POINTER(CornerParams), C.POINTER(Report)]),
    "pdhgc_kkt_report": (C.c_int, [_vp, C.c_int, C.POINTER(Report)]),
    "pdhgc_get_solution": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, C.c_int]),
    "pdhgc_get_iterates": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, C.c_int]),
    "pdhgc_get_scaling": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int]),
    "pdhgc_get_layout": (C.c_int, [_vp, _vp]),
    "pdhgc_set_primal_layout": (C.c_int, [_vp, C.c_int32]),
    "pdhgc_set_launch_mode": (C.c_int, [_vp, C.c_int32]),
    "pdhgc_uniform": (C.c_int, [C.c_uint64, C.c_int64, C.c_double, _vp, _vp]),
    "pdhgc_kkt_eval": (C.c_int, [C.c_int32, C.c_int32, C.c_int64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                 _vp, C.POINTER(Report), _vp]),
    "pdhgc_kernel_launches": (C.c_int64, [_vp]),
    "pdhgc_profile_iteration": (C.c_int, [_vp, C.c_int32, _vp]),
    "pdhgc_lp_destroy": (None, [_vp]),
    "pdhgc_batch_create": (C.c_int, [C.POINTER(_vp), C.c_int32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                     _vp, _vp]),
    "pdhgc_batch_solve": (C.c_int, [_vp, C.POINTER(Params), _vp]),
    "pdhgc_batch_corner_phase": (C.c_int, [_vp, C.POINTER(CornerParams), _vp]),
    "pdhgc_batch_solve_corner": (C.c_int, [_vp, C.POINTER(Params), C.POINTER(CornerParams), _vp, _vp]),
    "pdhgc_batch_get_solution": (C.c_int, [_vp, C.c_int32, C.c_int, _vp, _vp]),
    "pdhgc_batch_set_block": (C.c_int, [_vp, C.c_int32]),
    "pdhgc_batch_set_lanes": (C.c_int, [_vp, C.c_int32, C.c_int32]),
    "pdhgc_batch_destroy": (None, [_vp]),
    "pdhgc_batch_set_layout": (C.c_int, [_vp, C.c_int32]),
    "pdhgc_batch_tune": (C.c_int, [_vp, C.POINTER(Params), C.c_int32, _vp, _vp]),
    "pdhgc_batch_kernel_launches": (C.c_int64, [_vp]),
    "pdhgc_batch_set_handoff": (C.c_int, [_vp, C.c_int32, C.c_int64]),
    "pdhgc_batch_handed_off": (C.c_int32, [_vp, C.c_int32, C.c_int]),
    "pdhgc_probe_gather": (C.c_int, [C.c_int64, C.c_int64, C.c_int32, C.c_int32, _vp, _vp]),
    "pdhgc_get_state": (C.c_int, [_vp, _vp, C.POINTER(C.c_size_t)]),
    "pdhgc_set_state": (C.c_int, [_vp, _vp, C.c_size_t]),
    "pdhgc_default_guide_params": (None, [C.POINTER(GuideParams)]),
    "pdhgc_guide_create": (C.c_int, [C.POINTER(_vp), C.c_uint64, _vp]),
    "pdhgc_guide_destroy": (None, [_vp]),
    "pdhgc_guide_set_weights": (C.c_int, [_vp, _vp]),
    "pdhgc_guide_get_weights": (C.c_int, [_vp, _vp]),
    "pdhgc_guide_save": (C.c_int, [_vp, C.c_char_p]),
    "pdhgc_guide_load": (C.c_int, [_vp, C.c_char_p]),
    "pdhgc_guide_infer": (C.c_int, [_vp, _vp, C.c_int64, _vp]),
    "pdhgc_guide_grad": (C.c_int, [_vp, _vp, _vp, C.c_int64, _vp, C.c_int32, _vp, _vp]),
    "pdhgc_guide_train": (C.c_int, [_vp, _vp, _vp, C.c_int64, C.c_int32, C.c_int64, C.c_float, C.c_uint64, _vp]),
    "pdhgc_guide_features": (C.c_int, [_vp, C.POINTER(CornerParams), _vp, _vp]),
    "pdhgc_guide_dataset_append": (C.c_int, [_vp, _vp, _vp, C.c_int64, C.POINTER(C.c_int64)]),
    "pdhgc_corner_phase_guided": (C.c_int, [_vp, C.POINTER(CornerParams), C.POINTER(GuideParams), _vp, _vp,
                                            C.c_int, C.POINTER(Report), C.POINTER(GuideReport)]),
    "pdhgc_guide_kernel_launches": (C.c_int64, [_vp]),
    "pdhgc_guide_set_wait_limit": (C.c_int, [_vp, C.c_int64]),
    "pdhgc_strerror": (C.c_char_p, [C.c_int]),
    "pdhgc_last_error_detail": (C.c_char_p, []),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def _check(rc, where):
    if rc != OK:
        raise PdhgcError(rc, where)


def default_params(**kw) -> Params:
    p = Params()
    lib.pdhgc_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


def default_corner_params(**kw) -> CornerParams:
    p = CornerParams()
    lib.pdhgc_default_corner_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown corner parameter {k}")
        setattr(p, k, v)
    return p


def _torch():
    import torch
    return torch


def _ptr_host(a, dtype):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(np.asarray(a, dtype=dtype))
    return arr, arr.ctypes.data


def _is_cuda_tensor(a):
    return hasattr(a, "is_cuda") and a.is_cuda


def _current_stream():
    torch = _torch()
    return torch.cuda.current_stream().cuda_stream


class LP:
    """One LP on the GPU (owns the library handle)."""

    def __init__(self, handle, m, n, stream):
        self._h = handle
        self.m = m
        self.n = n
        self.stream = stream

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib.pdhgc_lp_destroy(h)
            self._h = None

    def close(self):
        self.__del__()

    # -- phases --------------------------------------------------------------
    def solve(self, params: Params | None = None, **kw) -> dict:
        p = params if params is not None else default_params(**kw)
        r = Report()
        _check(lib.pdhgc_solve(self._h, C.byref(p), C.byref(r)), "pdhgc_solve")
        return r.as_dict()

    def corner_phase(self, params: CornerParams | None = None, **kw) -> dict:
        p = params if params is not None else default_corner_params(**kw)
        r = Report()
        _check(lib.pdhgc_corner_phase(self._h, C.byref(p), C.byref(r)), "pdhgc_corner_phase")
        return r.as_dict()

    def dual_corner_phase(self, params: CornerParams | None = None, **kw) -> dict:
        """pdhgc_dual_corner_phase: the dual corner push from the phase-1 point."""
        p = params if params is not None else default_corner_params(**kw)
        r = Report()
        _check(lib.pdhgc_dual_corner_phase(self._h, C.byref(p), C.byref(r)), "pdhgc_dual_corner_phase")
        return r.as_dict()

    def kkt_report(self, which: int = PHASE1) -> dict:
        r = Report()
        _check(lib.pdhgc_kkt_report(self._h, which, C.byref(r)), "pdhgc_kkt_report")
        return r.as_dict()

    # -- accessors -------------------------------------------------------------
    def _outs(self, sizes, device):
        if device:
            torch = _torch()
            bufs = [torch.empty(s, dtype=torch.float64, device="cuda") if s else None for s in sizes]
            ptrs = [b.data_ptr() if b is not None else None for b in bufs]
        else:
            bufs = [np.empty(s, dtype=np.float64) if s else None for s in sizes]
            ptrs = [b.ctypes.data if b is not None else None for b in bufs]
        return bufs, ptrs

    def get_solution(self, which: int = PHASE1, device: bool = False):
        (x, y, z), (px, py, pz) = self._outs([self.n, self.m, self.n], device)
        _check(lib.pdhgc_get_solution(self._h, which, px, py, pz, int(device)), "pdhgc_get_solution")
        return x, y, z

    def get_iterates(self, device: bool = False):
        """Scaled iterates; x_avg / y_avg hold T(z) after a Halpern-loop phase."""
        (x, y, xa, ya), ptrs = self._outs([self.n, self.m, self.n, self.m], device)
        it = (C.c_int64 * 3)()
        _check(lib.pdhgc_get_iterates(self._h, *ptrs, C.cast(it, _vp), int(device)), "pdhgc_get_iterates")
        return dict(x=x, y=y, x_avg=xa, y_avg=ya, k=it[0], t=it[1], restarts=it[2])

    def get_scaling(self):
        dr = np.empty(self.m)
        dc = np.empty(self.n)
        sc = np.empty(5)
        _check(lib.pdhgc_get_scaling(self._h, dr.ctypes.data, dc.ctypes.data, sc.ctypes.data, 0),
               "pdhgc_get_scaling")
        return dict(Dr=dr, Dc=dc, sigma_max=sc[0], eta=sc[1], omega=sc[2], tau=sc[3], sigma=sc[4])

    def kernel_launches(self) -> int:
        return int(lib.pdhgc_kernel_launches(self._h))

    def set_launch_mode(self, mode: int):
        """pdhgc_set_launch_mode: LAUNCH_GRAPH (default, one conditional graph
        per phase) or LAUNCH_STREAM (plain launches, one body at a time)."""
        _check(lib.pdhgc_set_launch_mode(self._h, int(mode)), "pdhgc_set_launch_mode")

    def set_primal_layout(self, chunked: bool):
        """pdhgc_set_primal_layout: 0 gathers from global memory (default), 1 stages y in shared memory."""
        _check(lib.pdhgc_set_primal_layout(self._h, int(bool(chunked))), "pdhgc_set_primal_layout")

    def get_layout(self):
        """pdhgc_get_layout: SpMV row-segment blocks of A and A'."""
        out = np.zeros(8, dtype=np.int64)
        _check(lib.pdhgc_get_layout(self._h, out.ctypes.data), "pdhgc_get_layout")
        keys = ("nb_cta", "nb_warp", "nb_sell", "cta_rows")
        return dict(A={k: int(out[i]) for i, k in enumerate(keys)},
                    AT={k: int(out[4 + i]) for i, k in enumerate(keys)})

    # -- checkpoint ----------------------------------------------------------------
    def get_state(self) -> bytes:
        """pdhgc_get_state: the handle's results as a byte string."""
        n = C.c_size_t(0)
        _check(lib.pdhgc_get_state(self._h, None, C.byref(n)), "pdhgc_get_state")
        buf = C.create_string_buffer(n.value)
        _check(lib.pdhgc_get_state(self._h, buf, C.byref(n)), "pdhgc_get_state")
        return buf.raw[:n.value]

    def set_state(self, state: bytes):
        """pdhgc_set_state: restore results taken from a handle of the same LP."""
        buf = C.create_string_buffer(state, len(state))
        _check(lib.pdhgc_set_state(self._h, buf, len(state)), "pdhgc_set_state")

    # -- learned corner guidance ------------------------------------------------
    def guide_features(self, params: CornerParams | None = None, **kw):
        """pdhgc_guide_features: (feat, eligible) as CUDA tensors: feat n x 32
        bfloat16 (18 features then zeros), eligible n uint8; user column order."""
        torch = _torch()
        p = params if params is not None else default_corner_params(**kw)
        feat = torch.zeros((self.n, GUIDE_FEAT_STRIDE), dtype=torch.bfloat16, device="cuda")
        elig = torch.zeros(self.n, dtype=torch.uint8, device="cuda")
        _check(lib.pdhgc_guide_features(self._h, C.byref(p), feat.data_ptr(), elig.data_ptr()),
               "pdhgc_guide_features")
        return feat, elig

    def dataset_append(self, feat, labels, count: int) -> int:
        """pdhgc_guide_dataset_append into CUDA tensors (feat rows x 32
        bfloat16, labels uint8) at row `count`; returns the new count."""
        c = C.c_int64(int(count))
        _check(lib.pdhgc_guide_dataset_append(self._h, feat.data_ptr(), labels.data_ptr(), int(feat.shape[0]),
                                              C.byref(c)), "pdhgc_guide_dataset_append")
        return int(c.value)

    def corner_phase_guided(self, guide=None, hold=None, threshold: float = 0.9, fallback: bool = True,
                            guided_max_iters: int = 0, params: CornerParams | None = None, **kw):
        """pdhgc_corner_phase_guided with a Guide network or a hold mask
        (numpy bool/uint8 per user column, or a CUDA uint8 tensor).
        Returns (report, guide_report)."""
        p = params if params is not None else default_corner_params(**kw)
        gp = GuideParams()
        lib.pdhgc_default_guide_params(C.byref(gp))
        gp.threshold = float(threshold)
        gp.fallback = int(bool(fallback))
        gp.guided_max_iters = int(guided_max_iters)
        r, gr = Report(), GuideReport()
        keep = None
        hold_ptr, on_dev = None, 0
        if hold is not None:
            if _is_cuda_tensor(hold):
                hold_ptr, on_dev = hold.data_ptr(), 1
            else:
                keep = np.ascontiguousarray(np.asarray(hold).astype(np.uint8))
                if keep.shape[0] != self.n:
                    raise ValueError("hold mask must have one entry per column")
                hold_ptr = keep.ctypes.data
        _check(lib.pdhgc_corner_phase_guided(self._h, C.byref(p), C.byref(gp), guide._h if guide else None,
                                             hold_ptr, on_dev, C.byref(r), C.byref(gr)),
               "pdhgc_corner_phase_guided")
        return r.as_dict(), gr.as_dict()

    def profile_iteration(self, iters: int = 20):
        """Mean ms per launch of the primal (A' pass) and dual (A pass)
        kernels over `iters` event-bracketed replays (advances the iterates)."""
        out = np.zeros(2)
        _check(lib.pdhgc_profile_iteration(self._h, int(iters), out.ctypes.data), "pdhgc_profile_iteration")
        return float(out[0]), float(out[1])


def lp_create(m, n, row_ptr, col_idx, val, b, c, lb=None, ub=None, sense=None, stream=None) -> LP:
    """pdhgc_lp_create.  Arrays may be numpy (host) or torch CUDA tensors
    (device; then all of them must be, with dtypes int64 / int32 / float64 /
    int8 as the header states).  `stream` is a raw cudaStream_t (int); by
    default torch's current stream."""
    arrays = [row_ptr, col_idx, val, b, c, lb, ub, sense]
    on_device = any(_is_cuda_tensor(a) for a in arrays if a is not None)
    keep = []
    if on_device:
        torch = _torch()
        dts = [torch.int64, torch.int32, torch.float64, torch.float64, torch.float64, torch.float64,
               torch.float64, torch.int8]
        ptrs = []
        for a, dt in zip(arrays, dts):
            if a is None:
                ptrs.append(None)
                continue
            if not _is_cuda_tensor(a) or a.dtype != dt or not a.is_contiguous():
                raise TypeError("device inputs must all be contiguous CUDA tensors of the documented dtypes")
            ptrs.append(a.data_ptr())
    else:
        dts = [np.int64, np.int32, np.float64, np.float64, np.float64, np.float64, np.float64, np.int8]
        ptrs = []
        for a, dt in zip(arrays, dts):
            arr, p = _ptr_host(a, dt)
            keep.append(arr)
            ptrs.append(p)
    nnz = int(row_ptr[-1]) if not on_device else int(row_ptr[-1].item())
    if stream is None:
        stream = _current_stream() if (on_device or _cuda_available()) else None
    h = _vp()
    rc = lib.pdhgc_lp_create(C.byref(h), int(m), int(n), nnz, *ptrs, int(on_device), stream)
    _check(rc, "pdhgc_lp_create")
    return LP(h, int(m), int(n), stream)


def lp_from_dict(lp: dict, stream=None, device=False) -> LP:
    """lp_create from a generator dict (keys m, n, row_ptr, col_idx, val, b,
    c, lb, ub, sense); device=True first copies the arrays to the GPU."""
    keys = ["row_ptr", "col_idx", "val", "b", "c", "lb", "ub", "sense"]
    arrs = [lp.get(k) for k in keys]
    if device:
        torch = _torch()
        dts = [torch.int64, torch.int32, torch.float64, torch.float64, torch.float64, torch.float64,
               torch.float64, torch.int8]
        arrs = [None if a is None else torch.as_tensor(np.ascontiguousarray(a)).to(dtype=dt, device="cuda")
                for a, dt in zip(arrs, dts)]
    return lp_create(lp["m"], lp["n"], *arrs, stream=stream)


class Batch:
    """Many LPs solved by one persistent launch (pdhgc_batch_*).  `lps` is a
    list of generator dicts (host arrays)."""

    _KEYS = (("row_ptr", np.int64), ("col_idx", np.int32), ("val", np.float64), ("b", np.float64),
             ("c", np.float64), ("lb", np.float64), ("ub", np.float64), ("sense", np.int8))

    def __init__(self, lps, stream=None):
        self.count = len(lps)
        self.m = [int(lp["m"]) for lp in lps]
        self.n = [int(lp["n"]) for lp in lps]
        self._keep = []
        ptrs = {}
        for key, dt in self._KEYS:
            arr = (C.c_void_p * self.count)()
            for k, lp in enumerate(lps):
                a = lp.get(key)
                if a is None:
                    arr[k] = None
                    continue
                a = np.ascontiguousarray(a, dtype=dt)
                self._keep.append(a)
                arr[k] = a.ctypes.data
            ptrs[key] = arr
        m = np.array(self.m, dtype=np.int32)
        n = np.array(self.n, dtype=np.int32)
        nnz = np.array([int(lp["row_ptr"][-1]) for lp in lps], dtype=np.int64)
        self._keep += [m, n, nnz]
        if stream is None:
            stream = _current_stream()
        self.stream = stream
        h = _vp()
        _check(lib.pdhgc_batch_create(C.byref(h), self.count, m.ctypes.data, n.ctypes.data, nnz.ctypes.data,
                                      *[C.cast(ptrs[k], _vp) for k, _ in self._KEYS], stream),
               "pdhgc_batch_create")
        self._h = h
        self._keep = None  # create copied everything

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib.pdhgc_batch_destroy(h)
            self._h = None

    def close(self):
        self.__del__()

    def solve(self, params: Params | None = None, **kw):
        p = params if params is not None else default_params(**kw)
        reps = (Report * self.count)()
        _check(lib.pdhgc_batch_solve(self._h, C.byref(p), C.cast(reps, _vp)), "pdhgc_batch_solve")
        return [r.as_dict() for r in reps]

    def corner_phase(self, params: CornerParams | None = None, **kw):
        p = params if params is not None else default_corner_params(**kw)
        reps = (Report * self.count)()
        _check(lib.pdhgc_batch_corner_phase(self._h, C.byref(p), C.cast(reps, _vp)), "pdhgc_batch_corner_phase")
        return [r.as_dict() for r in reps]

    def solve_corner(self, params: Params | None = None, cparams: CornerParams | None = None):
        """pdhgc_batch_solve_corner: both phases per LP in one launch; returns
        (phase-1 reports, corner reports)."""
        p = params if params is not None else default_params()
        cp = cparams if cparams is not None else default_corner_params()
        r1 = (Report * self.count)()
        rc = (Report * self.count)()
        _check(lib.pdhgc_batch_solve_corner(self._h, C.byref(p), C.byref(cp), C.cast(r1, _vp), C.cast(rc, _vp)),
               "pdhgc_batch_solve_corner")
        return [r.as_dict() for r in r1], [r.as_dict() for r in rc]

    def get_solution(self, k: int, which: int = PHASE1):
        x = np.empty(self.n[k])
        y = np.empty(self.m[k])
        _check(lib.pdhgc_batch_get_solution(self._h, k, which, x.ctypes.data, y.ctypes.data),
               "pdhgc_batch_get_solution")
        return x, y

    def kernel_launches(self) -> int:
        return int(lib.pdhgc_batch_kernel_launches(self._h))

    def set_handoff(self, max_running: int = 8, min_iters: int = 8192):
        """pdhgc_batch_set_handoff (max_running = 0 disables the tail handoff)."""
        _check(lib.pdhgc_batch_set_handoff(self._h, int(max_running), int(min_iters)), "pdhgc_batch_set_handoff")

    def handed_off(self, k: int, which: int = PHASE1) -> bool:
        return bool(lib.pdhgc_batch_handed_off(self._h, int(k), int(which)))

    def set_block(self, threads: int):
        _check(lib.pdhgc_batch_set_block(self._h, threads), "pdhgc_batch_set_block")

    def set_lanes(self, lanes_a: int = 0, lanes_t: int = 0):
        _check(lib.pdhgc_batch_set_lanes(self._h, lanes_a, lanes_t), "pdhgc_batch_set_lanes")

    def set_layout(self, sell: int):
        _check(lib.pdhgc_batch_set_layout(self._h, int(sell)), "pdhgc_batch_set_layout")

    def tune(self, tune_iters: int = 256, params: Params | None = None, **kw):
        """pdhgc_batch_tune: returns the chosen schedule and the candidates' times."""
        p = params if params is not None else default_params(**kw)
        chosen = np.zeros(4, dtype=np.int32)
        ms = np.zeros(7)
        _check(lib.pdhgc_batch_tune(self._h, C.byref(p), int(tune_iters), chosen.ctypes.data, ms.ctypes.data),
               "pdhgc_batch_tune")
        return dict(threads=int(chosen[0]), sell=int(chosen[1]), lanes_a=int(chosen[2]), lanes_t=int(chosen[3]),
                    timings_ms=ms.tolist())


class Guide:
    """The corner-guidance network (pdhgc_guide_*).  Feature and label arrays
    are CUDA tensors (rows x 32 bfloat16; uint8)."""

    def __init__(self, seed: int = 0, stream=None):
        if stream is None:
            stream = _current_stream()
        self.stream = stream
        h = _vp()
        _check(lib.pdhgc_guide_create(C.byref(h), C.c_uint64(seed), stream), "pdhgc_guide_create")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib.pdhgc_guide_destroy(h)
            self._h = None

    def close(self):
        self.__del__()

    def set_weights(self, w):
        w = np.ascontiguousarray(np.asarray(w, dtype=np.float32).reshape(-1))
        if w.shape[0] != GUIDE_PARAMS:
            raise ValueError(f"expected {GUIDE_PARAMS} parameters")
        _check(lib.pdhgc_guide_set_weights(self._h, w.ctypes.data), "pdhgc_guide_set_weights")

    def get_weights(self) -> np.ndarray:
        w = np.empty(GUIDE_PARAMS, dtype=np.float32)
        _check(lib.pdhgc_guide_get_weights(self._h, w.ctypes.data), "pdhgc_guide_get_weights")
        return w

    def save(self, path):
        """pdhgc_guide_save: the parameter vector to a file."""
        _check(lib.pdhgc_guide_save(self._h, os.fsencode(path)), "pdhgc_guide_save")

    def load(self, path):
        """pdhgc_guide_load: the parameter vector from a file written by save
        (Adam's moments reset)."""
        _check(lib.pdhgc_guide_load(self._h, os.fsencode(path)), "pdhgc_guide_load")

    def infer(self, feat):
        torch = _torch()
        p = torch.empty(int(feat.shape[0]), dtype=torch.float32, device="cuda")
        _check(lib.pdhgc_guide_infer(self._h, feat.data_ptr(), int(feat.shape[0]), p.data_ptr()),
               "pdhgc_guide_infer")
        return p

    def grad(self, feat, labels, idx):
        """Gradient of the mean BCE over the rows idx (no update): (grad, loss)."""
        idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int32))
        g = np.empty(GUIDE_PARAMS, dtype=np.float32)
        loss = C.c_float(0.0)
        _check(lib.pdhgc_guide_grad(self._h, feat.data_ptr(), labels.data_ptr(), int(feat.shape[0]),
                                    idx.ctypes.data, int(idx.shape[0]), g.ctypes.data, C.byref(loss)),
               "pdhgc_guide_grad")
        return g, float(loss.value)

    def train(self, feat, labels, rows: int, batch: int = 4096, steps: int = 1000, lr: float = 1e-3,
              seed: int = 0) -> np.ndarray:
        """`steps` Adam steps on minibatches drawn from the first `rows` rows;
        returns the per-step minibatch losses."""
        losses = np.zeros(int(steps), dtype=np.float32)
        _check(lib.pdhgc_guide_train(self._h, feat.data_ptr(), labels.data_ptr(), int(rows), int(batch),
                                     int(steps), float(lr), C.c_uint64(seed), losses.ctypes.data if steps else None),
               "pdhgc_guide_train")
        return losses

    def kernel_launches(self) -> int:
        return int(lib.pdhgc_guide_kernel_launches(self._h))

    def set_wait_limit(self, polls: int):
        """pdhgc_guide_set_wait_limit (failure-path tests)."""
        _check(lib.pdhgc_guide_set_wait_limit(self._h, int(polls)), "pdhgc_guide_set_wait_limit")


def _device_lp_args(lp: dict, x, y):
    """CUDA tensors for the LP arrays of a generator dict and for (x, y)."""
    torch = _torch()
    dts = {"row_ptr": torch.int64, "col_idx": torch.int32, "val": torch.float64, "b": torch.float64,
           "c": torch.float64, "lb": torch.float64, "ub": torch.float64, "sense": torch.int8}
    t = {}
    for k, dt in dts.items():
        a = lp.get(k)
        t[k] = None if a is None else torch.as_tensor(np.ascontiguousarray(a)).to(dtype=dt, device="cuda")
    t["x"] = torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64)).to(device="cuda")
    t["y"] = torch.as_tensor(np.ascontiguousarray(y, dtype=np.float64)).to(device="cuda")
    return t


def _ptr(t):
    return None if t is None else t.data_ptr()


def kkt_eval(lp: dict, x, y) -> dict:
    """pdhgc_kkt_eval of the point (x, y) (user scale) on a generator-dict LP."""
    t = _device_lp_args(lp, x, y)
    r = Report()
    nnz = int(lp["row_ptr"][-1])
    _check(lib.pdhgc_kkt_eval(int(lp["m"]), int(lp["n"]), nnz, _ptr(t["row_ptr"]), _ptr(t["col_idx"]),
                              _ptr(t["val"]), _ptr(t["b"]), _ptr(t["c"]), _ptr(t["lb"]), _ptr(t["ub"]),
                              _ptr(t["sense"]), _ptr(t["x"]), _ptr(t["y"]), C.byref(r), _current_stream()),
           "pdhgc_kkt_eval")
    return r.as_dict()


def uniform(seed: int, n: int, obj_scale: float = 1.0):
    """pdhgc_uniform into a new CUDA tensor."""
    torch = _torch()
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    _check(lib.pdhgc_uniform(C.c_uint64(seed), n, obj_scale, out.data_ptr(), _current_stream()),
           "pdhgc_uniform")
    return out


def probe_gather(n_vec: int, count: int, elem_bytes: int = 8, reps: int = 20) -> float:
    """pdhgc_probe_gather: ms per `count` random loads from an L2-resident
    vector of n_vec elements, at the steady-state rate of long launches."""
    out = np.zeros(1)
    _check(lib.pdhgc_probe_gather(int(n_vec), int(count), int(elem_bytes), int(reps), out.ctypes.data,
                                  _current_stream()), "pdhgc_probe_gather")
    return float(out[0])


def _cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False
