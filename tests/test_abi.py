"""The C-ABI library builds, loads without a GPU and exports every entry
point include/pdhgc.h declares; host-side validation rejects bad inputs
before any device work (no compute call here)."""
import ctypes
import os
import re

import numpy as np
import pytest

import lpgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2511_13894_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "pdhgc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(pdhgc_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("pdhgc_lp_create", "pdhgc_solve", "pdhgc_corner_phase", "pdhgc_kkt_report",
                     "pdhgc_get_solution", "pdhgc_lp_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_default_params_match_the_paper_and_readings(lib):
    from paper_2511_13894_gb300 import pdhgc as P
    p = P.default_params()
    assert p.eps_rel == 1e-6 and p.check_period == 64 and p.ruiz_iters == 10 and p.power_iters == 100
    assert (p.beta_suff, p.beta_nec, p.beta_art, p.theta, p.eta_factor) == (0.2, 0.8, 0.36, 0.5, 0.998)
    # the inner loop defaults to the averaged one; the Halpern loop's readings
    import oracle.halpern as H
    assert p.algorithm == P.AVERAGED
    assert (p.reflection, p.pid_kp, p.pid_ki, p.pid_kd) == (
        H.HALPERN_DEFAULTS["reflection"], H.HALPERN_DEFAULTS["pid_kp"],
        H.HALPERN_DEFAULTS["pid_ki"], H.HALPERN_DEFAULTS["pid_kd"])
    cp = P.default_corner_params()
    assert cp.eps_abs == 1e-6 and cp.min_iters == 100 and cp.obj_scale == 1.0
    assert cp.stop_rule == 0 and cp.row_rule == 0  # the Section 3.1 stop and Section 3 row rules
    assert cp.omega_rule == 0  # omega_0 from the corner objective
    gp = P.GuideParams()
    P.lib.pdhgc_default_guide_params(P.C.byref(gp))
    assert gp.threshold == 0.9 and gp.fallback == 1 and gp.guided_max_iters == 0


def test_ctypes_mirrors_match_the_c_structs(tmp_path):
    # sizes and field offsets of every struct the binding mirrors, taken from
    # the header by a C compiler
    import ctypes
    import shutil
    import subprocess
    from paper_2511_13894_gb300 import pdhgc as P
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = {"pdhgc_params": P.Params, "pdhgc_corner_params": P.CornerParams, "pdhgc_report": P.Report,
               "pdhgc_guide_params": P.GuideParams, "pdhgc_guide_report": P.GuideReport}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pdhgc.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("  return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    include = os.path.join(ROOT, "include")
    subprocess.run([cc, "-I", include, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        parts = line.split()
        if len(parts) == 3:
            got[(parts[0], parts[1])] = int(parts[2])
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def _expect(code, **override):
    from paper_2511_13894_gb300 import pdhgc as P
    lp = lpgen.small_face_lp(0)
    lp.update(override)
    with pytest.raises(P.PdhgcError) as ei:
        P.lp_create(lp["m"], lp["n"], lp["row_ptr"], lp["col_idx"], lp["val"], lp["b"], lp["c"],
                    lp.get("lb"), lp.get("ub"), lp.get("sense"), stream=0)
    assert ei.value.code == code


def test_host_validation_errors(lib):
    lp = lpgen.small_face_lp(0)
    rp = lp["row_ptr"].copy()
    rp[3], rp[4] = rp[4], rp[3] - 1
    _expect(-2, row_ptr=rp)
    col = lp["col_idx"].copy()
    col[7] = lp["n"]
    _expect(-2, col_idx=col)
    val = lp["val"].copy()
    val[0] = np.nan
    _expect(-3, val=val)
    b = lp["b"].copy()
    b[1] = np.inf
    _expect(-3, b=b)
    lb = lp["lb"].copy()
    lb[2] = 3.0
    ub = lp["ub"].copy()
    ub[2] = 2.0
    _expect(-4, lb=lb, ub=ub)
    sense = lp["sense"].copy()
    sense[0] = ord("x")
    _expect(-1, sense=sense)
    ub2 = lp["ub"].copy()
    ub2[0] = -np.inf
    _expect(-3, ub=ub2)


def test_package_exports_exist(lib):
    import paper_2511_13894_gb300 as pkg
    for name in pkg._EXPORTS:
        assert getattr(pkg, name) is not None, name


def _header_defines():
    src = open(os.path.join(ROOT, "include", "pdhgc.h")).read()
    return {k: int(v) for k, v in re.findall(r"^#define (PDHGC_[A-Z0-9_]+)\s+(-?\d+)", src, flags=re.M)}


def test_binding_constants_match_the_header(lib):
    # every error code, status, precision, result selector, inner loop, launch
    # mode and guidance size the binding names has the header's value
    from paper_2511_13894_gb300 import pdhgc as P
    d = _header_defines()
    errs = {v: k[len("PDHGC_ERR_"):] for k, v in d.items() if k.startswith("PDHGC_ERR_")}
    assert errs == P.ERR_NAMES
    stats = {v: k[len("PDHGC_STATUS_"):] for k, v in d.items() if k.startswith("PDHGC_STATUS_")}
    assert stats == P.STATUS_NAMES
    pairs = {"PDHGC_OK": P.OK, "PDHGC_FP64": P.FP64, "PDHGC_FP32_BULK": P.FP32_BULK, "PDHGC_PHASE1": P.PHASE1,
             "PDHGC_CORNER": P.CORNER, "PDHGC_DUAL_CORNER": P.DUAL_CORNER, "PDHGC_ALG_AVERAGED": P.AVERAGED,
             "PDHGC_ALG_HALPERN": P.HALPERN, "PDHGC_LAUNCH_GRAPH": P.LAUNCH_GRAPH,
             "PDHGC_LAUNCH_STREAM": P.LAUNCH_STREAM, "PDHGC_GUIDE_FEATURES": P.GUIDE_FEATURES,
             "PDHGC_GUIDE_FEAT_STRIDE": P.GUIDE_FEAT_STRIDE, "PDHGC_GUIDE_PARAMS": P.GUIDE_PARAMS}
    for name, value in pairs.items():
        assert d[name] == value, name


def test_every_error_code_has_a_message(lib):
    from paper_2511_13894_gb300 import pdhgc as P
    for code in P.ERR_NAMES:
        msg = P.lib.pdhgc_strerror(code).decode()
        assert msg and "unknown" not in msg.lower(), (code, msg)
