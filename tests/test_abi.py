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
    cp = P.default_corner_params()
    assert cp.eps_abs == 1e-6 and cp.min_iters == 100 and cp.obj_scale == 1.0


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
