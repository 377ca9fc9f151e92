"""Plain FP64 CPU reference of the learned corner guidance (TEST INFRASTRUCTURE).

Not in the paper: an extension of Algorithm 1 in which a per-column network
predicts which columns the corner phase may hold at a bound.  This module
states, in plain numpy, what the CUDA path computes around the network:

* the 18 per-column features of a phase-1 result (`features`);
* which columns may be held (`eligible`): not fixed by Algorithm 1's
  reduced-cost rule and with a finite bound;
* the training labels of a corner result (`labels`): x_j within the metric
  tolerance (Section 4.2) of the bound a hold would fix it at;
* the guided corner phase with its fallback (`guided_corner_phase`).

The network itself is `oracle/mlp.py`.  Only `tests/`, the smoke check and
the benchmark's CPU leg import this; it shares no code with the CUDA path.

Readings (the paper has no such component):
* c_j is the objective of the LP the corner phase solves, i.e. Algorithm 1's
  random objective c' scaled like c (on the optimal face the user's reduced
  costs vanish, so the user's c carries no information on which columns end
  at a bound);
* ||A_j|| is the 2-norm of column j of the scaled matrix;
* the history holds (x_hat, z_hat) at the phase-1 start point and at every
  restart, newest first, the last 8 kept, padded by repeating the oldest;
  z_hat = proj_Lambda(c_hat - A_hat' y_hat) at the same point;
* each of the four groups (c, ||A_j||, the 8 x values, the 8 z values) is
  divided by its root mean square over all columns (1 when that is 0);
* the label is "the corner phase ends with x_j at the bound nearest to its
  phase-1 value", the bound a hold uses: a column that ends at its other
  bound would be held at the wrong one, which can make the held corner
  model infeasible.
"""
from __future__ import annotations

import numpy as np

from . import pdhg
from .mlp import forward

N_FEATURES = 18
HISTORY = 8
LABEL_TOL = pdhg.METRIC_TOL


def history(state) -> tuple[np.ndarray, np.ndarray]:
    """(X, Z), each n x 8, newest restart value first, padded with the oldest."""
    ring = state.ring[-HISTORY:]
    xs = [r[0] for r in reversed(ring)]
    zs = [r[1] for r in reversed(ring)]
    while len(xs) < HISTORY:
        xs.append(xs[-1])
        zs.append(zs[-1])
    return np.stack(xs, axis=1), np.stack(zs, axis=1)


def _rms_scaled(v: np.ndarray) -> np.ndarray:
    r = float(np.sqrt(np.mean(v * v))) if v.size else 0.0
    return v / (r if r > 0.0 else 1.0)


def features(phase1, corner_params=None):
    """n x 18 FP64 features of the phase-1 result, user column order:
    [c'_hat, ||A_hat_j||, x_hat history (8), z_hat history (8)], each group
    divided by its RMS.  Returns (F, eligible)."""
    cp = dict(pdhg.CORNER_DEFAULTS)
    if corner_params:
        cp.update(corner_params)
    model = phase1["model"]
    cm, info = pdhg.corner_model(model, phase1["x_hat"], phase1["y_hat"], cp)
    colnorm = np.sqrt(np.asarray(model.Ahat.multiply(model.Ahat).sum(axis=0)).ravel())
    X, Z = history(phase1["state"])
    F = np.empty((model.n, N_FEATURES))
    F[:, 0] = _rms_scaled(cm.chat)
    F[:, 1] = _rms_scaled(colnorm)
    F[:, 2:10] = _rms_scaled(X)
    F[:, 10:18] = _rms_scaled(Z)
    return F, eligible(phase1, cp)


def eligible(phase1, cp):
    """Columns the guidance may hold: not fixed by the reduced-cost rule of
    Algorithm 1 and with a finite bound nearest to the phase-1 point."""
    model = phase1["model"]
    _, info = pdhg.corner_model(model, phase1["x_hat"], phase1["y_hat"], cp)
    nb = pdhg.nearest_bound(phase1["x_hat"], model.lhat, model.uhat)
    return ~info["fixed"] & np.isfinite(nb)


def labels(model, x_hat, x_hat1, tol=LABEL_TOL):
    """1 where the user-space corner x_j lies within tol of the bound that a
    hold would use: the bound nearest to the phase-1 value x_hat1_j (in
    scaled space, then unscaled by D_c).  0 for a column without a finite
    bound."""
    nb = pdhg.nearest_bound(x_hat1, model.lhat, model.uhat)
    x = model.Dc * x_hat
    b = model.Dc * nb
    return np.isfinite(b) & (np.abs(x - b) <= tol)


def hold_mask(p, elig, threshold):
    """Columns to hold: predicted probability >= threshold and eligible."""
    return (np.asarray(p) >= threshold) & elig


def predict(weights, phase1, corner_params=None):
    """The network's probabilities for every column of the phase-1 result."""
    F, elig = features(phase1, corner_params)
    return forward(weights, F)[0], elig


def regressed(guided_report, ref_report, status, eps_rel):
    """Fallback rule: the guided corner hit a limit, or its relative KKT error
    exceeds max(reference, eps_rel), or its corner measure exceeds the
    reference's (the reference is the phase-1 point)."""
    return (status == pdhg.CORNER_LIMIT
            or guided_report["rel_kkt"] > max(ref_report["rel_kkt"], eps_rel)
            or guided_report["corner_measure"] > ref_report["corner_measure"])


def guided_corner_phase(phase1, hold, corner_params=None, fallback=True, guided_max_iters=0):
    """Algorithm 1 with `hold` columns fixed at their nearest bound (at most
    guided_max_iters iterations when > 0); when the result regresses against
    the phase-1 point, the plain corner phase runs and its result is returned
    (fell_back = True)."""
    cp = dict(pdhg.CORNER_DEFAULTS)
    if corner_params:
        cp.update(corner_params)
    model = phase1["model"]
    cpg = dict(cp)
    if guided_max_iters > 0:
        cpg["max_iters"] = min(cp["max_iters"], guided_max_iters)
    g = pdhg.corner_phase(phase1, cpg, hold=hold)
    g_rep = pdhg.kkt_report(model, g["x_hat"], g["y_hat"])
    p_rep = pdhg.kkt_report(model, phase1["x_hat"], phase1["y_hat"])
    out = dict(guided=g, guided_report=g_rep, fell_back=False, result=g, report=g_rep)
    if fallback and regressed(g_rep, p_rep, g["status"], cp["eps_rel"]):
        plain = pdhg.corner_phase(phase1, cp)
        out.update(fell_back=True, result=plain,
                   report=pdhg.kkt_report(model, plain["x_hat"], plain["y_hat"]))
    return out
