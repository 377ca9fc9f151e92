"""Reflected restarted Halpern PDHG: the second inner loop (TEST INFRASTRUCTURE).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
module.  Section 4.1 states that the paper's PDHG closely follows cuPDLP+
(Lu, Peng and Yang, 2025).  That method replaces the averaged iteration of
`oracle.pdhg` with Halpern's anchored iteration (Halpern, 1967) on the
reflected PDHG operator, restarts on the fixed-point residual, and steers the
primal weight with a PID controller.  The paper prints none of it; the steps
below follow the published method, and every constant the paper leaves open
is a reading:

  T(z)       one PDHG step from z = (x, y), as in `oracle.pdhg.pdhg_step`:
             x+ = proj_[l,u](x - tau (c - A'y)),
             y+ = proj_Y(y + sigma (b - A (2 x+ - x)))
  metric     PDHG is a proximal-point method in the metric
             M = [[I / tau, A'], [A, I / sigma]], under which T is firmly
             nonexpansive; ||dz||_M^2 = |dx|^2 / tau + |dy|^2 / sigma + 2 dy'A dx
             (sign from this y-update convention)
  step       z_{t+1} = w_t ((1 + rho) T(z_t) - rho z_t) + (1 - w_t) z_0,
             w_t = (t + 1) / (t + 2), z_0 the anchor (last restart point),
             rho = 1: the reflected operator 2T - I (reading)
  residual   r(z) = ||z - T(z)||_M, the quantity the restart tests use
  checks     every check period, the PDHG output T(z) of the last step is
             evaluated (Section 2 termination, or the Section 3.1 rule in the
             corner phase) and is the point returned and the restart point
  restart    r <= beta_suff r_0, or r <= beta_nec r_0 and r > r_prev, or
             t >= beta_art k (the same constants as the averaged loop);
             r_0 is the anchor's residual: measured by one uncounted
             application of T at the start of a phase, and after a restart
             the residual measured at that check (reading)
  weight     PID in log space on the movement of the anchor:
             e = log(omega) - log(|dy| / |dx|), I += e,
             log omega -= K_P e + K_I I + K_D (e - e_prev), gains 0.99 / 0.01 / 0
             (reading); skipped when |dx| or |dy| <= 1e-10

There are no averages: a phase returns T(z) of its last check.
"""
import math
import time

import numpy as np

from . import pdhg as P

HALPERN_DEFAULTS = dict(
    reflection=1.0,   # reading: the reflected operator 2T - I
    pid_kp=0.99,      # reading
    pid_ki=0.01,      # reading
    pid_kd=0.0,       # reading
)


def pdhg_map(model, x, y, tau, sigma):
    """T(z) = (x+, y+): one PDHG step (the map `oracle.pdhg.pdhg_step` applies)."""
    g = model.chat - model.AhatT @ y
    xp = P.project_box(x - tau * g, model.lhat, model.uhat)
    xbar = 2.0 * xp - x
    yp = y + sigma * (model.bhat - model.Ahat @ xbar)
    yp[model.ge] = np.maximum(yp[model.ge], 0.0)
    if model.y_zero is not None:
        yp[model.y_zero] = 0.0
    return xp, yp


def metric_norm2(model, dx, dy, tau, sigma):
    """||(dx, dy)||_M^2 = |dx|^2 / tau + |dy|^2 / sigma + 2 dy' A_hat dx."""
    return float(dx @ dx) / tau + float(dy @ dy) / sigma + 2.0 * float(dy @ (model.Ahat @ dx))


def fixed_point_residual(model, x, y, xp, yp, tau, sigma):
    """r(z) = ||z - T(z)||_M for z = (x, y) and T(z) = (xp, yp)."""
    return math.sqrt(max(metric_norm2(model, x - xp, y - yp, tau, sigma), 0.0))


def halpern_weight(t):
    """w_t = (t + 1) / (t + 2): the weight of the operator after t steps from the anchor."""
    return (t + 1.0) / (t + 2.0)


def halpern_update(z, zp, z0, t, rho):
    """w_t ((1 + rho) zp - rho z) + (1 - w_t) z0, zp = T(z)."""
    w = halpern_weight(t)
    return w * ((1.0 + rho) * zp - rho * z) + (1.0 - w) * z0


def pid_update(omega, dx, dy, integral, e_prev, kp, ki, kd):
    """One primal-weight update from the anchor movement (dx, dy) = (|x+ - x0|,
    |y+ - y0|).  Returns (omega, integral, e_prev); unchanged when either
    movement is <= 1e-10."""
    if not (dx > 1e-10 and dy > 1e-10):
        return omega, integral, e_prev
    e = math.log(omega) - math.log(dy / dx)
    integral = integral + e
    log_omega = math.log(omega) - (kp * e + ki * integral + kd * (e - e_prev))
    return math.exp(log_omega), integral, e


def restart_due(r, r0, r_prev, t, k, p):
    """The restart test on the fixed-point residual r of this check."""
    return (r <= p["beta_suff"] * r0
            or (r <= p["beta_nec"] * r0 and r > r_prev)
            or t >= p["beta_art"] * k)


class HState:
    """Halpern iterate, anchor and restart bookkeeping in scaled space."""

    def __init__(self, model, x0, y0, eta, omega):
        self.x = x0.copy()
        self.y = y0.copy()
        self.x0 = x0.copy()            # anchor z_0 (last restart point)
        self.y0 = y0.copy()
        self.xp = x0.copy()            # T(z) of the last step
        self.yp = y0.copy()
        self.t = 0                     # steps since the anchor
        self.k = 0                     # steps in this phase
        self.eta = eta
        self.omega = omega
        self.restarts = 0
        self.integral = 0.0            # PID integral term
        self.e_prev = 0.0
        xp, yp = pdhg_map(model, self.x, self.y, self.tau, self.sigma)
        self.r0 = fixed_point_residual(model, self.x, self.y, xp, yp, self.tau, self.sigma)
        self.r_prev = math.inf
        self.r = self.r0               # residual at the last check
        # restart history for the guidance features (same slots as the
        # averaged loop): the start point and every restart point
        self.ring = [(self.x.copy(), P.reduced_cost_hat(model, self.y))]

    @property
    def tau(self):
        return self.eta / self.omega

    @property
    def sigma(self):
        return self.eta * self.omega


def halpern_step(model, s, rho):
    """One anchored step: T(z) kept in (xp, yp), then z <- the Halpern combination.
    Returns the pre-step z for the residual of a check."""
    xp, yp = pdhg_map(model, s.x, s.y, s.tau, s.sigma)
    x_pre, y_pre = s.x, s.y
    s.x = halpern_update(x_pre, xp, s.x0, s.t, rho)
    s.y = halpern_update(y_pre, yp, s.y0, s.t, rho)
    s.xp, s.yp = xp, yp
    s.t += 1
    s.k += 1
    return x_pre, y_pre


def apply_restart(model, s, p, r):
    """Jump to T(z), make it the anchor, update the primal weight (PID)."""
    dx = float(np.linalg.norm(s.xp - s.x0))
    dy = float(np.linalg.norm(s.yp - s.y0))
    s.omega, s.integral, s.e_prev = pid_update(s.omega, dx, dy, s.integral, s.e_prev,
                                               p["pid_kp"], p["pid_ki"], p["pid_kd"])
    s.x, s.y = s.xp.copy(), s.yp.copy()
    s.x0, s.y0 = s.xp.copy(), s.yp.copy()
    s.r0 = r
    s.r_prev = math.inf
    s.t = 0
    s.restarts += 1
    s.ring.append((s.x.copy(), P.reduced_cost_hat(model, s.y)))
    del s.ring[:-8]


def _params(params):
    p = dict(P.DEFAULTS)
    p.update(HALPERN_DEFAULTS)
    if params:
        p.update(params)
    return p


def solve(lp, params=None, model=None):
    """Phase 1 with the Halpern loop: stop when the PDHG output of a check
    meets max(rel_p, rel_d, rel_gap) <= eps_rel (Section 2), or at a limit."""
    p = _params(params)
    if model is None:
        model = P.Model(lp, p["ruiz_iters"])
    sigma_max = P.power_iteration(model.Ahat, model.AhatT, p["power_iters"])
    eta = p["eta_factor"] / sigma_max if sigma_max > 0 else 1.0
    x0 = P.project_box(np.zeros(model.n), model.lhat, model.uhat)
    s = HState(model, x0, np.zeros(model.m), eta, P.initial_omega(model))
    t0 = time.perf_counter()
    status, ev = None, None
    while status is None:
        x_pre, y_pre = halpern_step(model, s, p["reflection"])
        at_check = s.k % p["check_period"] == 0
        at_limit = s.k >= p["max_iters"]
        if not (at_check or at_limit):
            continue
        ev = P.evaluate(model, s.xp, s.yp, s.omega)
        s.r = fixed_point_residual(model, x_pre, y_pre, s.xp, s.yp, s.tau, s.sigma)
        if not (np.isfinite(ev["kkt"]) and np.isfinite(s.r)):
            status = P.NUMERICAL
        elif at_check and ev["rel_kkt"] <= p["eps_rel"]:
            status = P.OPTIMAL
        elif at_limit:
            status = P.ITER_LIMIT
        elif time.perf_counter() - t0 > p["time_limit_s"]:
            status = P.TIME_LIMIT
        elif restart_due(s.r, s.r0, s.r_prev, s.t, s.k, p):
            apply_restart(model, s, p, s.r)
        else:
            s.r_prev = s.r
    return dict(status=status, iters=s.k, restarts=s.restarts, state=s, model=model,
                params=p, sigma_max=sigma_max, eta=eta, chosen="output",
                x_hat=s.xp.copy(), y_hat=s.yp.copy(), eval=ev,
                seconds=time.perf_counter() - t0)


def run_iterations(lp, iters, params=None):
    """Exactly `iters` Halpern steps with the phase-1 restart logic."""
    q = dict(params or {})
    q["max_iters"] = iters
    q["eps_rel"] = -1.0
    return solve(lp, q)


def corner_phase(phase1, corner_params=None, hold=None):
    """Algorithm 1 with the Halpern loop: the corner model of
    `oracle.pdhg.corner_model`, a fresh anchor at (proj(x1), 0) with its
    residual measured, the primal weight (oracle.pdhg.corner_omega0) and PID
    state reset; stop once
    k >= min_iters and the PDHG output of a check meets the Section 3.1
    primal rule (or the full test with stop_rule "kkt"); on a limit the
    phase-1 point is kept."""
    cp = dict(P.CORNER_DEFAULTS)
    if corner_params:
        cp.update(corner_params)
    model = phase1["model"]
    p = dict(phase1["params"])
    eta = phase1["eta"]
    x1, y1 = phase1["x_hat"], phase1["y_hat"]
    cm, info = P.corner_model(model, x1, y1, cp, hold)
    s = HState(cm, P.project_box(x1, cm.lhat, cm.uhat), np.zeros(model.m), eta, P.corner_omega0(phase1, cm, cp))
    t0 = time.perf_counter()
    nb = float(np.linalg.norm(model.b_user))
    status, x_corner = None, None
    while status is None:
        x_pre, y_pre = halpern_step(cm, s, p["reflection"])
        at_check = s.k % p["check_period"] == 0
        at_limit = s.k >= cp["max_iters"]
        if not (at_check or at_limit):
            continue
        ev = P.evaluate(cm, s.xp, s.yp, s.omega)
        s.r = fixed_point_residual(cm, x_pre, y_pre, s.xp, s.yp, s.tau, s.sigma)
        if at_check and s.k >= cp["min_iters"]:
            done = (ev["rel_kkt"] <= cp["eps_rel"] if cp["stop_rule"] == "kkt"
                    else ev["rP2"] <= cp["eps_rel"] * (1.0 + nb))
            if done:
                status, x_corner = P.CORNER_DONE, s.xp.copy()
                break
        if (at_limit or not (np.isfinite(ev["kkt"]) and np.isfinite(s.r))
                or time.perf_counter() - t0 > cp["time_limit_s"]):
            status, x_corner = P.CORNER_LIMIT, x1.copy()
            break
        if restart_due(s.r, s.r0, s.r_prev, s.t, s.k, p):
            apply_restart(cm, s, p, s.r)
        else:
            s.r_prev = s.r
    return dict(status=status, iters=s.k, restarts=s.restarts, state=s, corner_model=cm,
                model=model, info=info, x_hat=x_corner, y_hat=y1.copy(),
                seconds=time.perf_counter() - t0)


def dual_corner_phase(phase1, corner_params=None):
    """The dual corner push (oracle.pdhg.dual_corner_model) with the Halpern
    loop: a fresh anchor at (proj(0), y1) (y1 = 0 on rows whose dual is
    fixed), its residual measured, omega_0 from the new b' and the PID state
    reset; stop once k >= min_iters and the dual residual of the PDHG output
    of a check meets eps_rel (1 + ||c||) (or the full test with stop_rule
    "kkt"); on a limit the phase-1 y is kept."""
    cp = dict(P.CORNER_DEFAULTS)
    if corner_params:
        cp.update(corner_params)
    model = phase1["model"]
    p = dict(phase1["params"])
    eta = phase1["eta"]
    x1, y1 = phase1["x_hat"], phase1["y_hat"]
    dm, info = P.dual_corner_model(model, x1, y1, cp)
    y0 = np.where(dm.y_zero, 0.0, y1)
    s = HState(dm, P.project_box(np.zeros(model.n), dm.lhat, dm.uhat), y0, eta, P.initial_omega(dm))
    t0 = time.perf_counter()
    nc = float(np.linalg.norm(model.c_user))
    status, y_out = None, None
    while status is None:
        x_pre, y_pre = halpern_step(dm, s, p["reflection"])
        at_check = s.k % p["check_period"] == 0
        at_limit = s.k >= cp["max_iters"]
        if not (at_check or at_limit):
            continue
        ev = P.evaluate(dm, s.xp, s.yp, s.omega)
        s.r = fixed_point_residual(dm, x_pre, y_pre, s.xp, s.yp, s.tau, s.sigma)
        if at_check and s.k >= cp["min_iters"]:
            done = (ev["rel_kkt"] <= cp["eps_rel"] if cp["stop_rule"] == "kkt"
                    else ev["rD2"] <= cp["eps_rel"] * (1.0 + nc))
            if done:
                status, y_out = P.CORNER_DONE, s.yp.copy()
                break
        if (at_limit or not (np.isfinite(ev["kkt"]) and np.isfinite(s.r))
                or time.perf_counter() - t0 > cp["time_limit_s"]):
            status, y_out = P.CORNER_LIMIT, y1.copy()
            break
        if restart_due(s.r, s.r0, s.r_prev, s.t, s.k, p):
            apply_restart(dm, s, p, s.r)
        else:
            s.r_prev = s.r
    return dict(status=status, iters=s.k, restarts=s.restarts, state=s, dual_model=dm,
                model=model, info=info, x_hat=x1.copy(), y_hat=y_out,
                seconds=time.perf_counter() - t0)
