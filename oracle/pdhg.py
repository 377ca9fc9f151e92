"""Plain FP64 CPU oracle of restarted PDHG and the corner push (test infrastructure).

THIS IS TEST INFRASTRUCTURE, NOT THE PRODUCT.  Only the test-suite, the smoke
check and the benchmark's CPU-baseline leg may import it.  It shares no code
with the CUDA path: no kernels, headers, constants or helpers.  It is written
for a reader who checks it against the paper by eye: whole-vector numpy
operations and a scipy CSR matrix-vector product, in the order the method
states them, with no blocking, fusion or reordering.

What the paper fixes, and what is a reading (the paper prints no PDHG
iteration; Section 4.1 says its PDHG follows cuPDLP+ closely):

* LP and dual, Section 2: min c'x s.t. Ax = b, x >= 0 / max b'y s.t.
  A'y + z = c, z >= 0; inequality rows and bounds handled implicitly.
* Residuals r_P = b - Ax, r_D = c - A'y - z and the optimality conditions,
  Section 2.  Relative termination (the three A5 ratios), Section 2, with
  eps_rel = 1e-6 (Gurobi's default, Section 4.1).
* Algorithm 1 (corner push): new bounds from the reduced costs with eps_abs,
  a Uniform([0,1]^n) objective, restart from (x, 0), return (x_hat, y, z).
  Inequality rows whose (slack) reduced cost is non-trivial become '='
  (Section 3).  Corner-phase stopping rule: primal residual back at the
  original tolerance after >= 100 iterations, no dual test (Section 3.1).
* Primal/dual push estimates p - m and m - d (Section 2.1) and the candidate
  count with the 1e-6 tolerances and max(2m, 100000) threshold (Section 4.2).

Readings (the paper is silent; the cited PDLP / cuPDLP.jl family is followed):
Ruiz (10 passes) + Pock-Chambolle (alpha = 1) diagonal scaling; a constant
step eta = 0.998 / sigma_max(A_hat) from 100 power iterations; primal weight
omega_0 = ||c_hat|| / ||b_hat||; uniform averaging; KKT-based adaptive
restarts with beta = 0.2 / 0.8 / 0.36 and the theta = 0.5 primal-weight
update; checks every 64 iterations.  Each reading is listed in the design
notes with its justification.
"""
from __future__ import annotations

import math
import time

import numpy as np
import scipy.sparse as sp

EQ, LE, GE = ord("="), ord("<"), ord(">")

# solver outcome codes (same meaning as the C-ABI's report.status)
OPTIMAL, ITER_LIMIT, TIME_LIMIT, NUMERICAL = 1, 2, 3, 4
CORNER_DONE, CORNER_LIMIT = 5, 6

DEFAULTS = dict(
    eps_rel=1e-6,        # Section 4.1: Gurobi 13 default PDHG tolerance
    max_iters=1_000_000,
    time_limit_s=float("inf"),
    check_period=64,     # reading: restart / termination checks every 64 iterations
    beta_suff=0.2,       # reading: sufficient-decay restart
    beta_nec=0.8,        # reading: necessary-decay + no-progress restart
    beta_art=0.36,       # reading: artificial restart when t >= 0.36 k
    theta=0.5,           # reading: primal-weight smoothing
    eta_factor=0.998,    # reading: eta = 0.998 / sigma_max
    ruiz_iters=10,       # reading
    power_iters=100,     # reading
    algorithm="averaged",  # inner loop: "averaged" (this module) or "halpern" (oracle.halpern)
)

CORNER_DEFAULTS = dict(
    eps_abs=1e-6,        # Section 2.1 / Algorithm 1
    eps_rel=1e-6,        # the original tolerance, Section 3.1
    min_iters=100,       # Section 3.1: at least 100 corner iterations
    max_iters=1_000_000,
    time_limit_s=float("inf"),
    obj_seed=0,
    obj_scale=1.0,       # Algorithm 1: obj = Uniform([0,1]^n); Section 5 studies smaller scales
    stop_rule="primal",  # Section 3.1 rule; "kkt" (full convergence) exists for tests only
    row_rule=0,          # 0: Section 3's row rule; 1: an option, only rows active at the phase-1 point
    omega_rule=0,        # 0: omega_0 from the corner objective (reading); 1: keep phase 1's final omega
)

METRIC_TOL = 1e-6        # Section 4.2: both tolerances 1e-6


# ---------------------------------------------------------------------------
# Problem data, Section 2
# ---------------------------------------------------------------------------

def csr_matrix(lp) -> sp.csr_matrix:
    return sp.csr_matrix((np.asarray(lp["val"], dtype=np.float64),
                          np.asarray(lp["col_idx"], dtype=np.int64),
                          np.asarray(lp["row_ptr"], dtype=np.int64)),
                         shape=(lp["m"], lp["n"]))


class Model:
    """The LP in the solver's internal form: every '<' row is negated into a
    '>' row (Section 2: inequalities handled implicitly), then diagonally
    scaled, A_hat = D_r A_int D_c (reading: Ruiz + Pock-Chambolle)."""

    def __init__(self, lp, ruiz_iters=10):
        self.m, self.n = int(lp["m"]), int(lp["n"])
        sense = np.asarray(lp.get("sense", np.full(self.m, EQ)), dtype=np.int64)
        self.user_sense = sense.copy()
        self.sign = np.where(sense == LE, -1.0, 1.0)
        self.ge = sense != EQ                      # '>' after negation of '<'
        self.ineq = self.ge.copy()                 # original inequality rows
        A = csr_matrix(lp)
        self.A_user = A
        self.A_int = sp.diags(self.sign) @ A
        self.A_int = self.A_int.tocsr()
        self.b_user = np.asarray(lp["b"], dtype=np.float64)
        self.c_user = np.asarray(lp["c"], dtype=np.float64)
        self.b_int = self.sign * self.b_user
        n = self.n
        self.l = np.asarray(lp["lb"], dtype=np.float64) if lp.get("lb") is not None else np.zeros(n)
        self.u = np.asarray(lp["ub"], dtype=np.float64) if lp.get("ub") is not None else np.full(n, np.inf)
        self.Dr, self.Dc = ruiz_pock_chambolle(self.A_int, ruiz_iters)
        self.Ahat = (sp.diags(self.Dr) @ self.A_int @ sp.diags(self.Dc)).tocsr()
        self.AhatT = self.Ahat.T.tocsr()
        self.bhat = self.Dr * self.b_int
        self.set_objective(self.c_user)
        self.lhat = self.l / self.Dc
        self.uhat = self.u / self.Dc
        # rows whose dual is fixed at 0 (the dual corner model's inactive
        # inequality rows; None: no such row)
        self.y_zero = None

    def set_objective(self, c_user):
        self.c_cur = np.asarray(c_user, dtype=np.float64)
        self.chat = self.Dc * self.c_cur

    def copy(self):
        other = object.__new__(Model)
        other.__dict__.update({k: (v.copy() if isinstance(v, np.ndarray) else v)
                               for k, v in self.__dict__.items()})
        return other


def ruiz_pock_chambolle(A, ruiz_iters=10, pock_chambolle=True):
    """Reading (PDLP family): `ruiz_iters` Ruiz passes, each taking
    r_i = 1/sqrt(max_j |a_ij|) and c_j = 1/sqrt(max_i |a_ij|) of the current
    scaled matrix (1 for an empty row or column), then one Pock-Chambolle pass
    with alpha = 1: r_i = 1/sqrt(sum_j |a_ij|), c_j = 1/sqrt(sum_i |a_ij|).
    Factors multiply cumulatively.  Returns (D_r, D_c)."""
    m, n = A.shape
    absA = abs(A).tocsr()
    Dr = np.ones(m)
    Dc = np.ones(n)
    for _ in range(ruiz_iters):
        S = (sp.diags(Dr) @ absA @ sp.diags(Dc)).tocsr()
        rmax = S.max(axis=1).toarray().ravel()
        cmax = S.max(axis=0).toarray().ravel()
        r = np.where(rmax > 0, 1.0 / np.sqrt(np.where(rmax > 0, rmax, 1.0)), 1.0)
        c = np.where(cmax > 0, 1.0 / np.sqrt(np.where(cmax > 0, cmax, 1.0)), 1.0)
        Dr = Dr * r
        Dc = Dc * c
    if not pock_chambolle:
        return Dr, Dc
    S = (sp.diags(Dr) @ absA @ sp.diags(Dc)).tocsr()
    rsum = np.asarray(S.sum(axis=1)).ravel()
    csum = np.asarray(S.sum(axis=0)).ravel()
    r = np.where(rsum > 0, 1.0 / np.sqrt(np.where(rsum > 0, rsum, 1.0)), 1.0)
    c = np.where(csum > 0, 1.0 / np.sqrt(np.where(csum > 0, csum, 1.0)), 1.0)
    return Dr * r, Dc * c


def power_iteration(Ahat, AhatT, iters=100):
    """Reading: sigma_max(A_hat) by `iters` power iterations on A_hat' A_hat
    from v = 1/sqrt(n); sigma = ||A_hat v|| with ||v|| = 1 (0 if A_hat = 0)."""
    n = Ahat.shape[1]
    v = np.full(n, 1.0 / math.sqrt(n))
    for _ in range(iters):
        w = AhatT @ (Ahat @ v)
        nw = np.linalg.norm(w)
        if nw == 0.0:
            return 0.0
        v = w / nw
    return float(np.linalg.norm(Ahat @ v))


# ---------------------------------------------------------------------------
# Projections, Section 2 (bounds and senses handled implicitly)
# ---------------------------------------------------------------------------

def project_box(x, l, u):
    return np.minimum(np.maximum(x, l), u)


def project_dual_cone(lam, l, u):
    """z = proj_Lambda(lam): the reduced cost allowed by the finite bounds.
    Both finite: lam; only l finite: max(lam, 0); only u finite: min(lam, 0);
    free: 0.  For the canonical x >= 0 this is the best z >= 0 of Section 2."""
    lf, uf = np.isfinite(l), np.isfinite(u)
    z = np.zeros_like(lam)
    both = lf & uf
    z[both] = lam[both]
    lo = lf & ~uf
    z[lo] = np.maximum(lam[lo], 0.0)
    up = ~lf & uf
    z[up] = np.minimum(lam[up], 0.0)
    return z


def reduced_cost_hat(model, y_hat):
    """z_hat = proj_Lambda(c_hat - A_hat' y_hat): the scaled reduced costs."""
    return project_dual_cone(model.chat - model.AhatT @ y_hat, model.lhat, model.uhat)


def primal_residual(b, Ax, ge):
    """r_P = b - Ax on '=' rows; max(b - Ax, 0) on '>' rows (implicit slack)."""
    r = b - Ax
    r[ge] = np.maximum(r[ge], 0.0)
    return r


def dual_objective(b, y, z, l, u):
    """b'y + sum_{l finite} l_j z_j^+ - sum_{u finite} u_j z_j^-, the dual
    objective of Section 2 with finite bounds."""
    lz = np.where(np.isfinite(l), l, 0.0) * np.maximum(z, 0.0)
    uz = np.where(np.isfinite(u), u, 0.0) * np.maximum(-z, 0.0)
    return float(b @ y + lz.sum() - uz.sum())


# ---------------------------------------------------------------------------
# KKT evaluation, Section 2 (residuals, gap, relative tolerances)
# ---------------------------------------------------------------------------

def evaluate(model: Model, x, y, omega):
    """All quantities of the optimality test for a scaled iterate (x, y).

    Scaled space (restart test, reading): ||r_P_hat||^2, ||r_D_hat||^2, gap and
    KKT_omega = sqrt(omega ||r_P_hat||^2 + ||r_D_hat||^2 / omega + gap^2).
    Unscaled space (termination, Section 2): r_P = r_P_hat / D_r,
    r_D = r_D_hat / D_c, objectives (scale invariant) and the three ratios."""
    Ax = model.Ahat @ x
    rp = primal_residual(model.bhat, Ax, model.ge)
    if model.y_zero is not None:
        rp[model.y_zero] = 0.0  # a row whose dual is fixed at 0 constrains nothing
    lam = model.chat - model.AhatT @ y
    z = project_dual_cone(lam, model.lhat, model.uhat)
    rd = lam - z
    pobj = float(model.chat @ x)
    dobj = dual_objective(model.bhat, y, z, model.lhat, model.uhat)
    gap = pobj - dobj
    nrp2 = float(rp @ rp)
    nrd2 = float(rd @ rd)
    rp_u = rp / model.Dr
    rd_u = rd / model.Dc
    nb = float(np.linalg.norm(model.b_user))
    nc = float(np.linalg.norm(model.c_cur))
    rP2 = float(np.linalg.norm(rp_u))
    rD2 = float(np.linalg.norm(rd_u))
    rel_p = rP2 / (1.0 + nb)
    rel_d = rD2 / (1.0 + nc)
    rel_gap = abs(gap) / (1.0 + abs(pobj) + abs(dobj))
    return dict(nrp2=nrp2, nrd2=nrd2, gap=gap,
                kkt=math.sqrt(omega * nrp2 + nrd2 / omega + gap * gap),
                rP2=rP2, rD2=rD2,
                rPinf=float(np.max(np.abs(rp_u))) if rp_u.size else 0.0,
                rDinf=float(np.max(np.abs(rd_u))) if rd_u.size else 0.0,
                pobj=pobj, dobj=dobj, rel_p=rel_p, rel_d=rel_d, rel_gap=rel_gap,
                rel_kkt=max(rel_p, rel_d, rel_gap))


def kkt_omega(ev, omega):
    return math.sqrt(omega * ev["nrp2"] + ev["nrd2"] / omega + ev["gap"] ** 2)


# ---------------------------------------------------------------------------
# Restarted PDHG (reading of "PDHG", Sections 1-2 and 4.1)
# ---------------------------------------------------------------------------

class State:
    """Iterates in scaled space plus the restart bookkeeping."""

    def __init__(self, model: Model, x0, y0, eta, omega):
        self.x = x0.copy()
        self.y = y0.copy()
        self.sum_x = np.zeros_like(self.x)   # sum of iterates since the last restart
        self.sum_y = np.zeros_like(self.y)
        self.t = 0                           # iterations since the last restart
        self.k = 0                           # iterations in this phase
        self.eta = eta
        self.omega = omega
        self.x_r = self.x.copy()             # last restart point
        self.y_r = self.y.copy()
        self.kkt_r = kkt_omega(evaluate(model, self.x, self.y, omega), omega)
        self.kkt_prev = math.inf             # KKT_omega of the previous check's candidate
        self.restarts = 0
        # restart history: (x, z) at the start point and at every restart,
        # z = proj_Lambda(c_hat - A_hat' y) in scaled space (guidance features)
        self.ring = [(self.x.copy(), reduced_cost_hat(model, self.y))]

    @property
    def tau(self):
        return self.eta / self.omega

    @property
    def sigma(self):
        return self.eta * self.omega

    def average(self):
        return self.sum_x / self.t, self.sum_y / self.t


def pdhg_step(model: Model, s: State):
    """One PDHG iteration, primal first then dual on the extrapolated point:
    x' = proj_[l,u](x - tau (c - A'y)),  x_bar = 2 x' - x,
    y' = proj_Y(y + sigma (b - A x_bar))  (y_i >= 0 on '>' rows).
    Averages are uniform over the iterates since the last restart."""
    g = model.chat - model.AhatT @ s.y
    x_new = project_box(s.x - s.tau * g, model.lhat, model.uhat)
    x_bar = 2.0 * x_new - s.x
    y_new = s.y + s.sigma * (model.bhat - model.Ahat @ x_bar)
    y_new[model.ge] = np.maximum(y_new[model.ge], 0.0)
    if model.y_zero is not None:
        y_new[model.y_zero] = 0.0
    s.x, s.y = x_new, y_new
    s.sum_x += x_new
    s.sum_y += y_new
    s.t += 1
    s.k += 1


def restart_check(model: Model, s: State, p, ev_cur, ev_avg):
    """Reading (cuPDLP.jl-style adaptive restart): the candidate is the point
    with the smaller KKT_omega (ties: the average); restart on sufficient decay,
    on necessary decay without progress, or when t >= beta_art * k.  On restart
    the primal weight moves toward ||dy|| / ||dx|| (theta smoothing in log
    space), the iterate jumps to the candidate and the averages are reset."""
    use_avg = ev_avg["kkt"] <= ev_cur["kkt"]
    kc = ev_avg["kkt"] if use_avg else ev_cur["kkt"]
    do = (kc <= p["beta_suff"] * s.kkt_r
          or (kc <= p["beta_nec"] * s.kkt_r and kc > s.kkt_prev)
          or s.t >= p["beta_art"] * s.k)
    if not do:
        s.kkt_prev = kc
        return False
    if use_avg:
        xc, yc = s.average()
        evc = ev_avg
    else:
        xc, yc = s.x.copy(), s.y.copy()
        evc = ev_cur
    dx = float(np.linalg.norm(xc - s.x_r))
    dy = float(np.linalg.norm(yc - s.y_r))
    if dx > 1e-10 and dy > 1e-10:
        s.omega = math.exp(p["theta"] * math.log(dy / dx) + (1.0 - p["theta"]) * math.log(s.omega))
    s.x, s.y = xc, yc
    s.x_r, s.y_r = xc.copy(), yc.copy()
    s.kkt_r = kkt_omega(evc, s.omega)
    s.kkt_prev = math.inf
    s.sum_x = np.zeros_like(s.x)
    s.sum_y = np.zeros_like(s.y)
    s.t = 0
    s.restarts += 1
    s.ring.append((xc.copy(), reduced_cost_hat(model, yc)))
    del s.ring[:-8]
    return True


def initial_omega(model: Model):
    """Reading: omega_0 = ||c_hat|| / ||b_hat|| when both exceed 1e-10, else 1."""
    nc = float(np.linalg.norm(model.chat))
    nb = float(np.linalg.norm(model.bhat))
    return nc / nb if (nc > 1e-10 and nb > 1e-10) else 1.0


def setup(lp, params=None):
    p = dict(DEFAULTS)
    if params:
        p.update(params)
    model = Model(lp, p["ruiz_iters"])
    sigma_max = power_iteration(model.Ahat, model.AhatT, p["power_iters"])
    eta = p["eta_factor"] / sigma_max if sigma_max > 0 else 1.0
    return model, p, sigma_max, eta


def _pick(ev_cur, ev_avg):
    """The point to return: smaller relative KKT error, ties to the average."""
    return "avg" if ev_avg["rel_kkt"] <= ev_cur["rel_kkt"] else "cur"


def solve(lp, params=None, model=None):
    """Phase 1: restarted PDHG until max(rel_p, rel_d, rel_gap) <= eps_rel
    (Section 2, eps_rel = 1e-6 per Section 4.1) at a check, or a limit.
    params["algorithm"] == "halpern" runs the Halpern loop of oracle.halpern."""
    if params and params.get("algorithm", "averaged") == "halpern":
        from . import halpern
        return halpern.solve(lp, params, model)
    if model is None:
        model, p, sigma_max, eta = setup(lp, params)
    else:
        p = dict(DEFAULTS)
        if params:
            p.update(params)
        sigma_max = power_iteration(model.Ahat, model.AhatT, p["power_iters"])
        eta = p["eta_factor"] / sigma_max if sigma_max > 0 else 1.0
    x0 = project_box(np.zeros(model.n), model.lhat, model.uhat)
    y0 = np.zeros(model.m)
    s = State(model, x0, y0, eta, initial_omega(model))
    t0 = time.perf_counter()
    status = None
    chosen = None
    ev_cur = ev_avg = None
    while status is None:
        pdhg_step(model, s)
        at_check = s.k % p["check_period"] == 0
        at_limit = s.k >= p["max_iters"]
        if not (at_check or at_limit):
            continue
        xa, ya = s.average()
        ev_cur = evaluate(model, s.x, s.y, s.omega)
        ev_avg = evaluate(model, xa, ya, s.omega)
        if not (np.isfinite(ev_cur["kkt"]) and np.isfinite(ev_avg["kkt"])):
            status, chosen = NUMERICAL, "cur"
            break
        if at_check and min(ev_cur["rel_kkt"], ev_avg["rel_kkt"]) <= p["eps_rel"]:
            status, chosen = OPTIMAL, _pick(ev_cur, ev_avg)
            break
        if at_limit:
            status, chosen = ITER_LIMIT, _pick(ev_cur, ev_avg)
            break
        if time.perf_counter() - t0 > p["time_limit_s"]:
            status, chosen = TIME_LIMIT, _pick(ev_cur, ev_avg)
            break
        restart_check(model, s, p, ev_cur, ev_avg)
    if chosen == "avg":
        xr, yr = s.average()
        ev = ev_avg
    else:
        xr, yr = s.x.copy(), s.y.copy()
        ev = ev_cur
    return dict(status=status, iters=s.k, restarts=s.restarts, state=s, model=model,
                params=p, sigma_max=sigma_max, eta=eta, chosen=chosen,
                x_hat=xr, y_hat=yr, eval=ev, seconds=time.perf_counter() - t0)


def run_iterations(lp, iters, params=None):
    """Exactly `iters` PDHG iterations with the phase-1 restart logic (used by
    the iterate-parity tests).  Returns the State after the last step."""
    q = dict(params or {})
    q["max_iters"] = iters
    q["eps_rel"] = -1.0  # never terminate on tolerance
    return solve(lp, q)


# ---------------------------------------------------------------------------
# Unscaled solution, reduced costs and metrics
# ---------------------------------------------------------------------------

def unscale(model: Model, x_hat, y_hat):
    """(x, y, z) of the user's model: x = D_c x_hat, y = sign * D_r y_hat,
    z = proj_Lambda(c - A'y) computed in scaled space and unscaled (z = z_hat / D_c)."""
    x = model.Dc * x_hat
    y = model.sign * (model.Dr * y_hat)
    lam_hat = model.chat - model.AhatT @ y_hat
    z = project_dual_cone(lam_hat, model.lhat, model.uhat) / model.Dc
    return x, y, z


def splitmix64(seed: int, n: int) -> np.ndarray:
    """The first n outputs of the SplitMix64 generator (Steele, Lea and Flood
    2014) started at state `seed`: output j is mix(seed + (j+1) * gamma) with
    gamma = 0x9E3779B97F4A7C15 and mix the published xor-shift-multiply
    finaliser.  Counter-based: output j depends on (seed, j) only."""
    gamma = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.arange(1, n + 1, dtype=np.uint64) * gamma)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def splitmix64_uniform(seed: int, n: int) -> np.ndarray:
    """U[0,1) for j = 0..n-1: the top 53 bits of splitmix64 output j times 2^-53."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def corner_metrics(model: Model, x, y, z, tol=METRIC_TOL):
    """Section 2.1 push estimates and Section 4.2 candidate count, on the
    user's model with explicit slacks for inequality rows.

    p: structurals with min(x - l, u - x) > tol, plus inequality slacks
       (A_int x - b_int)_i > tol;
    d: structurals with |z_j| <= tol, plus inequality rows with |y_i| <= tol;
    candidates: off bound and |reduced cost| <= tol (structural + slack);
    corner measure max(0, candidates - m); primal push estimate
    max(0, p - m); dual push estimate max(0, m - d); should_corner when
    candidates >= max(2m, 100000)."""
    m = model.m
    off = np.minimum(x - model.l, model.u - x) > tol
    zero = np.abs(z) <= tol
    slack = model.A_int @ x - model.b_int
    off_s = (slack > tol) & model.ineq
    zero_s = (np.abs(y) <= tol) & model.ineq
    p = int(off.sum() + off_s.sum())
    d = int(zero.sum() + zero_s.sum())
    cand = int((off & zero).sum() + (off_s & zero_s).sum())
    return dict(off_bound_p=p, zero_rc_d=d, candidates=cand,
                corner_measure=max(0, cand - m),
                primal_push_est=max(0, p - m), dual_push_est=max(0, m - d),
                should_corner=int(cand >= max(2 * m, 100_000)))


def kkt_report(model: Model, x_hat, y_hat, omega=1.0):
    """KKT numbers and metrics of a scaled point on the user's (original) model."""
    ev = evaluate(model, x_hat, y_hat, omega)
    x, y, z = unscale(model, x_hat, y_hat)
    rep = dict(ev)
    rep.update(corner_metrics(model, x, y, z))
    return rep


# ---------------------------------------------------------------------------
# Algorithm 1: corner push PDHG (Section 3, 3.1)
# ---------------------------------------------------------------------------

def nearest_bound(x, l, u):
    """The bound of [l, u] nearest to x (ties to l); NaN where both are infinite."""
    dl = np.where(np.isfinite(l), x - l, np.inf)
    du = np.where(np.isfinite(u), u - x, np.inf)
    nb = np.where(dl <= du, l, u)
    return np.where(np.isfinite(dl) | np.isfinite(du), nb, np.nan)


def corner_model(model: Model, x_hat1, y_hat1, cp, hold=None):
    """The secondary model M_hat of Algorithm 1 in scaled space.

    z from the phase-1 point (unscaled, eps_abs):  ub_j <- x_j if z_j > eps_abs,
    lb_j <- x_j if z_j < -eps_abs (set to the iterate's own scaled value so that
    the start point stays inside the new box); inequality rows whose dual is
    non-trivial (|y_i| > eps_abs) become '=' with the same right-hand side
    (Section 3: slack upper bound fixed to zero); objective Uniform([0,1]^n)
    times obj_scale, drawn in unscaled space and scaled like c.

    `hold` (guided form, not in the paper): a boolean mask of columns to hold
    at the bound nearest to x_hat1 (l_hat = u_hat = that bound); columns the
    rule above already fixed, and columns without a finite bound, are left."""
    _, y1, z1 = unscale(model, x_hat1, y_hat1)
    cm = model.copy()
    fix_up = z1 > cp["eps_abs"]
    fix_lo = z1 < -cp["eps_abs"]
    cm.uhat = np.where(fix_up, x_hat1, model.uhat)
    cm.lhat = np.where(fix_lo, x_hat1, model.lhat)
    cm.u = np.where(fix_up, x_hat1 * model.Dc, model.u)
    cm.l = np.where(fix_lo, x_hat1 * model.Dc, model.l)
    held = np.zeros(model.n, dtype=bool)
    if hold is not None:
        nb = nearest_bound(x_hat1, model.lhat, model.uhat)
        held = np.asarray(hold, dtype=bool) & ~fix_up & ~fix_lo & np.isfinite(nb)
        cm.lhat = np.where(held, nb, cm.lhat)
        cm.uhat = np.where(held, nb, cm.uhat)
        cm.l = np.where(held, nb * model.Dc, cm.l)
        cm.u = np.where(held, nb * model.Dc, cm.u)
    to_eq = model.ge & (np.abs(y1) > cp["eps_abs"])
    if cp.get("row_rule", 0) == 1:
        # option (not the paper's): a row turns '=' only when it also looks
        # active at the phase-1 point, its slack no larger than its dual
        # (complementarity: an inactive row has slack >> |y_i|)
        x1 = model.Dc * x_hat1
        to_eq &= (model.A_int @ x1 - model.b_int) <= np.abs(y1)
    cm.ge = model.ge & ~to_eq
    cm.set_objective(cp["obj_scale"] * splitmix64_uniform(cp["obj_seed"], model.n))
    return cm, dict(fixed_upper=int(fix_up.sum()), fixed_lower=int(fix_lo.sum()),
                    rows_to_eq=int(to_eq.sum()), held=int(held.sum()),
                    fixed=fix_up | fix_lo, held_mask=held)


def corner_omega0(phase1, cm, cp):
    """The corner phase's starting primal weight.  omega_rule 0 (reading):
    ||c_hat'|| / ||b_hat|| of the corner model, as at a phase start; PDHG with
    omega proportional to ||c|| is scale-equivariant (c, y and omega scaled
    together leave the x iterates unchanged), so obj_scale then has no effect
    beyond rounding and the averaged loop's gap term.  omega_rule 1: phase 1's
    final primal weight, so that obj_scale rescales the dual's share of the
    iteration, the setting of Section 5's objective-scale study."""
    if cp.get("omega_rule", 0) == 1:
        return phase1["state"].omega
    return initial_omega(cm)


def corner_phase(phase1, corner_params=None, hold=None):
    """Algorithm 1 on the phase-1 result: build M_hat, run PDHG from (x, 0)
    with the same step size, stop once k >= min_iters and the primal residual
    of the current (else the average) point meets eps_rel (1 + ||b||) on M_hat,
    checked every check period (Section 3.1); return (x_hat, y, z) with the
    phase-1 y and z (Algorithm 1, last step).  A phase 1 run with the Halpern
    loop continues with it (oracle.halpern.corner_phase)."""
    if phase1["params"].get("algorithm", "averaged") == "halpern":
        from . import halpern
        return halpern.corner_phase(phase1, corner_params, hold)
    cp = dict(CORNER_DEFAULTS)
    if corner_params:
        cp.update(corner_params)
    model = phase1["model"]
    p = dict(phase1["params"])
    eta = phase1["eta"]
    x1, y1 = phase1["x_hat"], phase1["y_hat"]
    cm, info = corner_model(model, x1, y1, cp, hold)
    s = State(cm, project_box(x1, cm.lhat, cm.uhat), np.zeros(model.m), eta, corner_omega0(phase1, cm, cp))
    t0 = time.perf_counter()
    nb = float(np.linalg.norm(model.b_user))
    status = None
    x_corner = None
    while status is None:
        pdhg_step(cm, s)
        at_check = s.k % p["check_period"] == 0
        at_limit = s.k >= cp["max_iters"]
        if not (at_check or at_limit):
            continue
        xa, ya = s.average()
        ev_cur = evaluate(cm, s.x, s.y, s.omega)
        ev_avg = evaluate(cm, xa, ya, s.omega)
        if at_check and s.k >= cp["min_iters"] and cp["stop_rule"] == "kkt":
            if min(ev_cur["rel_kkt"], ev_avg["rel_kkt"]) <= cp["eps_rel"]:
                status = CORNER_DONE
                x_corner = xa if _pick(ev_cur, ev_avg) == "avg" else s.x.copy()
                break
        elif at_check and s.k >= cp["min_iters"]:
            if ev_cur["rP2"] <= cp["eps_rel"] * (1.0 + nb):
                status, x_corner = CORNER_DONE, s.x.copy()
                break
            if ev_avg["rP2"] <= cp["eps_rel"] * (1.0 + nb):
                status, x_corner = CORNER_DONE, xa
                break
        if at_limit or time.perf_counter() - t0 > cp["time_limit_s"]:
            status = CORNER_LIMIT
            x_corner = x1.copy()     # the phase-1 point is kept on a limit
            break
        restart_check(cm, s, p, ev_cur, ev_avg)
    return dict(status=status, iters=s.k, restarts=s.restarts, state=s, corner_model=cm,
                model=model, info=info, x_hat=x_corner, y_hat=y1.copy(),
                seconds=time.perf_counter() - t0)


# ---------------------------------------------------------------------------
# The dual corner push (Section 6, Discussion): Algorithm 1 read for the dual
# ---------------------------------------------------------------------------

def dual_corner_model(model: Model, x_hat1, y_hat1, cp):
    """The model whose PDHG run pushes the dual toward a vertex of the dual
    optimal face, in scaled space.  Section 6 proposes reducing the dual
    superbasics "with similar techniques" and gives no construction; this is
    the reading (each step is the dual counterpart of a step of Algorithm 1):

    * Complementary slackness with the phase-1 point decides (user space,
      tolerance eps_abs): of a complementary pair (the distance of x_j from
      a bound and the part of z_j that bound allows, or an inequality row's
      slack and |y_i|) the first is read as nonzero when it exceeds both
      eps_abs and the second.  A phase-1 point meets the tolerances only
      approximately, and a pair of two small numbers (an active row with a
      slack of 1.4e-6 and a dual of 0.47, say) must not be read as inactive:
      that would fix a dual the optimal face needs and leave the model's
      dual empty.
    * Columns: a bound is removed (l_j -> -inf, u_j -> +inf) where x_j is
      off it in that sense, so a column strictly inside its bounds becomes
      free and its reduced cost is fixed at 0 (Algorithm 1 fixes primal
      variables where z_j != 0; this frees them where x_j is off its bounds).
    * Rows: an inequality row whose slack (A_int x - b_int)_i is nonzero in
      that sense is inactive, and its dual is fixed at 0 (y_zero); every
      other row keeps its sense.
    * Objective: the dual objective becomes b' = obj_scale * U[0,1)^m, drawn
      per user row with SplitMix64 (seed obj_seed), in user space, then
      negated on '<' rows and scaled by D_r like b (the counterpart of
      Algorithm 1's random primal objective); c is unchanged.  Rows with a
      fixed dual get b'_i = 0 (they constrain nothing).
    On the optimal face every dual-feasible point of this model is dual
    optimal for the original LP, so maximising the random b' drives the dual
    to a vertex of the dual optimal face: at least m zero reduced costs."""
    x1, y1, z1 = unscale(model, x_hat1, y_hat1)
    dm = model.copy()
    eps = cp["eps_abs"]
    dl, du = x1 - model.l, model.u - x1
    off_l = (dl > eps) & (dl > np.maximum(z1, 0.0))
    off_u = (du > eps) & (du > np.maximum(-z1, 0.0))
    keep_l = np.isfinite(model.l) & ~off_l
    keep_u = np.isfinite(model.u) & ~off_u
    dm.l = np.where(keep_l, model.l, -np.inf)
    dm.u = np.where(keep_u, model.u, np.inf)
    dm.lhat = dm.l / model.Dc
    dm.uhat = dm.u / model.Dc
    slack = model.A_int @ x1 - model.b_int
    y_zero = model.ge & (slack > eps) & (slack > np.abs(y1))
    dm.y_zero = y_zero
    b_new = cp["obj_scale"] * splitmix64_uniform(cp["obj_seed"], model.m)
    b_new = np.where(y_zero, 0.0, b_new)
    dm.b_user = b_new
    dm.b_int = model.sign * b_new
    dm.bhat = model.Dr * dm.b_int
    return dm, dict(freed=int((~keep_l & ~keep_u).sum()), kept_lower=int(keep_l.sum()),
                    kept_upper=int(keep_u.sum()), rows_zero=int(y_zero.sum()), y_zero=y_zero)


def dual_corner_phase(phase1, corner_params=None):
    """The dual corner push on the phase-1 result: build the model of
    dual_corner_model, run PDHG from (proj(0), y1) with y1 = 0 on the rows
    whose dual is fixed (reading: Algorithm 1 keeps the pushed primal point
    and restarts the dual at 0; here the dual is pushed, so y1 is kept and
    the primal restarts at proj(0)), the same step size and omega_0 from the
    new b'; stop once k >= min_iters and the dual residual of the current
    (else the average) point meets eps_rel (1 + ||c||) on that model,
    checked every check period (the dual counterpart of Section 3.1's rule;
    stop_rule "kkt": the full test, for tests); return (x1, y_hat, z_hat) with
    phase 1's x.  On a limit the phase-1 y is kept.  A phase 1 run with the
    Halpern loop continues with it (oracle.halpern.dual_corner_phase)."""
    if phase1["params"].get("algorithm", "averaged") == "halpern":
        from . import halpern
        return halpern.dual_corner_phase(phase1, corner_params)
    cp = dict(CORNER_DEFAULTS)
    if corner_params:
        cp.update(corner_params)
    model = phase1["model"]
    p = dict(phase1["params"])
    eta = phase1["eta"]
    x1, y1 = phase1["x_hat"], phase1["y_hat"]
    dm, info = dual_corner_model(model, x1, y1, cp)
    y0 = np.where(dm.y_zero, 0.0, y1)
    s = State(dm, project_box(np.zeros(model.n), dm.lhat, dm.uhat), y0, eta, initial_omega(dm))
    t0 = time.perf_counter()
    nc = float(np.linalg.norm(model.c_user))
    status, y_out = None, None
    while status is None:
        pdhg_step(dm, s)
        at_check = s.k % p["check_period"] == 0
        at_limit = s.k >= cp["max_iters"]
        if not (at_check or at_limit):
            continue
        xa, ya = s.average()
        ev_cur = evaluate(dm, s.x, s.y, s.omega)
        ev_avg = evaluate(dm, xa, ya, s.omega)
        if at_check and s.k >= cp["min_iters"] and cp["stop_rule"] == "kkt":
            if min(ev_cur["rel_kkt"], ev_avg["rel_kkt"]) <= cp["eps_rel"]:
                status = CORNER_DONE
                y_out = ya if _pick(ev_cur, ev_avg) == "avg" else s.y.copy()
                break
        elif at_check and s.k >= cp["min_iters"]:
            if ev_cur["rD2"] <= cp["eps_rel"] * (1.0 + nc):
                status, y_out = CORNER_DONE, s.y.copy()
                break
            if ev_avg["rD2"] <= cp["eps_rel"] * (1.0 + nc):
                status, y_out = CORNER_DONE, ya
                break
        if at_limit or time.perf_counter() - t0 > cp["time_limit_s"]:
            status, y_out = CORNER_LIMIT, y1.copy()   # the phase-1 dual is kept on a limit
            break
        restart_check(dm, s, p, ev_cur, ev_avg)
    return dict(status=status, iters=s.k, restarts=s.restarts, state=s, dual_model=dm,
                model=model, info=info, x_hat=x1.copy(), y_hat=y_out,
                seconds=time.perf_counter() - t0)
