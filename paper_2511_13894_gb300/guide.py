"""Driver of the learned corner guidance: training rows from the method's own
corners, training, and a guided-versus-plain comparison.

Orchestration only: every numeric step is a C-ABI call (phase 1, Algorithm 1,
the training rows, the network's training and inference kernels); this module
only sequences the calls and collects their reports.  The comparison's hold
precision is evaluation bookkeeping on host copies of the results.
"""
from __future__ import annotations

import time

import numpy as np

from . import pdhgc as P


def build_dataset(lps, corner_seeds, corner_max_iters=300_000, phase1_params=None, capacity=None):
    """Training rows from the plain corner phase of each LP (a list of
    generator dicts): for every eligible column, its features and whether the
    corner phase left it at the bound a hold would use.  LPs whose corner
    phase hits its limit are skipped (their returned point is the phase-1
    one).  Returns a dict with the device arrays feat (rows x 32 bfloat16)
    and labels (uint8), the row count and per-LP records."""
    import torch
    if capacity is None:
        capacity = sum(int(lp["n"]) for lp in lps)
    feat = torch.zeros((capacity, P.GUIDE_FEAT_STRIDE), dtype=torch.bfloat16, device="cuda")
    labels = torch.zeros(capacity, dtype=torch.uint8, device="cuda")
    rows, records = 0, []
    t0 = time.perf_counter()
    for lp, seed in zip(lps, corner_seeds):
        g = P.lp_from_dict(lp)
        r1 = g.solve(phase1_params) if phase1_params is not None else g.solve()
        rc = g.corner_phase(obj_seed=int(seed), max_iters=int(corner_max_iters))
        used = rc["status_name"] == "CORNER_DONE"
        before = rows
        if used:
            rows = g.dataset_append(feat, labels, rows)
        records.append(dict(phase1_iters=r1["iters"], corner_status=rc["status_name"], corner_iters=rc["iters"],
                            rows=rows - before))
        g.close()
    torch.cuda.synchronize()
    return dict(feat=feat, labels=labels, rows=rows, records=records, seconds=time.perf_counter() - t0)


def train(net, data, steps=3000, batch=4096, lr=1e-3, seed=0):
    """Adam on minibatches of the dataset's rows; returns the per-step losses."""
    if data["rows"] == 0:
        raise ValueError("empty dataset")
    return net.train(data["feat"], data["labels"], rows=data["rows"], batch=batch, steps=steps, lr=lr, seed=seed)


def _nearest(x, lb, ub):
    dl = np.where(np.isfinite(lb), x - lb, np.inf)
    du = np.where(np.isfinite(ub), ub - x, np.inf)
    return np.where(dl <= du, lb, ub)


def compare(net, lp, corner_seed, threshold=0.9, corner_max_iters=300_000, guided_max_iters=0,
            phase1_params=None, upper_bound=False, extra_thresholds=()):
    """Plain corner phase versus the guided one on the same phase-1 result.
    The plain run judges the network: a held column is wrong when the plain
    corner did not leave it at the bound it was held at.  `phase1_params`
    (a Params, as for build_dataset) selects e.g. the Halpern loop.  With
    `upper_bound`, a third corner phase holds exactly the eligible columns
    the plain corner left at their hold bound (a perfect predictor, no
    fallback): the most any hold decision can gain on this LP.  Each of
    `extra_thresholds` adds a guided run without fallback at that threshold
    (its holds, wrong holds, status, iterations and seconds)."""
    import torch
    g = P.lp_from_dict(lp)
    r1 = g.solve(phase1_params) if phase1_params is not None else g.solve()
    t0 = time.perf_counter()
    rp = g.corner_phase(obj_seed=int(corner_seed), max_iters=int(corner_max_iters))
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    x_plain, _, _ = g.get_solution(P.CORNER)
    x1, _, _ = g.get_solution(P.PHASE1)
    feat, elig = g.guide_features(obj_seed=int(corner_seed))
    hold = ((net.infer(feat) >= threshold) & (elig > 0)).cpu().numpy()
    lb = np.asarray(lp["lb"]) if lp.get("lb") is not None else np.zeros(lp["n"])
    ub = np.asarray(lp["ub"]) if lp.get("ub") is not None else np.full(lp["n"], np.inf)
    at_hold_bound = np.abs(x_plain - _nearest(x1, lb, ub)) <= 1e-6
    t0 = time.perf_counter()
    rg, gr = g.corner_phase_guided(guide=net, threshold=threshold, fallback=True, guided_max_iters=guided_max_iters,
                                   obj_seed=int(corner_seed), max_iters=int(corner_max_iters))
    torch.cuda.synchronize()
    t_guided = time.perf_counter() - t0
    bound = None
    if upper_bound:
        perfect = at_hold_bound & (elig.cpu().numpy() > 0)
        t0 = time.perf_counter()
        ru, gu = g.corner_phase_guided(hold=perfect, fallback=False, guided_max_iters=guided_max_iters,
                                       obj_seed=int(corner_seed), max_iters=int(corner_max_iters))
        torch.cuda.synchronize()
        t_perfect = time.perf_counter() - t0
        bound = dict(held=gu["held"], status=ru["status_name"], iters=ru["iters"], seconds=t_perfect,
                     corner_measure=ru["corner_measure"], rel_kkt=ru["rel_kkt"],
                     speedup=t_plain / t_perfect if t_perfect > 0 else None,
                     iters_ratio=rp["iters"] / ru["iters"] if ru["iters"] else None)
    sweep = []
    probs = net.infer(feat) if extra_thresholds else None
    for th in extra_thresholds:
        h_th = ((probs >= th) & (elig > 0)).cpu().numpy()
        t0 = time.perf_counter()
        rt, gt = g.corner_phase_guided(guide=net, threshold=float(th), fallback=False,
                                       guided_max_iters=guided_max_iters, obj_seed=int(corner_seed),
                                       max_iters=int(corner_max_iters))
        torch.cuda.synchronize()
        t_th = time.perf_counter() - t0
        sweep.append(dict(threshold=float(th), held=gt["held"], wrong_holds=int((h_th & ~at_hold_bound).sum()),
                          status=rt["status_name"], iters=rt["iters"], seconds=t_th,
                          corner_measure=rt["corner_measure"],
                          speedup=t_plain / t_th if rt["status_name"] == "CORNER_DONE" and t_th > 0 else None))
    g.close()
    held = int(hold.sum())
    wrong = int((hold & ~at_hold_bound).sum())
    return dict(phase1_iters=r1["iters"], phase1_corner_measure=r1["corner_measure"],
                plain_status=rp["status_name"], plain_iters=rp["iters"], plain_seconds=t_plain,
                plain_corner_measure=rp["corner_measure"], plain_rel_kkt=rp["rel_kkt"],
                eligible=gr["eligible"], held=gr["held"], held_host=held, wrong_holds=wrong,
                precision=(held - wrong) / held if held else None,
                guided_status=gr["status_name"], guided_iters=gr["guided_iters"], fell_back=bool(gr["fell_back"]),
                final_status=rg["status_name"], final_iters=rg["iters"], final_corner_measure=rg["corner_measure"],
                final_rel_kkt=rg["rel_kkt"], guided_seconds=t_guided,
                speedup=t_plain / t_guided if t_guided > 0 else None, perfect_predictor=bound,
                thresholds=sweep)
