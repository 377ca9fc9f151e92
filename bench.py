#!/usr/bin/env python
"""Benchmark: restarted PDHG (phase 1 to rel-KKT 1e-6) + the corner-push phase
of "Backing PDHG into a Corner" on one synthetic LP per GPU.

One step = pdhgc_solve (Ruiz + Pock-Chambolle scaling, power iteration,
restarted PDHG until the Section 2 relative test holds at 1e-6; the headline
runs the Halpern loop, the cuPDLP+ form Section 4.1 names, and the averaged
loop's arms follow as blocks) followed by
pdhgc_corner_phase (Algorithm 1, Section 3.1 stopping rule, capped at
--corner-max-iters), on the LP already resident in HBM.  The reported value is
PDHG iterations per second over the whole step (phase-1 plus corner
iterations divided by step time); time-to-corner is the step time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): a single LP does not shard without
two all-gathers per iteration, so every rank solves its own replica of the
workload (weak scaling); the only collectives are the timing barrier and the
max-over-ranks reduction.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# the CPU oracle legs report one core: keep numpy's BLAS single-threaded
# (set before numpy loads; an explicit setting in the environment wins)
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

import lpgen  # noqa: E402

METRIC = "PDHG iters/s, time-to-corner at rel-KKT 1e-6, %HBM peak vs plain FP64"
FALLBACK_HBM_GBS = 6800.0
# FP64 peak from the part's published unit rate (1.25 TFLOP/s FP64 on GB300):
# one DFMA is 2 flops, so 0.625e12 FP64 operations per second for FMA-only code.
FP64_PEAK_TFLOPS = 1.25

WORKLOADS = {
    "power_law_m100k_n400k": lambda: lpgen.large_power_law_lp(0),
    "transportation_1000x2000": lambda: lpgen.large_transportation_lp(0),
    "random_face_m200_n500": lambda: lpgen.small_face_lp(0),
    # 512 uneven LPs solved together (run_batch_workload)
    "batch_512": None,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="power_law_m100k_n400k")
    ap.add_argument("--precision", choices=["fp64", "fp32", "both"], default="both",
                    help="fp64: plain FP64 only; fp32: FP32 bulk only; both: FP64 headline plus an "
                         "fp32_bulk block measured on the same workload")
    ap.add_argument("--phase1-max-iters", type=int, default=1_000_000)
    ap.add_argument("--corner-max-iters", type=int, default=200_000)
    ap.add_argument("--corner-seed", type=int, default=1)
    ap.add_argument("--row-option", action="store_true",
                    help="add the averaged loop's arms (FP64, FP32 bulk) that time the corner phase with the "
                         "row_rule = 1 option (kept out of the default run to hold its timed work near a minute)")
    ap.add_argument("--no-row-option", action="store_true", help="leave the row-option arms out (the default)")
    ap.add_argument("--corner-rows", choices=["paper", "active"], default="paper",
                    help="paper: Section 3's row rule; active: the option that keeps rows inactive at the "
                         "phase-1 point as inequalities (row_rule = 1)")
    ap.add_argument("--algorithm", choices=["averaged", "halpern", "both"], default="halpern",
                    help="inner loop of the headline: halpern (the default; FP64 headline plus an FP32-bulk "
                         "block), averaged, or both (the Halpern headline plus the averaged loop's arms)")
    ap.add_argument("--blocks", type=str, default="transport,small,batch",
                    help="comma-separated extra workloads measured after the headline (Halpern loop only): "
                         "transport (transportation_1000x2000, FP64 and FP32 bulk), small (random_face_m200_n500, "
                         "FP64), batch (batch_512); '' for none")
    ap.add_argument("--batch-handoff", type=str, default=None,
                    help="R,MIN: the batched solver's tail handoff (at most R LPs running, MIN iterations; "
                         "default: the library's)")
    ap.add_argument("--block-warmup", type=int, default=1, help="untimed steps of each extra block")
    ap.add_argument("--block-steps", type=int, default=2, help="timed steps of each extra block")
    ap.add_argument("--cpu-threads", type=int, default=0,
                    help="threads of the all-core oracle sample (0: every core os.cpu_count() reports)")
    ap.add_argument("--obj-scale-sweep", type=str, default=None,
                    help="comma-separated corner objective scales (Section 5's study): one phase 1 with the "
                         "headline loop, then one timed corner phase per scale; prints its own JSON line")
    ap.add_argument("--guidance-study", type=str, default=None,
                    help="TRAIN,TEST: the learned-guidance study on 20k x 80k power-law LPs (the guidance "
                         "configuration's size): corners of TRAIN seed-generated LPs (Halpern loop) label "
                         "the training rows, the network trains on the GPU, and TEST held-out LPs compare "
                         "the guided corner phase with the plain one; prints its own JSON line")
    ap.add_argument("--guidance-steps", type=int, default=3000, help="training steps of --guidance-study")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--profile-iters", type=int, default=50)
    ap.add_argument("--cpu-iters", type=int, default=640,
                    help="oracle iterations of the CPU baseline sample (about 10 s on the default LP)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-sample", type=int, default=16,
                    help="batch_512: LPs solved one by one with the single-LP FP64 path for the "
                         "sequential reference time (every count/sample-th LP by size)")
    ap.add_argument("--mode", choices=["bench", "kernels", "stream"], default="bench",
                    help="kernels: short solve, then --profile-iters replays of the two iteration "
                         "kernels as plain launches inside the NVTX range 'pdhg_kernels' (for ncu); "
                         "stream: phase 1 of the headline loop for --profile-iters iterations (rounded up to "
                         "check periods) with every kernel a plain stream launch (for ncu's launch list)")
    return ap.parse_args()


def aggregate(dist, total_ms, total_work, device):
    """Whole-job figures over the ranks: the slowest rank's timed region (max)
    and the work of all ranks (sum).  Single process: unchanged."""
    if dist is None:
        return float(total_ms), float(total_work)
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([float(total_work)], dtype=torch.float64, device=device)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())


def shard(items, rank, world):
    """The items of one rank when a fixed set is split round-robin."""
    return items[rank::world]


def lpt_partition(weights, world):
    """Longest-processing-time-first split of items with the given weights
    over `world` bins: items in decreasing weight (ties by index) each go to
    the bin with the smallest load so far (ties: the lowest bin).  Graham's
    bound: the largest load is at most (4/3 - 1/(3 world)) times the optimum.
    Returns one sorted index list per bin."""
    order = sorted(range(len(weights)), key=lambda k: (-weights[k], k))
    loads = [0.0] * world
    bins = [[] for _ in range(world)]
    for k in order:
        b = min(range(world), key=lambda r: (loads[r], r))
        bins[b].append(k)
        loads[b] += weights[k]
    return [sorted(b) for b in bins]


def lp_weight(lp):
    """Per-iteration cost proxy of one LP for the batch split: nonzeros plus
    rows plus columns (the bytes of an iteration grow with each)."""
    return int(lp["row_ptr"][-1]) + int(lp["m"]) + int(lp["n"])


def shard_lpt(items, weights, rank, world):
    """The items of one rank under the LPT split of their weights."""
    return [items[k] for k in lpt_partition(weights, world)[rank]]


def dist_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# the SpMV kernel and the data layout it reads: a recorded ncu traffic figure is
# valid only while these files are unchanged
KERNEL_SOURCES = ("kernels.cuh", "host_prep.h", "host_prep.cpp")


def traffic_record():
    """dram bytes per launch recorded from an ncu capture (profiles/ncu_traffic.txt),
    valid only while the kernel sources hash to the recorded value."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    rec = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                rec[k.strip()] = v.strip()
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2511_13894_gb300", "csrc")
    for fn in KERNEL_SOURCES:
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(f.read())
    if rec.get("sources_sha256") != h.hexdigest():
        return None
    return rec


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id=None):
        self.lines = []
        self.proc = None
        self.device_id = device_id

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.device_id:
            cmd += ["-i", self.device_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def algorithmic_bytes(m, n, nnz, s_v=8, s_x=8, s_sum=8, s_lo=0):
    """Bytes one PDHG iteration must move (gathers counted once per element):
    primal (A' pass): values + indices, row pointers, reads of c, l, u, x and
    the running sum, writes of x, x_bar and the running sum, y gathered once;
    dual (A pass): values + indices, row pointers, reads of b, y, the running
    sum and the sense byte, writes of y and the running sum, x_bar gathered once.
    s_v, s_x, s_sum: bytes of a matrix value, an iterate / model entry and a
    running-sum entry (8, 8, 8 in FP64; 4, 4, 8 in FP32 bulk); s_lo: bytes of
    the low part of a float-float iterate, read and written (0; 4 in FP32 bulk)."""
    primal = nnz * (s_v + 4) + n * 4 + n * (6 * s_x + 2 * s_sum + 2 * s_lo) + m * s_x
    dual = nnz * (s_v + 4) + m * 4 + m * (3 * s_x + 2 * s_sum + 2 * s_lo + 1) + n * s_x
    return primal, dual


def algorithmic_bytes_halpern(m, n, nnz):
    """Bytes per launch of the Halpern loop's kernels (FP64), a step inside a
    chunk: primal reads values + indices, column pointers, c, l, u, x and the
    anchor x_0, writes x_bar and x, gathers y once; dual reads values +
    indices, row pointers, b, y, the anchor y_0 and the sense byte, writes y,
    gathers x_bar once.  (A check step, one in 64, also writes T(z) and
    z - T(z); not counted.)"""
    primal = nnz * 12 + n * 4 + n * 7 * 8 + m * 8
    dual = nnz * 12 + m * 4 + m * (4 * 8 + 1) + n * 8
    return primal, dual


def algorithmic_bytes_halpern32(m, n, nnz):
    """Bytes per launch of the Halpern loop's FP32-bulk kernels, a step inside
    a chunk: primal reads FP32 values + int32 indices, column pointers, c, l,
    u (FP32), the float-float x (8 B) and anchor (8 B), writes x (8 B) and the
    FP32 x_bar, gathers the FP32 y once; dual reads values + indices, row
    pointers, b, the float-float y and anchor and the sense byte, writes y
    (8 B), gathers x_bar once."""
    primal = nnz * 8 + n * 4 + n * (3 * 4 + 8 + 8 + 8 + 4) + m * 4
    dual = nnz * 8 + m * 4 + m * (4 + 8 + 8 + 8 + 1) + n * 4
    return primal, dual


def fp64_ops_halpern(m, n, nnz):
    """FP64 operations per launch of the Halpern loop's kernels: one FMA per
    nonzero plus the epilogue (primal: c - A'y, the step and x_bar, which is
    also the reflected point (rho = 1), then two for the anchored combination,
    5 per column; dual: b - A x_bar, the step, the reflected point and two for
    the anchored combination, 5 per row)."""
    return nnz + 5 * n, nnz + 5 * m


def step_roofline(bytes_per_iter, total_ms, total_iters, peak):
    """The whole step's rate: the algorithmic bytes of one iteration (primal +
    dual launch) times the iterations, over the step time.  Inside the graph
    the two kernels overlap through programmatic dependent launch, and the
    check passes (one per 64 iterations) count as time but not as bytes, so
    this is the in-graph rate the headline sees, not a per-kernel figure."""
    us = total_ms * 1e3 / max(1, total_iters)
    achieved = bytes_per_iter / (us * 1e-6) / 1e9 if us > 0 else 0.0
    return {"bytes_per_iter": bytes_per_iter, "us_per_iter": us, "achieved": achieved, "unit": "GB/s",
            "peak": peak, "frac": achieved / peak if peak else None,
            "note": "algorithmic bytes of the primal + dual launch per iteration over the measured step "
                    "time per iteration (checks included)"}


def kernel_roofline(m, n, nnz, fp32, halpern, ms_primal, ms_dual, peak, peak_kind, traffic_rec):
    """Roofline of the dominant iteration kernel from its replayed duration:
    algorithmic bytes and FP64 operations per launch of the loop's kernels,
    the HBM and FP64-pipe views, the bound they name (headline_bound), and
    the recorded ncu DRAM traffic when the record matches the sources."""
    if halpern and fp32:
        b_primal, b_dual = algorithmic_bytes_halpern32(m, n, nnz)
        f_primal, f_dual = 0, 0  # float-float iterates and anchors: no FP64 work inside a chunk
    elif halpern:
        b_primal, b_dual = algorithmic_bytes_halpern(m, n, nnz)
        f_primal, f_dual = fp64_ops_halpern(m, n, nnz)
    elif not fp32:
        b_primal, b_dual = algorithmic_bytes(m, n, nnz)
        f_primal, f_dual = fp64_ops(m, n, nnz)
    else:
        b_primal, b_dual = algorithmic_bytes(m, n, nnz, s_v=4, s_x=4, s_sum=8, s_lo=4)
        f_primal, f_dual = 0, 0  # the running sums are float-float pairs: no FP64 work per launch
    dom = "primal" if ms_primal >= ms_dual else "dual"
    ms_dom, b_dom, f_dom = (ms_primal, b_primal, f_primal) if dom == "primal" else (ms_dual, b_dual, f_dual)
    achieved = b_dom / (ms_dom * 1e-3) / 1e9
    key = ("halpern32_" if halpern and fp32 else "halpern_" if halpern else "fp32_" if fp32 else "") \
        + "dram_bytes_per_launch_" + dom
    roofline = {
        # the record holds the counters of the kernels it names (null for others)
        "traffic": float(traffic_rec[key]) if traffic_rec and key in traffic_rec else None,
        "kernel": ("spmv<PrimalOp" if dom == "primal" else "spmv<DualOp")
                  + ("H32>" if halpern and fp32 else "H>" if halpern else "32>" if fp32 else ">")
                  + f" ({dom} step)",
        "algorithmic_bytes_per_launch": b_dom, "bytes_per_launch": [b_primal, b_dual], "launch_ms": ms_dom,
        "other_kernel_ms": ms_dual if dom == "primal" else ms_primal,
        "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": f"{peak_kind} hbm_gbs"},
        "fp64": {"ops_per_launch": f_dom, "achieved_tflops": 2.0 * f_dom / (ms_dom * 1e-3) / 1e12,
                 "peak_tflops": FP64_PEAK_TFLOPS,
                 "frac": 2.0 * f_dom / (ms_dom * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                 "note": "every FP64 pipe operation counted as one FMA (2 flops) against 1.25 TFLOP/s"},
    }
    return dict(headline_bound(roofline["hbm"], roofline["fp64"]), **roofline)


def headline_bound(hbm, fp64):
    """The roofline's top-level fields: the larger of the HBM and FP64-pipe
    fractions names the bound, and achieved / peak / unit / frac are that
    bound's.  The FP64 peak is the part's unit rate, 152 SMs x 2 DFMA per SM
    per clock x 2 flops x 2.07 GHz = 1.26 TFLOP/s (1.25 nominal, used)."""
    if fp64["frac"] > hbm["frac"]:
        return {"bound": "alu", "achieved": fp64["achieved_tflops"], "peak": fp64["peak_tflops"],
                "unit": "TFLOP/s", "frac": fp64["frac"],
                "peak_source": "FP64 unit rate: 152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz (1.25 nominal)"}
    return {"bound": "hbm", "achieved": hbm["achieved"], "peak": hbm["peak"], "unit": "GB/s",
            "frac": hbm["frac"], "peak_source": hbm["peak_source"]}


def fp64_ops(m, n, nnz):
    """FP64 operations per launch: one FMA per nonzero plus the epilogue
    (primal: c - A'y, the step, x_bar and the running sum, 4 per column;
    dual: b - A x_bar, the step and the running sum, 3 per row; the clamps
    run on the integer pipe)."""
    return nnz + 4 * n, nnz + 3 * m


def oracle_setup(lp):
    """The oracle's model, parameters and step size for lp (untimed setup)."""
    import oracle
    return oracle.setup(lp)


def oracle_sample(model, p, eta, iters, algorithm):
    """`iters` phase-1 steps of the oracle's loop ("averaged" or "halpern")
    from the start point, with the restart checks every check period; returns
    (seconds taken, final state).  The start point's setup (for the Halpern
    loop, the anchor's residual) is not timed."""
    import oracle
    from oracle import halpern as H
    x0 = oracle.project_box(np.zeros(model.n), model.lhat, model.uhat)
    if algorithm == "halpern":
        q = H._params(dict(p, algorithm="halpern"))
        s = H.HState(model, x0, np.zeros(model.m), eta, oracle.initial_omega(model))
        t0 = time.perf_counter()
        for _ in range(iters):
            x_pre, y_pre = H.halpern_step(model, s, q["reflection"])
            if s.k % q["check_period"] == 0:
                oracle.evaluate(model, s.xp, s.yp, s.omega)
                r = H.fixed_point_residual(model, x_pre, y_pre, s.xp, s.yp, s.tau, s.sigma)
                if H.restart_due(r, s.r0, s.r_prev, s.t, s.k, q):
                    H.apply_restart(model, s, q, r)
                else:
                    s.r_prev = r
        return time.perf_counter() - t0, s
    s = oracle.State(model, x0, np.zeros(model.m), eta, oracle.initial_omega(model))
    t0 = time.perf_counter()
    for _ in range(iters):
        oracle.pdhg_step(model, s)
        if s.k % p["check_period"] == 0:
            xa, ya = s.average()
            ec = oracle.evaluate(model, s.x, s.y, s.omega)
            ea = oracle.evaluate(model, xa, ya, s.omega)
            oracle.restart_check(model, s, p, ec, ea)
    return time.perf_counter() - t0, s


def headline_algorithm(args):
    """The loop the headline line measures: the Halpern loop unless
    --algorithm averaged (the batched workload included)."""
    if args.algorithm == "averaged":
        return "averaged"
    return "halpern"


def run_reference(args, rank, world):
    """The oracle (plain FP64 numpy/scipy, as it stands) on this machine's CPU: each
    step is a bounded sample of the workload, `cpu_iters` phase-1 PDHG
    iterations from the start on the same LP; the scaling and power-iteration
    setup runs once before the warm-up and is not timed."""
    if rank != 0:
        return
    import oracle
    if args.workload == "batch_512":
        lp = sorted(lpgen.batch_lps(512), key=lambda d: d["n"])[256]  # the median-size LP of the batch
    else:
        lp = WORKLOADS[args.workload]()
    model, p, sigma_max, eta = oracle.setup(lp)
    iters = args.cpu_iters
    alg = headline_algorithm(args)

    for _ in range(args.warmup):
        oracle_sample(model, p, eta, iters, alg)
    times = [oracle_sample(model, p, eta, iters, alg)[0] for _ in range(args.steps)]
    total = sum(times)
    value = iters * args.steps / total
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "m": lp["m"], "n": lp["n"], "nnz": int(lp["row_ptr"][-1]),
                   "precision": "fp64", "algorithm": alg, "sample_iters_per_step": iters},
        "cpu_baseline": {"value": value, "unit": "iters/s", "cores": 1, "kind": "oracle",
                         "sample": f"{iters} phase-1 PDHG iterations of the {alg} loop (with their restart "
                                   f"checks) per step on the same LP; numpy/scipy single-threaded; setup untimed"},
        "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def _replica_sample(workload, iters, algorithm, barrier, out_q):
    """One all-core replica (a spawned process): builds the workload's LP and
    the oracle's model untimed, waits at the barrier, then times `iters`
    oracle iterations."""
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    import oracle
    lp = WORKLOADS[workload]()
    model, p, sigma_max, eta = oracle.setup(lp)
    barrier.wait()
    dt, _ = oracle_sample(model, p, eta, iters, algorithm)
    out_q.put(dt)


def cpu_all_cores_sample(workload, iters, algorithm, procs):
    """The oracle on every core: `procs` spawned processes, one replica of
    the workload each (as the GPU replicas of a multi-GPU run), timed from a
    common barrier; the value is all replicas' iterations over the slowest
    one's time.  (The oracle's scipy products hold the GIL, so threads would
    not run them in parallel; a replica per core is the all-core rate.)"""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(procs)
    q = ctx.Queue()
    ps = [ctx.Process(target=_replica_sample, args=(workload, iters, algorithm, barrier, q)) for _ in range(procs)]
    for pr in ps:
        pr.start()
    times = [q.get() for _ in range(procs)]
    for pr in ps:
        pr.join()
    return {"value": procs * iters / max(times), "unit": "iters/s", "cores": procs, "kind": "oracle replicas",
            "sample": f"{procs} processes, one replica of {workload} each, {iters} phase-1 iterations of the "
                      f"{algorithm} loop per replica from a common barrier; slowest replica {max(times):.1f} s"}


def cpu_time_to_corner(lp, algorithm):
    """The oracle's own time-to-corner (phase 1 to 1e-6, then Algorithm 1 to
    the Section 3.1 rule) on a small LP, single-threaded."""
    import oracle
    t0 = time.perf_counter()
    r1 = oracle.solve(lp, dict(algorithm=algorithm))
    rc = oracle.corner_phase(r1, dict(obj_seed=1))
    return {"seconds": time.perf_counter() - t0, "phase1_iters": r1["iters"], "corner_iters": rc["iters"],
            "corner_status": "CORNER_DONE" if rc["status"] == oracle.CORNER_DONE else "CORNER_LIMIT",
            "workload": lp.get("name")}


def cpu_baseline_sample(lp, iters, algorithm="averaged", threads=0, workload=None, gpu_step_iters=None):
    """The oracle timed on this host on a bounded sample (rank 0, N = 1):
    one core, then (when `workload` names it) every core as replicas; the
    core count; the time-to-corner the one-core rate implies for the GPU
    step's iteration count; the oracle's measured time-to-corner on the
    200 x 500 LP."""
    import oracle
    t0 = time.perf_counter()
    model, p, sigma_max, eta = oracle.setup(lp)
    t_setup = time.perf_counter() - t0
    dt, _ = oracle_sample(model, p, eta, iters, algorithm)
    nproc = os.cpu_count() or 1
    out = {"value": iters / dt, "unit": "iters/s", "cores": 1, "kind": "oracle", "nproc": nproc,
           "sample": f"{iters} phase-1 PDHG iterations of the {algorithm} loop with restart checks on the same "
                     f"LP ({dt:.1f} s; scaling + power-iteration setup {t_setup:.1f} s not counted); "
                     f"numpy/scipy, single-threaded"}
    if gpu_step_iters:
        out["time_to_corner_extrapolated_s"] = gpu_step_iters / out["value"]
        out["time_to_corner_note"] = ("the GPU step's phase-1 + corner iterations at the one-core oracle rate "
                                      "(an extrapolation, not a run)")
    if workload is not None and nproc > 1:
        procs = threads if threads > 0 else nproc
        out["cores_all"] = cpu_all_cores_sample(workload, max(64, iters // 4), algorithm, procs)
    small = lpgen.small_face_lp(0)
    out["random_face_m200_n500_time_to_corner"] = cpu_time_to_corner(small, algorithm)
    return out


def batch_bytes_per_iter(lp, halpern=False):
    """Algorithmic bytes of one FP32-bulk iteration of one LP of the batch."""
    m, n, nnz = int(lp["m"]), int(lp["n"]), int(lp["row_ptr"][-1])
    if halpern:
        p, d = algorithmic_bytes_halpern32(m, n, nnz)
    else:
        p, d = algorithmic_bytes(m, n, nnz, 4, 4, 8, 4)
    return p + d


def run_batch_workload(args, rank, world, local, torch, P, dist, barrier):
    """512 uneven LPs (random-face construction, m ~ U{50..5000}) in one
    persistent, graph-captured launch with the autotuned schedule, FP32 bulk,
    the headline's inner loop.  One step = phase 1 of every LP to rel-KKT
    1e-6 plus Algorithm 1 on every LP, both in the same launch.  Ranks split
    the LPs longest-processing-time-first by their per-iteration cost
    (strong scaling: the batch is fixed).  The single-LP FP64 path on a
    size-stratified sample of the LPs, one after another, gives the
    sequential reference time."""
    all_lps = lpgen.batch_lps(512)
    lps = shard_lpt(all_lps, [lp_weight(lp) for lp in all_lps], rank, world)
    alg = headline_algorithm(args)
    algorithm = P.HALPERN if alg == "halpern" else P.AVERAGED
    stream = torch.cuda.current_stream()
    B = P.Batch(lps, stream=stream.cuda_stream)
    params = P.default_params(precision=P.FP32_BULK, max_iters=args.phase1_max_iters, algorithm=algorithm)
    tuned = B.tune(256, params)  # schedule autotuner (untimed setup)
    if args.batch_handoff:
        B.set_handoff(*(int(v) for v in args.batch_handoff.split(",")))
    cparams = P.default_corner_params(max_iters=args.corner_max_iters, obj_seed=args.corner_seed)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        # both phases of every LP in one persistent launch (no batch-wide
        # barrier between phase 1 and the corner phase)
        return B.solve_corner(params, cparams)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    clocks.start()
    l0 = B.kernel_launches()
    step_ms, iters, last = [], [], None
    byte_iters = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r1, rc = step()
        e1.record(stream)
        e1.synchronize()
        barrier()
        step_ms.append(e0.elapsed_time(e1))
        iters.append(sum(a["iters"] + b["iters"] for a, b in zip(r1, rc)))
        byte_iters += sum((a["iters"] + b["iters"]) * batch_bytes_per_iter(lp, alg == "halpern")
                          for a, b, lp in zip(r1, rc, lps))
        last = (r1, rc)
    clk = clocks.stop()
    launches = B.kernel_launches() - l0
    total_ms, total_iters = aggregate(dist, sum(step_ms), sum(iters), "cuda")
    value = total_iters / (total_ms * 1e-3)
    r1, rc = last
    peak, peak_kind = measured_peaks()
    achieved = byte_iters / (sum(step_ms) * 1e-3) / 1e9
    # sequential reference: the single-LP FP64 path, LP after LP, on a sample
    seq = None
    if rank == 0 and args.batch_sample > 0:
        order = sorted(range(len(all_lps)), key=lambda k: all_lps[k]["n"] + all_lps[k]["m"])
        stride = max(1, len(order) // args.batch_sample)
        sample = [order[k] for k in range(stride // 2, len(order), stride)][:args.batch_sample]
        t_s = 0.0
        for k in sample:
            g = P.lp_from_dict(all_lps[k], stream=stream.cuda_stream)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g.solve(max_iters=args.phase1_max_iters, algorithm=algorithm)
            g.corner_phase(cparams)
            torch.cuda.synchronize()
            t_s += time.perf_counter() - t0
            g.close()
        est = t_s * len(all_lps) / len(sample)
        seq = {"sample_lps": len(sample), "sample_seconds": t_s, "estimated_seconds_all": est,
               "speedup_batched_vs_sequential_fp64": est / (total_ms / args.steps * 1e-3),
               "note": f"single-LP FP64 path ({alg} loop, graph-driven, one LP at a time), size-stratified "
                       "sample scaled to all LPs"}
    # end to end: batch created from host arrays, both phases, every x and y back
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Be = P.Batch(lps, stream=stream.cuda_stream)
    Be.set_block(tuned["threads"])
    Be.set_layout(tuned["sell"])
    Be.set_lanes(tuned["lanes_a"], tuned["lanes_t"])
    if args.batch_handoff:
        Be.set_handoff(*(int(v) for v in args.batch_handoff.split(",")))
    a1, a2 = Be.solve_corner(params, cparams)
    d2h = 0
    for k in range(len(lps)):
        x, y = Be.get_solution(k, P.CORNER)
        d2h += x.nbytes + y.nbytes
    torch.cuda.synchronize()
    e_ms = (time.perf_counter() - t0) * 1e3
    h2d = sum(sum(np.asarray(lp[key]).nbytes for key in ("row_ptr", "col_idx", "val", "b", "c", "lb", "ub", "sense")
                  if lp.get(key) is not None) for lp in lps)
    e_it = float(sum(a["iters"] + b["iters"] for a, b in zip(a1, a2)))
    Be.close()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # 16 LPs spread over the size range, 4096 oracle iterations each (~10 s)
        by_size = sorted(all_lps, key=lambda lp: lp["n"] + lp["m"])
        picks = [by_size[k] for k in range(16, len(by_size), len(by_size) // 16)][:16]
        t_cpu, it_cpu = 0.0, 0
        for lp in picks:
            model, p, sigma_max, eta = oracle_setup(lp)
            dt, _ = oracle_sample(model, p, eta, 4096, alg)
            t_cpu += dt
            it_cpu += 4096
        cpu = {"value": it_cpu / t_cpu, "unit": "iters/s", "cores": 1, "kind": "oracle",
               "nproc": os.cpu_count(),
               "sample": f"4096 phase-1 PDHG iterations of the {alg} loop with restart checks on each of 16 LPs "
                         f"of the batch spread over its size range ({t_cpu:.1f} s; setup not counted); "
                         f"numpy/scipy, single-threaded"}
    if rank == 0:
        done = sum(r["status_name"] == "OPTIMAL" for r in r1)
        cdone = sum(r["status_name"] == "CORNER_DONE" for r in rc)
        h1 = sum(B.handed_off(k, P.PHASE1) for k in range(len(lps)))
        hc = sum(B.handed_off(k, P.CORNER) for k in range(len(lps)))
        out = {
            "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32+f32x2acc", "data": "synthetic",
            "config": {"workload": "batch_512", "algorithm": alg, "lps": len(all_lps), "lps_per_rank": len(lps),
                       "sum_m": sum(lp["m"] for lp in all_lps), "sum_n": sum(lp["n"] for lp in all_lps),
                       "sum_nnz": sum(int(lp["row_ptr"][-1]) for lp in all_lps), "precision": "fp32_bulk",
                       "schedule": tuned, "corner_max_iters": args.corner_max_iters, "eps_rel": 1e-6,
                       "l2": "flushed between steps (512 MiB write)", "parallelism": f"lpt-split x{world}"},
            "time_to_corner_s": total_ms / args.steps * 1e-3,
            "tail_handoff": {"phase1_lps": h1, "corner_lps": hc,
                             "rule": "once the queue is empty and <= 8 LPs run, an LP past 8192 iterations "
                                     "of its phase finishes on the single-LP path, concurrently"},
            "phase1": {"optimal": done, "lps": len(r1), "iters_sum": sum(r["iters"] for r in r1),
                       "iters_max": max(r["iters"] for r in r1),
                       "corner_measure_sum": sum(r["corner_measure"] for r in r1)},
            "corner": {"done": cdone, "lps": len(rc), "iters_sum": sum(r["iters"] for r in rc),
                       "iters_max": max(r["iters"] for r in rc),
                       "corner_measure_sum": sum(r["corner_measure"] for r in rc)},
            "lp_seconds": {"note": "each LP's own phase-1 + corner device time (its slowest LP bounds the step)",
                           "max": max(a["seconds"] + b["seconds"] for a, b in zip(r1, rc)),
                           "p50": float(np.median([a["seconds"] + b["seconds"] for a, b in zip(r1, rc)])),
                           "p90": float(np.percentile([a["seconds"] + b["seconds"] for a, b in zip(r1, rc)], 90)),
                           "sum": sum(a["seconds"] + b["seconds"] for a, b in zip(r1, rc))},
            "sequential_fp64": seq,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "kernel": "k_batch (whole step)",
                         "peak_source": f"{peak_kind} hbm_gbs",
                         "note": "algorithmic bytes of every LP's iterations (FP32 bulk) over the step time"},
            "cpu_baseline": cpu,
            "e2e": {"value": e_it * world / (e_ms * 1e-3), "unit": "iters/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e_ms},
            "gpu_launches": launches, "clocks": clk,
        }
        return out
    return None


def run_obj_scale_sweep(args, g, P, torch, stream):
    """Section 5's objective-scale study on the workload: Algorithm 1's random
    objective is obj_scale * U[0,1).  Phase 1 runs once (headline loop); each
    (scale, omega_rule) then gets one corner phase from the same phase-1
    point, timed with CUDA events, reporting iterations, status, the corner
    measure and the primal push estimate of its result.  omega_rule 0 starts
    the corner phase's primal weight from the scaled objective (the phase is
    then scale-equivariant); 1 keeps phase 1's weight, the setting in which
    the scale changes the dual's share of the iteration."""
    alg = P.HALPERN if headline_algorithm(args) == "halpern" else P.AVERAGED
    r1 = g.solve(P.default_params(max_iters=args.phase1_max_iters, algorithm=alg))
    rows_rule = 1 if args.corner_rows == "active" else 0

    def cparams(scale, omega_rule):
        return P.default_corner_params(max_iters=args.corner_max_iters, obj_seed=args.corner_seed,
                                       obj_scale=scale, row_rule=rows_rule, omega_rule=omega_rule)

    scales = [float(v) for v in args.obj_scale_sweep.split(",")]
    g.corner_phase(cparams(scales[0], 1))  # warm-up
    rows = []
    for omega_rule in (1, 0):
        for scale in scales:
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc = g.corner_phase(cparams(scale, omega_rule))
            e1.record(stream)
            e1.synchronize()
            rows.append({"obj_scale": scale, "omega_rule": omega_rule, "status": rc["status_name"],
                         "iters": rc["iters"], "restarts": rc["restarts"], "ms": e0.elapsed_time(e1),
                         "corner_measure": rc["corner_measure"], "primal_push_est": rc["primal_push_est"],
                         "candidates": rc["candidates"], "off_bound_p": rc["off_bound_p"],
                         "rel_kkt": rc["rel_kkt"]})
    print(json.dumps({"mode": "obj_scale_sweep", "workload": args.workload,
                      "algorithm": "halpern" if alg == P.HALPERN else "averaged",
                      "corner_rows": args.corner_rows, "corner_max_iters": args.corner_max_iters,
                      "phase1": {"status": r1["status_name"], "iters": r1["iters"], "omega": r1["omega"],
                                 "corner_measure": r1["corner_measure"], "primal_push_est": r1["primal_push_est"]},
                      "runs": rows}), flush=True)


def run_guidance_study(args, torch, P):
    """The learned-guidance study at 20k x 80k (m, n of the guidance
    configuration; power-law construction, |S| = m + 1000).  Training rows
    come from the plain corner phases of `train` LPs (seeds 0..train-1, each
    with the Halpern loop's phase 1 and Algorithm 1 under Section 3's row
    rule); the network trains with the library's kernels; each of `test`
    held-out LPs (seeds 1000..) runs phase 1 once, then the plain and the
    guided corner phase from it.  Reports the dataset, the loss against the
    label entropy, and per held-out LP the two corner phases' iterations,
    seconds and status, the holds and their precision as the plain corner
    judges them, and the plain/guided time ratio; beside them the guided
    run at higher thresholds (no fallback) and a perfect predictor that
    holds exactly the columns the plain corner left at their hold bound."""
    from paper_2511_13894_gb300 import guide as G
    n_train, n_test = (int(v) for v in args.guidance_study.split(","))
    p1 = P.default_params(max_iters=args.phase1_max_iters, algorithm=P.HALPERN)
    t0 = time.perf_counter()
    train_lps = [lpgen.guidance_lp(s) for s in range(n_train)]
    t_gen = time.perf_counter() - t0
    data = G.build_dataset(train_lps, [s + 1 for s in range(n_train)], corner_max_iters=args.corner_max_iters,
                           phase1_params=p1)
    del train_lps
    rows = int(data["rows"])
    pos = float(data["labels"][:rows].float().mean().item()) if rows else 0.0
    entropy = -(pos * math.log(pos) + (1 - pos) * math.log(1 - pos)) if 0 < pos < 1 else 0.0
    net = P.Guide(seed=0)
    t0 = time.perf_counter()
    losses = G.train(net, data, steps=args.guidance_steps, batch=4096, lr=1e-3, seed=5) if rows else []
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    tests = []
    for s in range(1000, 1000 + n_test):
        r = G.compare(net, lpgen.guidance_lp(s), s + 1, threshold=0.9, corner_max_iters=args.corner_max_iters,
                      guided_max_iters=2 * 64 * 1024, phase1_params=p1, upper_bound=True,
                      extra_thresholds=(0.97, 0.995))
        r["seed"] = s
        tests.append(r)
    done = [r for r in tests if r["plain_status"] == "CORNER_DONE" and r["final_status"] == "CORNER_DONE"]
    print(json.dumps({
        "mode": "guidance_study", "workload": "power_law_m20k_n80k", "algorithm": "halpern",
        "train_lps": n_train, "test_lps": n_test, "generate_seconds": t_gen,
        "dataset": {"rows": rows, "positive_frac": pos, "seconds": data["seconds"], "records": data["records"]},
        "training": {"steps": args.guidance_steps, "seconds": t_train, "label_entropy": entropy,
                     "loss_first50": float(np.mean(losses[:50])) if len(losses) else None,
                     "loss_last50": float(np.mean(losses[-50:])) if len(losses) else None},
        "held_out": tests,
        "time_ratio_plain_over_guided": [r["speedup"] for r in done],
        "time_ratio_plain_over_perfect_predictor": [r["perfect_predictor"]["speedup"] for r in done
                                                    if r["perfect_predictor"]["status"] == "CORNER_DONE"],
        "by_threshold": [{"threshold": t["threshold"],
                          "corner_done": sum(r["thresholds"][k]["status"] == "CORNER_DONE" for r in tests),
                          "mean_wrong_holds": float(np.mean([r["thresholds"][k]["wrong_holds"] for r in tests])),
                          "time_ratio_plain_over_guided": [r["thresholds"][k]["speedup"] for r in tests
                                                           if r["plain_status"] == "CORNER_DONE"]}
                         for k, t in enumerate(tests[0]["thresholds"])] if tests else [],
        "data": "synthetic (seeded power-law LPs; the paper's models are not available)",
    }), flush=True)


def corner_speedup(base, other):
    """Time-to-corner speedup of `other` over `base` (ratio of their step
    times), reported only when every timed step of both arms ended its
    corner phase at Section 3.1's rule (CORNER_DONE); otherwise null with
    the reason, so that two runs stopped at a limit are never compared."""
    sb = [rc["status_name"] for _, rc in base["reps"]]
    so = [rc["status_name"] for _, rc in other["reps"]]
    ok = all(v == "CORNER_DONE" for v in sb + so)
    return {"value": (base["total_ms"] / other["total_ms"]) if ok and other["total_ms"] > 0 else None,
            "base_corner_status": sorted(set(sb)), "corner_status": sorted(set(so)),
            "reason": None if ok else "a corner phase stopped at its limit: no time-to-corner to compare"}


def main():
    args = parse()
    rank, world, local = dist_info()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    from paper_2511_13894_gb300 import pdhgc as P

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    if args.guidance_study:
        if rank == 0:
            run_guidance_study(args, torch, P)
        if dist is not None:
            dist.destroy_process_group()
        return
    if args.workload == "batch_512" and args.mode == "kernels":
        # --profile-iters iterations of every LP in one batched launch (FP32 bulk), for ncu
        B = P.Batch(lpgen.batch_lps(512), stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("batch_kernel")
        B.solve(max_iters=args.profile_iters, eps_rel=-1.0, precision=P.FP32_BULK,
                algorithm=P.HALPERN if args.algorithm == "halpern" else P.AVERAGED)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"mode": "kernels", "workload": "batch_512", "iters": args.profile_iters}))
        return
    if args.workload == "batch_512":
        out = run_batch_workload(args, rank, world, local, torch, P, dist, barrier)
        if rank == 0 and out is not None:
            print(json.dumps(out), flush=True)
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return

    lp_dict = WORKLOADS[args.workload]()
    m, n, nnz = lp_dict["m"], lp_dict["n"], int(lp_dict["row_ptr"][-1])
    stream = torch.cuda.current_stream()
    g = P.lp_from_dict(lp_dict, stream=stream.cuda_stream)
    if args.mode == "kernels":
        g.solve(max_iters=64, precision=P.FP32_BULK if args.precision == "fp32" else P.FP64,
                algorithm=P.AVERAGED if args.algorithm == "averaged" else P.HALPERN)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("pdhg_kernels")
        ms = g.profile_iteration(args.profile_iters)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"mode": "kernels", "workload": args.workload, "primal_ms": ms[0], "dual_ms": ms[1]}))
        return
    if args.mode == "stream":
        iters = max(64, -(-args.profile_iters // 64) * 64)
        g.set_launch_mode(P.LAUNCH_STREAM)
        l0 = g.kernel_launches()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = g.solve(max_iters=iters, eps_rel=-1.0, precision=P.FP32_BULK if args.precision == "fp32" else P.FP64,
                      algorithm=P.AVERAGED if args.algorithm == "averaged" else P.HALPERN)
        torch.cuda.synchronize()
        print(json.dumps({"mode": "stream", "workload": args.workload, "iters": rep["iters"],
                          "launches": g.kernel_launches() - l0, "seconds": time.perf_counter() - t0}))
        return
    if args.obj_scale_sweep:
        run_obj_scale_sweep(args, g, P, torch, stream)
        return
    cparams = P.default_corner_params(max_iters=args.corner_max_iters, obj_seed=args.corner_seed,
                                      row_rule=1 if args.corner_rows == "active" else 0)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    peak, peak_kind = measured_peaks()

    def run_arm(h, dims, precision, cparams=cparams, algorithm=P.HALPERN, warmup=None, steps=None):
        """Times `steps` steps (phase 1 + corner phase) of handle h after
        `warmup` untimed ones, L2 flushed between steps; then the kernel
        replays, the roofline and the gather ceiling."""
        warmup = args.warmup if warmup is None else warmup
        steps = args.steps if steps is None else steps
        mm, nn, nz = dims
        params = P.default_params(max_iters=args.phase1_max_iters, precision=precision, algorithm=algorithm)
        halpern = algorithm == P.HALPERN

        def step():
            r1 = h.solve(params)
            rc = h.corner_phase(cparams)
            return r1, rc

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        clocks = ClockSampler(uuid)
        clocks.start()
        launches0 = h.kernel_launches()
        step_ms, iters, reps = [], [], []
        for _ in range(steps):
            flush.fill_(1.0)  # L2 flush: 512 MiB write between steps
            torch.cuda.synchronize()
            barrier()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r1, rc = step()
            e1.record(stream)
            e1.synchronize()
            barrier()
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            iters.append(r1["iters"] + rc["iters"])
            reps.append((r1, rc))
        launches = h.kernel_launches() - launches0
        clk = clocks.stop()
        total_iters = sum(iters)
        total_ms, total_iters_all = aggregate(dist, sum(step_ms), total_iters, "cuda")
        value = total_iters_all / (total_ms * 1e-3)
        # kernel durations: event-bracketed replays of the two iteration kernels
        ms_primal, ms_dual = h.profile_iteration(args.profile_iters)
        roofline = kernel_roofline(mm, nn, nz, precision == P.FP32_BULK, halpern, ms_primal, ms_dual, peak,
                                   peak_kind, traffic_record())
        dom = "primal" if ms_primal >= ms_dual else "dual"
        ms_dom = roofline["launch_ms"]
        b_primal, b_dual = roofline["bytes_per_launch"]
        # the random-gather ceiling: the same number of random loads from a
        # vector of the gathered length, warm in L2 (pdhgc_probe_gather)
        g_len = mm if dom == "primal" else nn
        g_bytes = 8 if precision == P.FP64 else 4
        ms_g = P.probe_gather(g_len, nz, g_bytes, reps=20)
        roofline["gather"] = {"gathers_per_launch": nz, "vector_elems": g_len, "elem_bytes": g_bytes,
                              "ceiling_ms": ms_g, "ceiling_gathers_per_s": nz / (ms_g * 1e-3),
                              "achieved_gathers_per_s": nz / (ms_dom * 1e-3), "frac": ms_g / ms_dom,
                              "note": "pdhgc_probe_gather: the same count of random loads alone, at the "
                                      "steady-state rate of a launch of 16 times as many"}
        roofline["step"] = step_roofline(b_primal + b_dual, total_ms, total_iters, peak)
        r1, rc = reps[-1]
        return dict(value=value, total_ms=total_ms, steps=steps, warmup=warmup, total_iters=total_iters,
                    launches=launches, clocks=clk, roofline=roofline, r1=r1, rc=rc, reps=reps, params=params)

    def summary(res):
        r1, rc = res["r1"], res["rc"]
        return {
            "phase1": {"status": r1["status_name"], "iters": r1["iters"], "restarts": r1["restarts"],
                       "rel_kkt": r1["rel_kkt"], "seconds": r1["seconds"], "corner_measure": r1["corner_measure"],
                       "candidates": r1["candidates"], "off_bound_p": r1["off_bound_p"],
                       "primal_push_est": r1["primal_push_est"], "should_corner": r1["should_corner"]},
            "corner": {"status": rc["status_name"], "iters": rc["iters"], "restarts": rc["restarts"],
                       "seconds": rc["seconds"], "corner_measure": rc["corner_measure"],
                       "candidates": rc["candidates"], "off_bound_p": rc["off_bound_p"],
                       "primal_push_est": rc["primal_push_est"], "rel_p": rc["rel_p"], "rel_kkt": rc["rel_kkt"]},
            "us_per_iter": res["total_ms"] * 1e3 / max(1, res["total_iters"]),
        }

    def block(res, note, dtype):
        b = {"note": note, "dtype": dtype, "value": res["value"], "unit": "iters/s",
             "steps": res["steps"], "warmup": res["warmup"],
             "time_to_corner_s": res["total_ms"] / res["steps"] * 1e-3,
             "roofline": res["roofline"], "gpu_launches": res["launches"], "clocks": res["clocks"]}
        b.update(summary(res))
        return b

    f32_dtype = "f32 values and gathers; float-float iterates, anchors and row sums; f64 checks and KKT"
    dims = (m, n, nnz)
    head_alg = headline_algorithm(args)
    arms = {}
    if head_alg == "halpern":
        arms["halpern"] = run_arm(g, dims, P.FP64)
        if args.precision in ("fp32", "both"):
            arms["halpern_fp32"] = run_arm(g, dims, P.FP32_BULK)
    if args.algorithm in ("averaged", "both"):
        if args.precision in ("fp64", "both"):
            arms["fp64"] = run_arm(g, dims, P.FP64, algorithm=P.AVERAGED)
        if args.precision in ("fp32", "both"):
            arms["fp32"] = run_arm(g, dims, P.FP32_BULK, algorithm=P.AVERAGED)
        if args.corner_rows == "paper" and args.row_option and not args.no_row_option and args.precision == "both":
            cp_opt = P.default_corner_params(max_iters=args.corner_max_iters, obj_seed=args.corner_seed,
                                             row_rule=1)
            arms["fp64_rows"] = run_arm(g, dims, P.FP64, cp_opt, algorithm=P.AVERAGED)
            arms["fp32_rows"] = run_arm(g, dims, P.FP32_BULK, cp_opt, algorithm=P.AVERAGED)
    if head_alg == "halpern":
        head = arms["halpern"]
    else:
        head = arms["fp64"] if "fp64" in arms else arms["fp32"]
    params = head["params"]
    value = head["value"]
    total_ms = head["total_ms"]
    launches = head["launches"]
    clk = head["clocks"]
    roofline = head["roofline"]

    # the other single-GPU workload: the degenerate transportation LP
    # (1000 x 2000, n = 2M), Halpern loop in FP64 and FP32 bulk
    extra = {}
    if head_alg == "halpern" and args.workload != "transportation_1000x2000" and "transport" in args.blocks:
        lt = lpgen.large_transportation_lp(0)
        dt = (lt["m"], lt["n"], int(lt["row_ptr"][-1]))
        gt = P.lp_from_dict(lt, stream=stream.cuda_stream)
        t64 = run_arm(gt, dt, P.FP64, warmup=args.block_warmup, steps=args.block_steps)
        t32 = run_arm(gt, dt, P.FP32_BULK, warmup=args.block_warmup, steps=args.block_steps)
        gt.close()
        extra["transportation_1000x2000"] = {
            "config": {"workload": "transportation_1000x2000", "m": dt[0], "n": dt[1], "nnz": dt[2],
                       "algorithm": "halpern", "corner_rows": args.corner_rows,
                       "l2": "flushed between steps (512 MiB write)"},
            "fp64": block(t64, "Halpern loop, FP64", "f64"),
            "fp32_bulk": block(t32, "Halpern loop, FP32 bulk", f32_dtype),
            "speedup_fp32_vs_fp64_time_to_corner": corner_speedup(t64, t32),
        }
    if head_alg == "halpern" and args.workload != "random_face_m200_n500" and "small" in args.blocks:
        # the 200 x 500 face LP: launch- and latency-bound, not a roofline case
        # (its iteration touches about 0.1 MB); phase 1 + corner phase per step
        ls = lpgen.small_face_lp(0)
        ds = (ls["m"], ls["n"], int(ls["row_ptr"][-1]))
        gs = P.lp_from_dict(ls, stream=stream.cuda_stream)
        s64 = run_arm(gs, ds, P.FP64, warmup=3, steps=10)
        gs.close()
        sb = block(s64, "Halpern loop, FP64; latency-bound (about 0.1 MB per iteration): iterations/s and "
                        "microseconds per iteration, not a roofline case", "f64")
        sb.pop("roofline")
        extra["random_face_m200_n500"] = {
            "config": {"workload": "random_face_m200_n500", "m": ds[0], "n": ds[1], "nnz": ds[2],
                       "algorithm": "halpern", "corner_rows": args.corner_rows},
            "fp64": sb,
        }
    if head_alg == "halpern" and "batch" in args.blocks and world == 1:
        bargs = argparse.Namespace(**vars(args))
        bargs.warmup, bargs.steps = args.block_warmup, args.block_steps
        extra["batch_512"] = run_batch_workload(bargs, rank, world, local, torch, P, None, barrier)

    # end-to-end through the public API with host buffers (pinned), per step:
    # H2D of the inputs in lp_create, solve, corner, D2H of x, y, z
    e2e = None
    if args.e2e_steps > 0:
        host = {}
        h2d = 0
        for k in ("row_ptr", "col_idx", "val", "b", "c", "lb", "ub", "sense"):
            a = np.ascontiguousarray(lp_dict[k])
            t = torch.from_numpy(a).pin_memory()
            host[k] = t.numpy()
            h2d += a.nbytes
        host["m"], host["n"] = m, n
        d2h = 8 * (2 * n + m)
        e_ms, e_it = [], []
        for _ in range(args.e2e_steps):
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            ge = P.lp_from_dict(host, stream=stream.cuda_stream)
            a1 = ge.solve(params)
            a2 = ge.corner_phase(cparams)
            ge.get_solution(P.CORNER)
            torch.cuda.synchronize()
            e_ms.append((time.perf_counter() - t0) * 1e3)
            e_it.append(a1["iters"] + a2["iters"])
            ge.close()
        e_total = sum(e_ms)
        if dist is not None:
            t = torch.tensor([e_total], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e_total = float(t.item())
        e2e = {"value": sum(e_it) * world / (e_total * 1e-3), "unit": "iters/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": e_total / args.e2e_steps}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample(lp_dict, args.cpu_iters, head_alg, args.cpu_threads, args.workload,
                                  head["r1"]["iters"] + head["rc"]["iters"])

    if rank == 0:
        head_is_fp64 = head_alg == "halpern" or "fp64" in arms
        out = {
            "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if head_is_fp64 else "f32+f32x2acc",
            "data": "synthetic",
            "config": {"workload": args.workload, "m": m, "n": n, "nnz": nnz,
                       "precision": "fp64" if head_is_fp64 else "fp32_bulk",
                       "phase1_max_iters": args.phase1_max_iters, "corner_max_iters": args.corner_max_iters,
                       "corner_seed": args.corner_seed, "corner_rows": args.corner_rows, "eps_rel": 1e-6,
                       "algorithm": head_alg,
                       "l2": "flushed between steps (512 MiB write)", "parallelism": f"replicas x{world}"},
            "time_to_corner_s": total_ms / args.steps * 1e-3,
        }
        out.update(summary(head))
        out.update({"roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                    "clocks": clk})
        if "halpern_fp32" in arms:
            b = block(arms["halpern_fp32"], "Halpern loop, FP32 bulk, same workload and corner rule", f32_dtype)
            b["speedup_vs_fp64_time_to_corner"] = corner_speedup(arms["halpern"], arms["halpern_fp32"])
            out["halpern_fp32_bulk"] = b
        if head_alg == "halpern" and "fp64" in arms:
            b = block(arms["fp64"], "the averaged loop (cuPDLP.jl-style restarts on the KKT error of the "
                                    "current and average points), FP64, the paper's corner row rule", "f64")
            b["halpern_speedup_time_to_corner"] = corner_speedup(arms["fp64"], arms["halpern"])
            out["averaged_fp64"] = b
        if "fp32" in arms:
            b = block(arms["fp32"], "the averaged loop, FP32 bulk", f32_dtype)
            if "fp64" in arms:
                b["speedup_vs_averaged_fp64_time_to_corner"] = corner_speedup(arms["fp64"], arms["fp32"])
            out["averaged_fp32_bulk"] = b
        if "fp64_rows" in arms:
            a64, a32 = arms["fp64_rows"], arms["fp32_rows"]
            out["corner_row_option"] = {
                "note": "corner phase with row_rule = 1 (an option, not the paper's rule): a row becomes '=' "
                        "only when its dual is non-trivial and it is active at the phase-1 point",
                "fp64": block(a64, "averaged loop, FP64, row option", "f64"),
                "fp32_bulk": block(a32, "averaged loop, FP32 bulk, row option", f32_dtype),
                "speedup_fp32_vs_fp64_time_to_corner": corner_speedup(a64, a32)}
        out.update(extra)
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
