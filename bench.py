"""Throughput benchmark of the smooth contact-manifold library on GB300.

Headline workload: 65536 independent pairs in one batch, each the convex hull of
N points uniform in the unit ball (N log-uniform in [8, 256], a pool of 4096
hulls) against a random smooth primitive (box, capsule, cylinder, ellipsoid;
dims U[0.2, 1]), tau drawn per pair from {1e-3, 1e-2, 1e-1}, penetration
U[0, 0.1] (every pair in contact), K = 8, FP32.  A step is one forward and
backward manifold over the whole batch (work ordering, forward kernel, work
ordering, adjoint kernel) replayed as one CUDA graph with autotuned launch
shapes.  Inputs are resident in HBM; L2 is flushed (512 MB write) between timed
steps.  The forward alone, the adjoint kernel (the difference of the two steps'
times) and the other settings are reported beside.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
(forward and backward) on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = ("65536 uneven pairs: hull(8-256 pts, log-uniform, pool of 4096) vs box/capsule/cylinder/ellipsoid "
            "(dims U[0.2,1]), tau in {1e-3,1e-2,1e-1}, penetration U[0,0.1], K=8")
WORKLOAD_2 = "hull(8-64 pts) vs primitive, 4096 pairs, tau=1e-2, K=8"
HEADLINE_PAIRS = 65536


# ----------------------------------------------------------------- algorithmic work
# MUFU (transcendental) operations the method needs, counted once per evaluation
# as the definition requires: exp / log / reciprocal / sqrt / rsqrt each 1.
def _sdf_mufu(kind, n_planes):
    if kind in (synth.KIND_BOX, synth.KIND_HULL):
        F = 6 if kind == synth.KIND_BOX else n_planes
        return F + 2            # F exps, one log, one reciprocal (value + gradient of the LSE)
    if kind == synth.KIND_ELLIPSOID:
        return 2                # |y| and f^-1/2
    if kind == synth.KIND_CAPSULE:
        return 6                # e^-|x| per clip side (2), log of the softplus ratio, two sigmoid reciprocals, 1/|w|
    if kind == synth.KIND_CYLINDER:
        return 7                # rho, 1/rho, 3-term LSE (3 exp, log, rcp)
    raise ValueError(kind)


QP_MUFU = 29        # 3 reciprocals, 4 soft clips (16), soft argmin (4 exp + rcp), 4 sigmoids under one reciprocal (5)
EE_EXTRA = 2 + 2 + 4 + 4 + 2 + 4 + 2   # dbar, nbar, 2 soft signs, 2 pen, cl, nn (2 row/col exps + 2 values), SoftSort 2
VS_EXTRA = 1 + 2 + 1                   # normal, activity sigmoid, SoftSort


def mufu_ops_per_pair(w, flags=0):
    nvA, nvB, neA, neB = w.pair_counts()
    out = np.zeros(w.n_pairs)
    for i in range(w.n_pairs):
        ga, gb = w.geoms[w.pair_geoms[i, 0]], w.geoms[w.pair_geoms[i, 1]]
        sa, sb = _sdf_mufu(ga.kind, ga.n_planes), _sdf_mufu(gb.kind, gb.n_planes)
        vs = nvA[i] * (sb + VS_EXTRA) + (0 if flags & 2 else nvB[i] * (sa + VS_EXTRA))
        ee = 0 if flags & 3 else neA[i] * neB[i] * (QP_MUFU + EE_EXTRA + 2 * sa + 2 * sb)
        out[i] = vs + ee
    return out


# FP32 operations of the method (FMA = 2, add / mul / min / max = 1), from the formulas
# the oracle evaluates, per SDF evaluation ("grad": value and gradient) and per step.
def _sdf_flops(kind, n_planes, grad):
    if kind == synth.KIND_HULL:            # per plane: n . y - o (6), shift (1), sum (1); gradient 3 FMA
        return n_planes * (14 if grad else 8) + (6 if grad else 3)
    if kind == synth.KIND_BOX:             # six axis planes (+-y_i - h_i), same LSE
        return 39 if grad else 33
    if kind == synth.KIND_ELLIPSOID:
        return 21
    if kind == synth.KIND_CAPSULE:
        return 40
    if kind == synth.KIND_CYLINDER:
        return 25
    raise ValueError(kind)


QP_FLOPS = 260      # set-up (38), unconstrained solve (60), 4 soft clips (68), 4 side costs (40), soft argmin, indicator, blend
EE_FLOPS = 180      # witnesses, n-bar, frame moves, 2 normals, soft signs, pen, cl, nn, weights, 2 SoftSort pushes, row/col minima
VS_FLOPS = 34       # normal, activity, score, SoftSort push


def fp32_flops_per_pair(w, flags=0):
    nvA, nvB, neA, neB = w.pair_counts()
    out = np.zeros(w.n_pairs)
    for i in range(w.n_pairs):
        ga, gb = w.geoms[w.pair_geoms[i, 0]], w.geoms[w.pair_geoms[i, 1]]
        vs = nvA[i] * (_sdf_flops(gb.kind, gb.n_planes, True) + VS_FLOPS)
        if not flags & 2:
            vs += nvB[i] * (_sdf_flops(ga.kind, ga.n_planes, True) + VS_FLOPS)
        ee = 0 if flags & 3 else neA[i] * neB[i] * (
            QP_FLOPS + EE_FLOPS + _sdf_flops(ga.kind, ga.n_planes, False) + _sdf_flops(ga.kind, ga.n_planes, True)
            + _sdf_flops(gb.kind, gb.n_planes, False) + _sdf_flops(gb.kind, gb.n_planes, True))
        out[i] = vs + ee
    return out


# Reverse-mode work of the adjoint, counted from the derivative formulas (the kernel's
# own recomputation is not counted): the adjoint's algorithmic work is the forward's
# (it needs every forward value) plus this.
#   per SDF evaluation (value at one point; value and gradient at the other, whose
#   normal needs the Hessian-vector product): a hull's reverse comes from moments the
#   forward pass over its planes accumulates -- the gradient at the value point (3 flops
#   per plane) and sum_f pi_f n_f n_f^T at the other (9 per plane) -- then
#   phibar g + H gbar (5 / 25 flops, no transcendental); a box's six planes are reversed
#   one by one (1 exp and 14 / 22 flops each); ellipsoid 2 MUFU and 30 / 50 flops;
#   capsule 6 and 80 / 110; cylinder 5 and 60 / 90;
#   per edge pair: SoftSort reverse of two candidates (one exp and 50 flops each),
#   indicators, soft signs and normals 200 flops, witnesses and the QP's smoothed
#   active set 420 flops and 24 MUFU (the derivatives of 4 soft clips and 2 soft
#   comparisons), distance-matrix adjoint 52 flops and 2 exps;
#   per vertex candidate: SoftSort reverse (1 exp, 50 flops), normal, activity and frame 70.
def _sdf_bwd_mufu(kind, n_planes):
    if kind == synth.KIND_HULL:
        return 0
    if kind == synth.KIND_BOX:
        return 6
    return {synth.KIND_ELLIPSOID: 2, synth.KIND_CAPSULE: 6, synth.KIND_CYLINDER: 5}[kind]


def _sdf_bwd_flops(kind, n_planes, grad):
    if kind == synth.KIND_HULL:
        return n_planes * (9 if grad else 3) + (25 if grad else 5)
    if kind == synth.KIND_BOX:
        return 6 * (22 if grad else 14) + 10
    return {synth.KIND_ELLIPSOID: (30, 50), synth.KIND_CAPSULE: (80, 110),
            synth.KIND_CYLINDER: (60, 90)}[kind][1 if grad else 0]


SS_BWD = (1, 50)            # SoftSort reverse of one candidate: (MUFU, flops)
EE_BWD = (24 + 2, 200 + 420 + 52)
VS_BWD_FLOPS = 70


def bwd_work_per_pair(w, flags=0):
    """(FP32 flops, MUFU ops) per pair of one adjoint launch: forward work plus reverse work."""
    nvA, nvB, neA, neB = w.pair_counts()
    flops = fp32_flops_per_pair(w, flags).copy()
    mufu = mufu_ops_per_pair(w, flags).copy()
    for i in range(w.n_pairs):
        ga, gb = w.geoms[w.pair_geoms[i, 0]], w.geoms[w.pair_geoms[i, 1]]
        fa, fb = ga.n_planes, gb.n_planes
        vs_n = nvA[i] + (0 if flags & 2 else nvB[i])
        flops[i] += vs_n * (SS_BWD[1] + VS_BWD_FLOPS) + nvA[i] * _sdf_bwd_flops(gb.kind, fb, True)
        mufu[i] += vs_n * SS_BWD[0] + nvA[i] * _sdf_bwd_mufu(gb.kind, fb)
        if not flags & 2:
            flops[i] += nvB[i] * _sdf_bwd_flops(ga.kind, fa, True)
            mufu[i] += nvB[i] * _sdf_bwd_mufu(ga.kind, fa)
        if not flags & 3:
            ee = neA[i] * neB[i]
            flops[i] += ee * (2 * SS_BWD[1] + EE_BWD[1] + _sdf_bwd_flops(ga.kind, fa, False) +
                              _sdf_bwd_flops(ga.kind, fa, True) + _sdf_bwd_flops(gb.kind, fb, False) +
                              _sdf_bwd_flops(gb.kind, fb, True))
            mufu[i] += ee * (2 * SS_BWD[0] + EE_BWD[0] + 2 * _sdf_bwd_mufu(ga.kind, fa) +
                             2 * _sdf_bwd_mufu(gb.kind, fb))
    return flops, mufu


# Peaks of the two arithmetic pipes from unit counts and the maximum SM clock, the
# denominators of the ALU roofline: SMs x 128 FP32 lanes x 2 flops (FFMA) x 2070 MHz
# (80.5 TFLOP/s on 152 SMs), and SMs x 32 ex2 results per clock x 2070 MHz (10.1 Top/s).
# The SM count is read from the device; the bench also measures an FFMA loop and an
# ex2.approx loop on the device and reports each fraction of those beside.
N_SMS, FP32_LANES_PER_SM, MUFU_EX2_PER_SM_CLK, SM_MAX_MHZ = 152, 128, 32, 2070


def alu_peaks(n_sms=N_SMS):
    return (n_sms * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6, n_sms * MUFU_EX2_PER_SM_CLK * SM_MAX_MHZ * 1e6)


FP32_PEAK_DERIVED, MUFU_PEAK_DERIVED = alu_peaks()
ALU_PEAKS = (FP32_PEAK_DERIVED, MUFU_PEAK_DERIVED)


def pipe_fracs(w, ms, peaks=ALU_PEAKS, flags=0, backward=False):
    """Useful-work fractions of the FP32 and MUFU peaks (default: from unit counts and
    clock) for one forward (or, with ``backward``, adjoint) launch over ``w`` taking ``ms``."""
    fma_peak, mufu_peak = peaks
    s = ms * 1e-3
    if backward:
        fl, mu = bwd_work_per_pair(w, flags)
    else:
        fl, mu = fp32_flops_per_pair(w, flags), mufu_ops_per_pair(w, flags)
    return {"fp32": float(fl.sum()) / s / fma_peak, "mufu": float(mu.sum()) / s / mufu_peak}


def alu_roofline(w, step_s, measured, backward=False, n_sms=N_SMS, traffic=None, kernel="cm_fwd_kernel"):
    """Roofline object of one launch of the forward (or adjoint) kernel over ``w`` taking
    ``step_s`` seconds: both pipes' achieved rates against the peaks from unit counts and
    clock, the larger fraction binding, with the fractions of the measured loop
    throughputs ``measured = (FFMA flop/s, ex2 op/s)`` beside them."""
    fma_meas, mufu_meas = measured
    fp32_peak, mufu_peak = alu_peaks(n_sms)
    if backward:
        fl, mu = bwd_work_per_pair(w)
    else:
        fl, mu = fp32_flops_per_pair(w), mufu_ops_per_pair(w)
    mufu = float(mu.sum()) / step_s
    flops = float(fl.sum()) / step_s
    pipes = {"mufu": {"achieved": mufu / 1e9, "peak": mufu_peak / 1e9, "unit": "Gop/s",
                      "frac": mufu / mufu_peak,
                      "peak_source": f"{n_sms} SMs x 32 ex2 per clock x 2070 MHz",
                      "peak_measured": mufu_meas / 1e9, "frac_of_measured": mufu / mufu_meas},
             "fp32": {"achieved": flops / 1e12, "peak": fp32_peak / 1e12, "unit": "TFLOP/s",
                      "frac": flops / fp32_peak,
                      "peak_source": f"{n_sms} SMs x 128 lanes x 2 flops x 2070 MHz",
                      "peak_measured": fma_meas / 1e12, "frac_of_measured": flops / fma_meas}}
    binding = max(pipes, key=lambda k: pipes[k]["frac"])
    return {"kernel": kernel, "bound": "alu", "pipe": binding, **pipes[binding],
            "traffic": traffic, "traffic_unit": "bytes per launch (ncu dram read + write)",
            "algorithmic_bytes": (348 + (56 + 24 + 256 if backward else 0)) * w.n_pairs,
            "work_per_launch": {"fp32_flops": float(fl.sum()), "mufu_ops": float(mu.sum())},
            "launch_ms": step_s * 1e3, "pipes": pipes}


def _hbm_peak():
    """Measured HBM copy bandwidth of this GPU pool (GB/s), else the stated fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return 6800.0


# ----------------------------------------------------------------- multi-rank helpers
def rank_seed(rank, cfg=4):
    """Seed of rank ``rank``'s replica of setting ``cfg``: every rank owns an independent
    batch (weak scaling)."""
    return synth.SEED_BASE + cfg + 1000 * rank


def headline_workload(rank=0, n=HEADLINE_PAIRS):
    """The headline batch of rank ``rank`` (its own seeded replica)."""
    return synth.config_mixed_pooled(n=n, seed=rank_seed(rank, 4))


def oracle_sample(w, frac=0.01, seed=synth.SEED_BASE + 99):
    """A seeded subsample of ``frac`` of the pairs of ``w`` (at least one), as a workload."""
    rng = np.random.default_rng(seed)
    n = max(1, int(round(frac * w.n_pairs)))
    return w.subset(np.sort(rng.choice(w.n_pairs, n, replace=False)))


def aggregate(total_ms, pairs_per_rank, steps, world, all_reduce_max):
    """Whole-job pairs/s: all ranks' pairs over the slowest rank's time."""
    ms = all_reduce_max(total_ms) if world > 1 else total_ms
    return world * pairs_per_rank * steps / (ms * 1e-3), ms


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in self.rows for j in range(4) if r[3 + j] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(self.rows)}


# ----------------------------------------------------------------- reference arm
def _oracle_pair(w, i, backward, g):
    import oracle
    if backward:
        oracle.batch_manifold_grad(w.geoms, w.pair_geoms, w.poses, w.dims, w.tau, g, idx=[i])
    else:
        oracle.batch_manifold(w.geoms, w.pair_geoms, w.poses, w.dims, w.tau, idx=[i])


def cpu_oracle_rate(w, budget_s=15.0, max_pairs=None, threads=None, backward=False):
    """Pairs/s of the FP64 oracle (as it stands: forward, or with ``backward`` forward and
    vector-Jacobian product) on the first pairs of ``w`` within ``budget_s``, on
    PyTorch's intra-op threads (``threads`` of them if given, else the default)."""
    import torch
    saved = torch.get_num_threads()
    if threads:
        torch.set_num_threads(int(threads))
    try:
        g = np.ones((1, 8, 8))
        done, t0 = 0, time.perf_counter()
        limit = w.n_pairs if max_pairs is None else min(max_pairs, w.n_pairs)
        while done < limit and time.perf_counter() - t0 < budget_s:
            _oracle_pair(w, done, backward, g)
            done += 1
        dt = time.perf_counter() - t0
        return done / dt, done, dt, torch.get_num_threads()
    finally:
        torch.set_num_threads(saved)


def _oracle_worker(job):
    """One process of the pair-parallel oracle timing: pairs r, r + P, r + 2P, ... of the
    workload until ``budget_s`` has passed."""
    w, r, procs, budget_s, backward = job
    import torch
    torch.set_num_threads(1)
    g = np.ones((1, 8, 8))
    done, t0 = 0, time.perf_counter()
    for i in range(r, w.n_pairs, procs):
        if time.perf_counter() - t0 >= budget_s:
            break
        _oracle_pair(w, i, backward, g)
        done += 1
    return done, time.perf_counter() - t0


def cpu_oracle_rate_over_pairs(w, budget_s=10.0, procs=None, timeout_s=180.0, backward=False):
    """Pairs/s of the FP64 oracle (as it stands) run over the pairs of ``w`` on all host
    cores: ``procs`` single-threaded processes (started with spawn, so safe after CUDA
    use), each on its own share of the pairs for ``budget_s``.  Returns (pairs/s, pairs,
    seconds, procs); the processes' start-up is outside the timed span."""
    import multiprocessing as mp
    if not procs:
        procs = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    procs = int(procs)
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map_async(_oracle_worker, [(w, r, procs, budget_s, backward) for r in range(procs)])
        out = res.get(timeout=timeout_s)
    pairs = sum(d for d, _ in out)
    span = max(t for _, t in out)
    return pairs / span, pairs, span, procs


def cpu_baseline_leg(w, cpu_seconds, pool_budget_s=10.0, backward=True, what="a seeded 1 % sample"):
    """The ``cpu_baseline`` object: the FP64 oracle (as it stands) on this host's cores over
    ``w`` (a bounded sample of the workload, ``what``), forward and backward.  The reported
    value is the oracle run over pairs, one single-threaded process per core; the same
    oracle on PyTorch's intra-op threads and on one thread stays beside it (and is the
    value if the process pool cannot run)."""
    mode = "forward + backward" if backward else "forward"
    r, n, dt, cores = cpu_oracle_rate(w, budget_s=cpu_seconds, backward=backward)
    cpu = {"value": r, "unit": "pairs/s", "cores": cores, "kind": "oracle",
           "sample": f"first {n} pairs of {what} of the workload ({mode}, {dt:.1f} s)"}
    r1, n1, dt1, _ = cpu_oracle_rate(w, budget_s=min(5.0, cpu_seconds / 3), threads=1, backward=backward)
    cpu["single_thread"] = {"value": r1, "unit": "pairs/s", "cores": 1,
                            "sample": f"first {n1} pairs of {what} ({mode}, {dt1:.1f} s)"}
    try:
        rp, npairs, dtp, procs = cpu_oracle_rate_over_pairs(w, budget_s=min(pool_budget_s, cpu_seconds),
                                                            backward=backward)
        cpu = {"value": rp, "unit": "pairs/s", "cores": procs, "kind": "oracle",
               "sample": f"{npairs} pairs of {what} of the workload ({mode}), every {procs}-th pair in each "
                         f"of {procs} single-threaded processes ({dtp:.1f} s)",
               "intra_op_threads": {k: cpu[k] for k in ("value", "unit", "cores", "sample")},
               "single_thread": cpu["single_thread"]}
    except Exception as e:  # this timing never costs the bench line
        cpu["over_pairs_error"] = f"{type(e).__name__}: {e}"
    return cpu


def run_reference(args, rank):
    """The oracle arm: the FP64 CPU oracle (forward and backward, as it stands) on a seeded
    1 % sample of the headline workload, run over pairs on every host core (one
    single-threaded process per core), each step a bounded pass over the sample."""
    if rank != 0:
        return
    w = oracle_sample(headline_workload())
    per_step_budget = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_oracle_rate_over_pairs(w, budget_s=per_step_budget / 4, backward=True)
    total_pairs, total_t = 0, 0.0
    for _ in range(args.steps):
        r, n, dt, cores = cpu_oracle_rate_over_pairs(w, budget_s=per_step_budget, backward=True)
        total_pairs += n
        total_t += dt
    value = total_pairs / total_t
    line = {"impl": "reference", "metric": "contact pairs/s (forward + backward manifold)", "value": value,
            "unit": "pairs/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                             "sample": f"{total_pairs} pairs of a seeded 1 % sample ({w.n_pairs} pairs) of the "
                                       f"workload, forward + backward, each step at most {per_step_budget:.1f} s of "
                                       f"{cores} single-threaded processes over the sample's pairs"},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- serving
def serve_benchmark(eng, api, seconds, seed=synth.SEED_BASE + 5, rate=2000.0):
    """Poisson trace of requests (`rate`/s, 1..8192 pairs log-uniform, forward or forward+backward
    50/50) over a pool of mixed pairs, once through the continuous-batching server and once
    through the plain path (one forward [+ adjoint] launch per request, in arrival order)."""
    import torch
    pool = synth.config_mixed(n=1024, seed=seed)
    ids = eng.add_geometries(pool.geoms)
    trace = synth.serving_trace(seed=seed, rate=rate, duration=seconds)
    rng = np.random.default_rng(seed)
    sizes = np.array([n for _, n, _ in trace])
    total = int(sizes.sum())
    idx = rng.integers(0, pool.n_pairs, total)
    P = lambda a, dt=torch.float32: torch.from_numpy(np.ascontiguousarray(a)).to(dt).pin_memory()  # noqa: E731
    pg_all, poses_all = P(ids[pool.pair_geoms[idx]], torch.int32), P(pool.poses[idx])
    dims_all, tau_all = P(pool.dims[idx]), P(pool.tau[idx])
    gout_all = P(rng.normal(size=(total, 8, 8)).astype(np.float32))
    out_all = torch.empty((total, 8, 8)).pin_memory()
    gp_all, gd_all = torch.empty((total, 14)).pin_memory(), torch.empty((total, 6)).pin_memory()
    offs = np.concatenate([[0], np.cumsum(sizes)])
    params = eng.params()

    def req(i):
        a, b = int(offs[i]), int(offs[i + 1])
        bwd = trace[i][2]
        return (pg_all[a:b], poses_all[a:b], out_all[a:b], dims_all[a:b], tau_all[a:b],
                gout_all[a:b] if bwd else None, gp_all[a:b] if bwd else None, gd_all[a:b] if bwd else None)

    # warm both paths (kernels, pools) on a few requests
    api.cm_server_start(eng.ctx, params, max_batch_pairs=65536, n_streams=4)
    for i in range(4):
        api.cm_wait(eng.ctx, api.cm_submit(eng.ctx, *req(i)), -1)
    t0 = time.perf_counter()
    tickets = []
    for i, (ta, n, bwd) in enumerate(trace):
        d = t0 + ta - time.perf_counter()
        if d > 0:
            time.sleep(d)
        tickets.append(api.cm_submit(eng.ctx, *req(i)))
    for t in tickets:
        api.cm_wait(eng.ctx, t, -1)
    t_end = time.perf_counter()
    lat = np.array([api.cm_request_latency(eng.ctx, t) for t in tickets])
    api.cm_server_stop(eng.ctx)
    served = {"p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
              "pairs_per_s": total / (t_end - t0), "requests": len(trace), "pairs": total,
              "trace_seconds": seconds}

    # plain path: one launch (two with the adjoint) per request, sequential
    dev = [torch.empty(t.shape, dtype=t.dtype, device="cuda") for t in (pg_all, poses_all, dims_all, tau_all)]
    dgo = torch.empty(gout_all.shape, device="cuda")
    lat_p = []
    t0 = time.perf_counter()
    for i, (ta, n, bwd) in enumerate(trace):
        d = t0 + ta - time.perf_counter()
        if d > 0:
            time.sleep(d)
        a, b = int(offs[i]), int(offs[i + 1])
        pg, poses, dims, tau = (x[a:b] for x in dev)
        for x, h in zip((pg, poses, dims, tau), (pg_all, poses_all, dims_all, tau_all)):
            x.copy_(h[a:b], non_blocking=True)
        out = eng.forward(pg, poses, dims, tau, params)
        out_all[a:b].copy_(out, non_blocking=True)
        if bwd:
            dgo[a:b].copy_(gout_all[a:b], non_blocking=True)
            gp, gd = eng.backward(pg, poses, dims, tau, dgo[a:b], params)
            gp_all[a:b].copy_(gp, non_blocking=True)
            gd_all[a:b].copy_(gd, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        lat_p.append(time.perf_counter() - (t0 + ta))
    t_end = time.perf_counter()
    lat_p = np.array(lat_p)
    plain = {"p50_ms": 1e3 * float(np.percentile(lat_p, 50)), "p99_ms": 1e3 * float(np.percentile(lat_p, 99)),
             "pairs_per_s": total / (t_end - t0)}
    return {"workload": f"Poisson {rate:g} req/s, 1..8192 pairs log-uniform of hull(8-256) vs primitive, "
                        "tau in {1e-3,1e-2,1e-1}, fwd or fwd+bwd 50/50", "served": served, "plain": plain}


# ----------------------------------------------------------------- extra settings
def plan_rate(eng, api, w, params, steps, with_bwd, flush, tune=True):
    """Pairs/s of graph-replayed steps (forward, or forward + adjoint) on workload ``w``."""
    import torch
    from paper_2602_20304_gb300.engine import workload_tensors
    ids = eng.add_geometries(w.geoms)
    pg, poses, dims, tau = workload_tensors(w, id_map=ids)
    out = torch.empty((w.n_pairs, params.K, 8), device="cuda")
    go = torch.randn_like(out) if with_bwd else None
    gp = torch.empty_like(poses) if with_bwd else None
    gd = torch.empty_like(dims) if with_bwd else None
    if tune:
        api.cm_autotune(eng.ctx, pg, poses, dims, tau, params, out, go, gp, gd)
    plan = api.cm_plan_create(eng.ctx, pg, poses, dims, tau, params, out, go, gp, gd)
    api.cm_plan_launch(plan)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ms = 0.0
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        api.cm_plan_launch(plan)
        b.record(stream)
        b.synchronize()
        ms += a.elapsed_time(b)
    api.cm_plan_destroy(plan)
    eng.check()
    return w.n_pairs * steps / (ms * 1e-3), ms / steps


def extra_settings(Engine, api, local, steps, flush, peaks, w4):
    """The 4096-pair hull-vs-primitive setting (forward and forward+backward), the paper's
    acceleration structure on the headline batch ``w4``, and the paper's two
    simplifications (vertex-SDF contacts only; one-sided) on the 4096-pair setting."""
    eng = Engine(local)
    try:
        params = eng.params()
        w2 = synth.config_hull_vs_primitive(n=4096, seed=rank_seed(0, 2))
        f2, f2_ms = plan_rate(eng, api, w2, params, steps, False, flush)
        fb2, fb2_ms = plan_rate(eng, api, w2, params, steps, True, flush)
        # the paper's acceleration structure: all vertices, the 16 deepest soft edges per body
        sel4, sel4_ms = plan_rate(eng, api, w4, eng.params(top_edges=16), steps, False, flush)
        # K = 4: the smallest hulls have fewer than 8 vertices for the one-sided mode
        full, _ = plan_rate(eng, api, w2, eng.params(K=4), steps, False, flush)
        ne, _ = plan_rate(eng, api, w2, eng.params(K=4, flags=1), steps, False, flush)
        nes, _ = plan_rate(eng, api, w2, eng.params(K=4, flags=2), steps, False, flush)
    finally:
        eng.close()
    return {"hull_vs_primitive_4096": {"workload": WORKLOAD_2, "fwd_pairs_per_s": f2, "fwd_ms": f2_ms,
                                       "fwd_bwd_pairs_per_s": fb2, "fwd_bwd_ms": fb2_ms,
                                       "fwd_pipe_fracs": pipe_fracs(w2, f2_ms, peaks),
                                       "bwd_pipe_fracs": pipe_fracs(w2, fb2_ms - f2_ms, peaks, backward=True)},
            "preselect_top_edges_16": {"workload": WORKLOAD + ", top_edges=16",
                                       "fwd_pairs_per_s": sel4, "fwd_ms": sel4_ms},
            "simplifications": {"workload": WORKLOAD_2.replace("K=8", "K=4"), "full_fwd_pairs_per_s": full,
                                "no_ee_fwd_pairs_per_s": ne, "one_sided_fwd_pairs_per_s": nes,
                                "speedup_no_ee": ne / full, "speedup_one_sided_vs_no_ee": nes / ne}}


def small_config_rates(Engine, api, local, steps, flush, peaks):
    """The two 1024-pair settings: box-box poses (batched launch, and the plain path of
    one launch per pose) and box vs the hull of 32 points on the sphere (forward and
    forward+backward)."""
    import torch
    from paper_2602_20304_gb300.engine import workload_tensors
    eng = Engine(local)
    try:
        res = {}
        w1 = synth.make_config(1)
        params = eng.params()
        r, ms = plan_rate(eng, api, w1, params, steps, False, flush)
        ids = eng.add_geometries(w1.geoms)
        pg, poses, dims, tau = workload_tensors(w1, id_map=ids)
        out = torch.empty((w1.n_pairs, params.K, 8), device="cuda")
        for i in range(8):   # warm the one-pair path
            eng.forward(pg[i:i + 1], poses[i:i + 1], dims[i:i + 1], tau[i:i + 1], params, out=out[i:i + 1])
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        a.record()
        for i in range(w1.n_pairs):
            eng.forward(pg[i:i + 1], poses[i:i + 1], dims[i:i + 1], tau[i:i + 1], params, out=out[i:i + 1])
        b.record()
        b.synchronize()
        plain = w1.n_pairs / (a.elapsed_time(b) * 1e-3)
        res["box_box_1024"] = {"workload": "two cubes h=0.5, 1024 poses, tau=1e-2, K=8", "fwd_pairs_per_s": r,
                               "fwd_ms": ms, "fwd_pipe_fracs": pipe_fracs(w1, ms, peaks),
                               "plain_one_launch_per_pose_pairs_per_s": plain}
        w3 = synth.make_config(3)
        f, fms = plan_rate(eng, api, w3, params, steps, False, flush)
        fb, fbms = plan_rate(eng, api, w3, params, steps, True, flush)
        res["box_vs_hull32_1024"] = {"workload": "box (dims U[0.2,1]) vs hull of 32 points on the unit sphere, "
                                                 "1024 pairs, tau=1e-2, K=8",
                                     "fwd_pairs_per_s": f, "fwd_ms": fms, "fwd_pipe_fracs": pipe_fracs(w3, fms, peaks),
                                     "fwd_bwd_pairs_per_s": fb, "fwd_bwd_ms": fbms}
    finally:
        eng.close()
    return res


def oracle_rates(seconds=4.0):
    """FP64 oracle pairs/s (as it stands, forward) on bounded samples of the other settings."""
    res = {}
    for name, w in (("box_box_1024", synth.make_config(1)), ("box_vs_hull32_1024", synth.make_config(3)),
                    ("hull_vs_primitive_4096", synth.make_config(2))):
        r, n, dt, cores = cpu_oracle_rate(w, budget_s=seconds)
        res[name] = {"pairs_per_s": r, "pairs": n, "seconds": dt, "cores": cores,
                     "sample": f"first {n} pairs of the workload (forward)"}
    return res


def sq_union_rates(Engine, api, local, steps, flush):
    """Pairs/s of the multi-superquadric bodies in the paper's armadillo setting (Sec. V:
    L superquadrics per body, every vertex, the L deepest soft edges per body), at the
    largest batch the paper vectorises (1024 pairs), with and without sphere tracing."""
    eng = Engine(local)
    try:
        res = {"workload": "1024 pairs of synthetic multi-superquadric bodies (pool of 8 per L), tau=1e-2, "
                           "K=8, all vertices, top_edges=L (one soft edge per superquadric)"}
        for L in (5, 18):
            w = synth.config_sq_union(n=1024, n_prims=L, seed=rank_seed(60 + L))
            res[f"L{L}"] = {"verts_mean": float(np.mean([g.n_verts for g in w.geoms])),
                            "edges_mean": float(np.mean([g.n_edges for g in w.geoms]))}
            r, ms = plan_rate(eng, api, w, eng.params(top_edges=L), steps, False, flush)
            res[f"L{L}"].update(fwd_pairs_per_s=r, fwd_ms=ms)
            r, ms = plan_rate(eng, api, w, eng.params(top_edges=L, trace_iters=3), steps, False, flush)
            res[f"L{L}"].update(trace3_fwd_pairs_per_s=r, trace3_fwd_ms=ms)
    finally:
        eng.close()
    return res


def witness_rates(api, n=10_000_000, steps=5):
    """Queries/s of the batched E-E and V-F witness routines, smoothed and non-smoothed
    (the paper's Ours-NS), queries uniform in the unit cube; the rows (48 B in, 32 / 16 B
    out) exceed L2, so each launch streams from HBM."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(synth.SEED_BASE + 6)
    q = torch.rand((n, 12), device="cuda", generator=g)
    res = {}
    soft, hard = api.cm_default_params(), api.cm_default_params(flags=api.CM_FLAG_HARD)
    for name, fn, width, p in (("ee", api.cm_ee_witness_batch, 8, soft), ("vf", api.cm_vf_witness_batch, 4, soft),
                               ("ee_hard", api.cm_ee_witness_batch, 8, hard),
                               ("vf_hard", api.cm_vf_witness_batch, 4, hard)):
        out = torch.empty((n, width), device="cuda")
        for _ in range(3):
            fn(q, p, out)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for _ in range(steps):
            fn(q, p, out)
        b.record()
        b.synchronize()
        s = a.elapsed_time(b) * 1e-3 / steps
        res[name] = {"queries_per_s": n / s, "ms": s * 1e3, "hbm_gbs": n * (48 + 4 * width) / s / 1e9}
    res["queries"] = n
    return res


# ----------------------------------------------------------------- our arm
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per pair of one forward and
# one adjoint launch of the current kernels on the 65536-pair headline batch, from one
# single-pass ncu capture of each (`--profile-case headline`, default launch shape):
# forward 0.523 + 3.018 GB, adjoint 8.119 + 13.788 GB per launch.
FWD_TRAFFIC_PER_PAIR = (0.522727e9 + 3.017795e9) / 65536
BWD_TRAFFIC_PER_PAIR = (8.119439e9 + 13.788441e9) / 65536


# Workloads of the ncu captures: the 4096-pair hull-vs-primitive setting (``--set full``
# fits its launches) and the 65536-pair headline batch (single-pass DRAM counters).
PROFILE_CASES = {"hull4096": lambda: synth.make_config(2), "headline": lambda: headline_workload(0)}


def profile_case(name, device, iters):
    """Forward with records, then the record-driven adjoint, ``iters`` times on the
    default launch shape (no autotuning, no graph) with a seeded upstream gradient: per
    iteration one cm_fwd_kernel and one cm_bwd_kernel launch (each after its work-order
    launch when the shape orders the batch)."""
    import torch
    from paper_2602_20304_gb300.engine import Engine, workload_tensors
    w = PROFILE_CASES[name]()
    eng = Engine(device)
    try:
        ids = eng.add_geometries(w.geoms)
        pg, poses, dims, tau = workload_tensors(w, id_map=ids)
        params = eng.params()
        g = torch.Generator(device="cuda").manual_seed(0)
        grad_out = torch.randn((w.n_pairs, params.K, 8), device="cuda", generator=g)
        for _ in range(iters):
            out, saved = eng.forward_save(pg, poses, dims, tau, params)
            gp, gd = eng.backward(pg, poses, dims, tau, grad_out, params, saved=saved)
        torch.cuda.synchronize()
        eng.check()
        ok = bool(torch.isfinite(out).all() and torch.isfinite(gp).all() and torch.isfinite(gd).all())
        print(json.dumps({"profile_case": name, "pairs": w.n_pairs, "iters": iters, "finite": ok}), flush=True)
        if not ok:
            raise SystemExit(1)
    finally:
        eng.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--pairs", type=int, default=HEADLINE_PAIRS, help="pairs per GPU (profiling uses fewer)")
    ap.add_argument("--no-autotune", action="store_true", help="default launch shapes (profiling)")
    ap.add_argument("--no-extra", action="store_true", help="skip the other settings")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="length of the Poisson serving trace at 2000 req/s (0 skips the serving comparison)")
    ap.add_argument("--serve-below-seconds", type=float, default=5.0,
                    help="length of the serving trace offered below capacity (400 req/s)")
    ap.add_argument("--profile-case", choices=list(PROFILE_CASES),
                    help="only run forward (with records) then adjoint, warmup + steps times, untimed: "
                         "the launches the ncu summaries capture")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist
    from paper_2602_20304_gb300 import api
    from paper_2602_20304_gb300.engine import Engine, workload_tensors

    torch.cuda.set_device(local)
    if args.profile_case:
        profile_case(args.profile_case, local, args.warmup + args.steps)
        return
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    # each rank owns an independent replica of the workload (weak scaling, no collective)
    w = headline_workload(rank, args.pairs)
    eng = Engine(local)
    ids = eng.add_geometries(w.geoms)
    pg, poses, dims, tau = workload_tensors(w, id_map=ids)
    params = eng.params()
    out = torch.empty((w.n_pairs, params.K, 8), device="cuda")
    grad_out = torch.randn(out.shape, device="cuda", generator=torch.Generator(device="cuda").manual_seed(rank))
    gp, gd = torch.empty_like(poses), torch.empty_like(dims)
    stream = torch.cuda.current_stream()
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 512 MB > L2

    # batching layer: autotuned launch shapes, then one CUDA-graph replay per step
    if not args.no_autotune:
        api.cm_autotune(eng.ctx, pg, poses, dims, tau, params, out, grad_out, gp, gd)
    shape_f = api.cm_get_launch_shape(eng.ctx, w.n_pairs, False)
    shape_b = api.cm_get_launch_shape(eng.ctx, w.n_pairs, True)
    plan_f = api.cm_plan_create(eng.ctx, pg, poses, dims, tau, params, out)
    plan_fb = api.cm_plan_create(eng.ctx, pg, poses, dims, tau, params, out, grad_out, gp, gd)
    launches_f = 1 + shape_f[2]                       # forward kernel (+ work-order kernel)
    launches_fb = launches_f + 1 + shape_b[2]         # + adjoint kernel (+ work-order kernel)

    for _ in range(max(3, args.warmup)):
        api.cm_plan_launch(plan_f)
        api.cm_plan_launch(plan_fb)
    torch.cuda.synchronize()
    eng.check()

    def timed(plan):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        barrier()
        torch.cuda.synchronize()
        for s in range(args.steps):
            flush.zero_()
            evs[s][0].record(stream)
            api.cm_plan_launch(plan)
            evs[s][1].record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = np.array([a.elapsed_time(b) for a, b in evs])
        return float(ms.sum()), ms

    def max_over_ranks(v):
        t = torch.tensor([v], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    with ClockSampler(local) as clk:
        total_fb_ms, step_fb_ms = timed(plan_fb)
        total_f_ms, step_f_ms = timed(plan_f)
    value, total_fb_ms = aggregate(total_fb_ms, w.n_pairs, args.steps, world, max_over_ranks)
    value_f, total_f_ms = aggregate(total_f_ms, w.n_pairs, args.steps, world, max_over_ranks)

    # ---- end to end through the public API: pinned host inputs (pairs, poses, dims, tau,
    # upstream gradient) -> the plan's buffers -> step -> host results (manifold, gradients)
    hin = [t.cpu().pin_memory() for t in (pg, poses, dims, tau, grad_out)]
    hout = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in (out, gp, gd)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e2e_ms = 0.0
    for s in range(args.steps):
        flush.zero_()
        e0.record(stream)
        for d, h in zip((pg, poses, dims, tau, grad_out), hin):
            d.copy_(h, non_blocking=True)
        api.cm_plan_launch(plan_fb)
        for h, d in zip(hout, (out, gp, gd)):
            h.copy_(d, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    barrier()
    e2e_value, e2e_ms = aggregate(e2e_ms, w.n_pairs, args.steps, world, max_over_ranks)
    e2e = {"value": e2e_value, "unit": "pairs/s",
           "h2d_bytes_per_step": int(sum(t.numel() * t.element_size() for t in hin)),
           "d2h_bytes_per_step": int(sum(t.numel() * t.element_size() for t in hout))}
    api.cm_plan_destroy(plan_f)
    api.cm_plan_destroy(plan_fb)
    eng.check()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- rooflines: algorithmic work per launch over the kernel's time.  The forward step
    # holds the work-order kernel and the forward kernel; the adjoint kernel's time is the
    # forward+backward step's less the forward step's (both timed above with CUDA events
    # on the launching stream; each difference also holds one few-microsecond ordering).
    fma_peak, mufu_peak = api.cm_measure_pipe_peaks(local)
    f_s = float(np.mean(step_f_ms)) * 1e-3
    b_s = float(np.mean(step_fb_ms) - np.mean(step_f_ms)) * 1e-3
    roof_b = alu_roofline(w, b_s, (fma_peak, mufu_peak), backward=True, n_sms=n_sms, kernel="cm_bwd_kernel",
                          traffic=None if BWD_TRAFFIC_PER_PAIR is None else BWD_TRAFFIC_PER_PAIR * w.n_pairs)
    roof_f = alu_roofline(w, f_s, (fma_peak, mufu_peak), n_sms=n_sms, kernel="cm_fwd_kernel",
                          traffic=None if FWD_TRAFFIC_PER_PAIR is None else FWD_TRAFFIC_PER_PAIR * w.n_pairs)

    extra = None
    if not args.no_extra and world == 1:
        extra = extra_settings(Engine, api, local, max(3, min(args.steps, 5)), flush, ALU_PEAKS, w)
        extra["witness_points"] = witness_rates(api)
        extra["sq_union"] = sq_union_rates(Engine, api, local, max(3, min(args.steps, 5)), flush)
        extra.update(small_config_rates(Engine, api, local, max(3, min(args.steps, 5)), flush, ALU_PEAKS))
        for k in ("ee", "vf"):
            extra["witness_points"][k]["hbm_frac_of_measured"] = extra["witness_points"][k]["hbm_gbs"] / _hbm_peak()

    serving = None
    if args.serve_seconds > 0 and world == 1:
        eng_s = Engine(local, hbm_budget_bytes=40 << 30)
        try:
            serving = serve_benchmark(eng_s, api, args.serve_seconds)
        finally:
            eng_s.close()
        # the same mix offered below the device's forward+backward capacity, where latency
        # is service time rather than queueing
        if args.serve_below_seconds > 0:
            eng_s = Engine(local, hbm_budget_bytes=40 << 30)
            try:
                serving["below_capacity"] = serve_benchmark(eng_s, api, args.serve_below_seconds, rate=400.0)
            finally:
                eng_s.close()

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline_leg(oracle_sample(w), args.cpu_seconds)
        if extra is not None:
            cpu["other_settings"] = oracle_rates()

    line = {"metric": "contact pairs/s (forward + backward manifold)", "value": value, "unit": "pairs/s",
            "fwd": {"value": value_f, "unit": "pairs/s", "ms_per_step": total_f_ms / args.steps,
                    "gpu_launches": launches_f * args.steps},
            "bwd_kernel_ms": b_s * 1e3,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_fb_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "pairs_per_gpu": w.n_pairs, "parallelism": f"replicas x{world}",
                       "l2": "flushed (512 MB write) between timed steps", "sms": n_sms},
            "gpu_launches": launches_fb * args.steps, "e2e": e2e, "roofline": roof_b, "roofline_fwd": roof_f,
            "serving": serving, "extra": extra,
            "launch_shape": {"fwd": {"block": shape_f[0], "ctas_per_sm": shape_f[1], "ordered": shape_f[2]},
                             "bwd": {"block": shape_b[0], "ctas_per_sm": shape_b[1], "ordered": shape_b[2]},
                             "cuda_graph": True}, "cpu_baseline": cpu,
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
