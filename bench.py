"""Throughput benchmark of the smooth contact-manifold library on GB300.

Workload (default): 4096 independent pairs, each the convex hull of 8..64 points
uniform in the unit ball against a random smooth primitive (box, capsule,
cylinder, ellipsoid; dims U[0.2, 1]), tau = 1e-2, penetration U[0, 0.1], K = 8,
FP32.  A step is one forward manifold over the whole batch (and, with
``--mode fwdbwd``, also the backward).  Inputs are resident in HBM; L2 is
flushed (512 MB write) between timed steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
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

WORKLOAD = "hull(8-64 pts) vs primitive, 4096 pairs, tau=1e-2, K=8"


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


# Peaks of the two arithmetic pipes from unit counts and the maximum SM clock, the
# denominators of the ALU roofline: 152 SMs x 128 FP32 lanes x 2 flops (FFMA) x 2070 MHz
# = 80.5 TFLOP/s, and 152 SMs x 32 ex2 results per clock x 2070 MHz = 10.1 Top/s.  The
# bench also measures an FFMA loop and an ex2.approx loop on the device and reports each
# fraction of those beside.
N_SMS, FP32_LANES_PER_SM, MUFU_EX2_PER_SM_CLK, SM_MAX_MHZ = 152, 128, 32, 2070
FP32_PEAK_DERIVED = N_SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6
MUFU_PEAK_DERIVED = N_SMS * MUFU_EX2_PER_SM_CLK * SM_MAX_MHZ * 1e6
ALU_PEAKS = (FP32_PEAK_DERIVED, MUFU_PEAK_DERIVED)


def pipe_fracs(w, ms, peaks=ALU_PEAKS, flags=0):
    """Useful-work fractions of the FP32 and MUFU peaks (default: from unit counts and
    clock) for one forward step of `w` taking `ms` milliseconds (the step also holds the
    work-order kernel)."""
    fma_peak, mufu_peak = peaks
    s = ms * 1e-3
    return {"fp32": float(fp32_flops_per_pair(w, flags).sum()) / s / fma_peak,
            "mufu": float(mufu_ops_per_pair(w, flags).sum()) / s / mufu_peak}


def alu_roofline(w, step_s, measured):
    """Roofline object of the forward kernel for one step of ``w`` taking ``step_s`` seconds:
    both pipes' achieved rates against the peaks from unit counts and clock, the larger
    fraction binding, with the fractions of the measured loop throughputs
    ``measured = (FFMA flop/s, ex2 op/s)`` beside them."""
    fma_meas, mufu_meas = measured
    mufu = float(mufu_ops_per_pair(w).sum()) / step_s
    flops = float(fp32_flops_per_pair(w).sum()) / step_s
    pipes = {"mufu": {"achieved": mufu / 1e9, "peak": MUFU_PEAK_DERIVED / 1e9, "unit": "Gop/s",
                      "frac": mufu / MUFU_PEAK_DERIVED,
                      "peak_source": "152 SMs x 32 ex2 per clock x 2070 MHz",
                      "peak_measured": mufu_meas / 1e9, "frac_of_measured": mufu / mufu_meas},
             "fp32": {"achieved": flops / 1e12, "peak": FP32_PEAK_DERIVED / 1e12, "unit": "TFLOP/s",
                      "frac": flops / FP32_PEAK_DERIVED,
                      "peak_source": "152 SMs x 128 lanes x 2 flops x 2070 MHz",
                      "peak_measured": fma_meas / 1e12, "frac_of_measured": flops / fma_meas}}
    binding = max(pipes, key=lambda k: pipes[k]["frac"])
    return {"bound": "alu", "pipe": binding, **pipes[binding],
            "traffic": FWD_TRAFFIC_BYTES_4096 * w.n_pairs / 4096 if FWD_TRAFFIC_CURRENT else None,
            "traffic_unit": "bytes per launch (ncu dram read + write)",
            "traffic_last_capture": {"value": FWD_TRAFFIC_BYTES_4096 * w.n_pairs / 4096,
                                     "note": "ncu capture taken before the destroyed-geometry check "
                                             "was added to pair setup"},
            "algorithmic_bytes": 348 * w.n_pairs, "pipes": pipes,
            "ncu_pipe_active_pct": FWD_NCU_PIPE_PCT}


# Pipe activity of the forward kernel on this workload (4096 pairs) from the same ncu
# capture: sm__pipe_fma_cycles_active and sm__inst_executed_pipe_xu, % of peak.
FWD_NCU_PIPE_PCT = {"fma": 39.9, "xu": 26.3}

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one forward-kernel launch
# on this workload at 4096 pairs, from one ncu capture; scaled by the pairs a launch
# processes (traffic grows in proportion).  The kernel has changed since that capture
# (pair setup now also rejects destroyed geometry, one branch on header fields it
# already reads), so the roofline's "traffic" is null and the figure is reported beside
# it as the last capture's.
FWD_TRAFFIC_BYTES_4096 = 5.426944e6 + 21.611264e6
FWD_TRAFFIC_CURRENT = False


def _hbm_peak():
    """Measured HBM copy bandwidth of this GPU pool (GB/s), else the stated fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return 6800.0


# ----------------------------------------------------------------- multi-rank helpers
def rank_seed(rank):
    """Seed of rank ``rank``'s replica: every rank owns an independent batch (weak scaling)."""
    return synth.SEED_BASE + 2 + 1000 * rank


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
def cpu_oracle_rate(w, budget_s=15.0, max_pairs=None, threads=None):
    """Pairs/s of the FP64 oracle (as it stands) on the first pairs of ``w`` within ``budget_s``,
    on PyTorch's intra-op threads (``threads`` of them if given, else the default)."""
    import torch
    import oracle
    saved = torch.get_num_threads()
    if threads:
        torch.set_num_threads(int(threads))
    try:
        done, t0 = 0, time.perf_counter()
        limit = w.n_pairs if max_pairs is None else min(max_pairs, w.n_pairs)
        while done < limit and time.perf_counter() - t0 < budget_s:
            oracle.batch_manifold(w.geoms, w.pair_geoms, w.poses, w.dims, w.tau, idx=[done])
            done += 1
        dt = time.perf_counter() - t0
        return done / dt, done, dt, torch.get_num_threads()
    finally:
        torch.set_num_threads(saved)


def _oracle_worker(job):
    """One process of the pair-parallel oracle timing: pairs r, r + P, r + 2P, ... of the
    workload (regenerated from its seeded recipe) until ``budget_s`` has passed."""
    cfg, n, r, procs, budget_s = job
    import torch
    torch.set_num_threads(1)
    import oracle
    w = synth.make_config(cfg, n)
    done, t0 = 0, time.perf_counter()
    for i in range(r, w.n_pairs, procs):
        if time.perf_counter() - t0 >= budget_s:
            break
        oracle.batch_manifold(w.geoms, w.pair_geoms, w.poses, w.dims, w.tau, idx=[i])
        done += 1
    return done, time.perf_counter() - t0


def cpu_oracle_rate_over_pairs(cfg, n, budget_s=10.0, procs=None, timeout_s=120.0):
    """Pairs/s of the FP64 oracle (as it stands) run over pairs on all host cores: ``procs``
    single-threaded processes (started with spawn, so safe after CUDA use), each on its
    own share of the pairs for ``budget_s``.  Returns (pairs/s, pairs, seconds, procs);
    the processes' start-up is outside the timed span."""
    import multiprocessing as mp
    if not procs:
        procs = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    procs = int(procs)
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map_async(_oracle_worker, [(cfg, n, r, procs, budget_s) for r in range(procs)])
        out = res.get(timeout=timeout_s)
    pairs = sum(d for d, _ in out)
    span = max(t for _, t in out)
    return pairs / span, pairs, span, procs


def cpu_baseline_leg(w, cfg, cpu_seconds, pool_budget_s=10.0):
    """The ``cpu_baseline`` object: the FP64 oracle (as it stands) on this host's cores over
    a bounded sample of workload ``w`` (the seeded setting ``cfg`` at ``w.n_pairs`` pairs).
    The reported value is the oracle run over pairs, one single-threaded process per core;
    the same oracle on PyTorch's intra-op threads and on one thread stays beside it (and
    is the value if the process pool cannot run)."""
    r, n, dt, cores = cpu_oracle_rate(w, budget_s=cpu_seconds)
    cpu = {"value": r, "unit": "pairs/s", "cores": cores, "kind": "oracle",
           "sample": f"first {n} pairs of the workload ({dt:.1f} s)"}
    r1, n1, dt1, _ = cpu_oracle_rate(w, budget_s=min(5.0, cpu_seconds / 3), threads=1)
    cpu["single_thread"] = {"value": r1, "unit": "pairs/s", "cores": 1,
                            "sample": f"first {n1} pairs of the workload ({dt1:.1f} s)"}
    try:
        rp, npairs, dtp, procs = cpu_oracle_rate_over_pairs(cfg, w.n_pairs, budget_s=min(pool_budget_s, cpu_seconds))
        cpu = {"value": rp, "unit": "pairs/s", "cores": procs, "kind": "oracle",
               "sample": f"{npairs} pairs of the workload, every {procs}-th pair in each of {procs} "
                         f"single-threaded processes ({dtp:.1f} s)",
               "intra_op_threads": {k: cpu[k] for k in ("value", "unit", "cores", "sample")},
               "single_thread": cpu["single_thread"]}
    except Exception as e:  # this timing never costs the bench line
        cpu["over_pairs_error"] = f"{type(e).__name__}: {e}"
    return cpu


def run_reference(args, rank):
    if rank != 0:
        return
    w = synth.make_config(2)
    steps = []
    per_step_budget = max(0.5, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_oracle_rate(w, budget_s=per_step_budget / 4)
    total_pairs, total_t = 0, 0.0
    for _ in range(args.steps):
        r, n, dt, cores = cpu_oracle_rate(w, budget_s=per_step_budget)
        steps.append(dt)
        total_pairs += n
        total_t += dt
    value = total_pairs / total_t
    line = {"impl": "reference", "metric": "contact pairs/s (forward manifold)", "value": value,
            "unit": "pairs/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                             "sample": f"{total_pairs} pairs of the workload, in order, "
                                       f"{per_step_budget:.1f} s per step"},
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


def extra_settings(Engine, api, local, steps, flush, peaks):
    """The uneven 65536-pair batch (forward and forward+backward) and the paper's two
    simplifications (vertex-SDF contacts only; one-sided) on the default workload."""
    eng = Engine(local)
    try:
        w4 = synth.config_mixed_pooled()
        params = eng.params()
        f4, f4_ms = plan_rate(eng, api, w4, params, steps, False, flush)
        fb4, fb4_ms = plan_rate(eng, api, w4, params, steps, True, flush)
        # the paper's acceleration structure: all vertices, the 16 deepest soft edges per body
        sel4, sel4_ms = plan_rate(eng, api, w4, eng.params(top_edges=16), steps, False, flush)
        w2 = synth.config_hull_vs_primitive(n=4096, seed=rank_seed(0))
        # K = 4: the smallest hulls have fewer than 8 vertices for the one-sided mode
        full, _ = plan_rate(eng, api, w2, eng.params(K=4), steps, False, flush)
        ne, _ = plan_rate(eng, api, w2, eng.params(K=4, flags=1), steps, False, flush)
        nes, _ = plan_rate(eng, api, w2, eng.params(K=4, flags=2), steps, False, flush)
    finally:
        eng.close()
    return {"uneven_65536": {"workload": "65536 pairs, hull(8-256 pts, pool of 4096) vs mixed primitives, "
                                         "tau in {1e-3,1e-2,1e-1}, one persistent launch per step, CUDA graph",
                             "fwd_pairs_per_s": f4, "fwd_ms": f4_ms, "fwd_bwd_pairs_per_s": fb4, "fwd_bwd_ms": fb4_ms,
                             "fwd_pipe_fracs": pipe_fracs(w4, f4_ms, peaks),
                             "preselect_top_edges_16_fwd_pairs_per_s": sel4, "preselect_fwd_ms": sel4_ms},
            "simplifications": {"workload": WORKLOAD.replace("K=8", "K=4"), "full_fwd_pairs_per_s": full,
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
    """FP64 oracle pairs/s (as it stands) on bounded samples of the other settings."""
    res = {}
    for name, w in (("box_box_1024", synth.make_config(1)), ("box_vs_hull32_1024", synth.make_config(3)),
                    ("uneven_65536", synth.config_mixed_pooled())):
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
    """Queries/s of the batched E-E and V-F witness routines, queries uniform in the unit
    cube; the rows (48 B in, 32 / 16 B out) exceed L2, so each launch streams from HBM."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(synth.SEED_BASE + 6)
    q = torch.rand((n, 12), device="cuda", generator=g)
    p = api.cm_default_params()
    res = {}
    for name, fn, width in (("ee", api.cm_ee_witness_batch, 8), ("vf", api.cm_vf_witness_batch, 4)):
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
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--pairs", type=int, default=4096, help="pairs per GPU (profiling uses fewer)")
    ap.add_argument("--no-autotune", action="store_true", help="default launch shapes (profiling)")
    ap.add_argument("--no-extra", action="store_true", help="skip the uneven-batch and simplification lines")
    ap.add_argument("--serve-seconds", type=float, default=0.5,
                    help="length of the Poisson serving trace (0 skips the serving comparison)")
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
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    # each rank owns an independent replica of the workload (weak scaling, no collective)
    w = synth.config_hull_vs_primitive(n=args.pairs, seed=rank_seed(rank))
    eng = Engine(local)
    ids = eng.add_geometries(w.geoms)
    pg, poses, dims, tau = workload_tensors(w, id_map=ids)
    params = eng.params()
    out = torch.empty((w.n_pairs, params.K, 8), device="cuda")
    grad_out = torch.randn_like(out)
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
    launches_fb = launches_f + 1 + shape_b[2]

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
        total_ms, step_ms = timed(plan_f)
        total_fb_ms, _ = timed(plan_fb)
    value, total_ms = aggregate(total_ms, w.n_pairs, args.steps, world, max_over_ranks)
    value_fb, total_fb_ms = aggregate(total_fb_ms, w.n_pairs, args.steps, world, max_over_ranks)

    # ---- end to end through the public API: pinned host inputs -> plan buffers -> host result
    hp = [t.cpu().pin_memory() for t in (pg, poses, dims, tau)]
    hout = torch.empty(out.shape, dtype=torch.float32).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e2e_ms = 0.0
    for s in range(args.steps):
        flush.zero_()
        e0.record(stream)
        for d, h in zip((pg, poses, dims, tau), hp):
            d.copy_(h, non_blocking=True)
        api.cm_plan_launch(plan_f)
        hout.copy_(out, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    barrier()
    e2e_value, e2e_ms = aggregate(e2e_ms, w.n_pairs, args.steps, world, max_over_ranks)
    h2d = sum(t.numel() * t.element_size() for t in hp)
    d2h = hout.numel() * hout.element_size()
    e2e = {"value": e2e_value, "unit": "pairs/s",
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
    api.cm_plan_destroy(plan_f)
    api.cm_plan_destroy(plan_fb)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- roofline of the forward kernel: algorithmic work per launch / step duration (the
    # step also holds the few-microsecond work-order kernel, so this slightly understates it).
    # Both arithmetic pipes are reported; the binding one is the larger fraction.
    fma_peak, mufu_peak = api.cm_measure_pipe_peaks(local)
    roof = alu_roofline(w, float(np.mean(step_ms)) * 1e-3, (fma_peak, mufu_peak))

    extra = None
    if not args.no_extra and world == 1:
        extra = extra_settings(Engine, api, local, max(3, min(args.steps, 5)), flush, ALU_PEAKS)
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
        # the same mix offered below the device's forward+backward capacity (~0.6 M pairs/s),
        # where latency is service time rather than queueing
        eng_s = Engine(local, hbm_budget_bytes=40 << 30)
        try:
            serving["below_capacity"] = serve_benchmark(eng_s, api, max(1.0, 2 * args.serve_seconds), rate=400.0)
        finally:
            eng_s.close()

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline_leg(w, 2, args.cpu_seconds)
        if extra is not None:
            cpu["other_settings"] = oracle_rates()

    line = {"metric": "contact pairs/s (forward manifold)", "value": value, "unit": "pairs/s",
            "fwd_bwd": {"value": value_fb, "unit": "pairs/s", "ms_per_step": total_fb_ms / args.steps,
                        "gpu_launches": launches_fb * args.steps},
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "pairs_per_gpu": w.n_pairs, "parallelism": f"replicas x{world}",
                       "l2": "flushed (512 MB write) between timed steps"},
            "gpu_launches": launches_f * args.steps, "e2e": e2e, "serving": serving, "extra": extra,
            "launch_shape": {"fwd": {"block": shape_f[0], "ctas_per_sm": shape_f[1], "ordered": shape_f[2]},
                             "bwd": {"block": shape_b[0], "ctas_per_sm": shape_b[1], "ordered": shape_b[2]},
                             "cuda_graph": True}, "roofline": roof, "cpu_baseline": cpu,
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
