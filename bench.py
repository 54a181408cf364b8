"""Benchmark: atom-steps/s of batched Frenkel-Ladd switching MD on one GB300.

Workload (default): the FP64-vs-mixed Frenkel-Ladd comparison -- ten seeds of
a bcc 10x10x10 cell (2000 atoms, a = 2.87 A) and ten of an fcc 8x8x8 cell
(2048 atoms, a = 3.65 A) at 1400 K, dt = 1 fs, damping 0.1 ps, t_eq = 10 ps,
t_s = 50 ps -- run as one batch of 20 replicas (40,480 atoms).  One "step" is
one MD step of every replica through the whole hot path (neighbour check,
pass 1, pass 2, fused blend/spring/work/BAOAB step).  Inputs are synthetic
(perfect lattices, Philox Maxwell-Boltzmann velocities).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--prec mixed|fp64] [--no-cpu-baseline]

Prints one JSON line.  --impl reference times the CPU FP64 oracle (the
baseline the library is checked against) on the host cores.  Under torchrun
(N > 1) every rank runs its own copy of the workload (replicas only: distinct
Philox replica indices, no data exchange); the time is the maximum over the
ranks and the value the whole job's atom-steps over that time.
"""
from __future__ import annotations

import argparse
import gc
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

from paper_2201_04622_gb300 import workloads as W  # noqa: E402

METRIC = "atom-steps/sec of switching MD (batched mixed vs plain FP64 GPU) at ≤1 meV/atom F error"
UNIT = "atom-steps/s"
T_K = 1400.0
K_SPRING = {W.BCC: W.K_BCC_1400, W.FCC: W.K_FCC_1400}  # eV/A^2, msd fits at 1400 K
SKIN = float(os.environ.get("NE_BENCH_SKIN", "2.6"))  # A
T_EQ, T_S = 10000, 50000
FP32_LANES_PER_SM = 128
# Algorithmic work of one atom-step of the mixed path (bcc at ~58 neighbours
# inside r_c + skin): ~2,700 FP32 lane instructions (pass 1 ~16 and pass 2
# ~30 per neighbour, plus the embedding and the integration), and ~200 bytes
# of state stream (x, v read and written, the site, the FP32 position copy):
# the figures the roofline is stated in.
ALG_LANE_OPS_PER_ATOM_STEP = 2700
ALG_BYTES_PER_ATOM_STEP = 200
FLOPS_PER_PAIR_PASS2 = 44    # FP32 lane operations per neighbour pair in pass 2 (multi-kernel path)
# crystal runner, lane operations (FP32 + INT32) the source issues, for the
# ratio of issued to algorithmic work:
OPS_VISIT = 26    # one lattice-stencil entry examined in pass 1, and its TMEM word tested in pass 2
OPS_PAIR = 54     # one pair inside r_c: splines of phi and f in pass 1, embedding force in pass 2
OPS_ATOM = 120    # per atom-step: F(rho), broadcasts, sums, Philox + Box-Muller, BAOAB


WORKLOADS = {
    "fl2": "fl_bcc10x10x10_fcc8x8x8_T1400K_10seeds_each_batched20",
    "batched256": "fl_256_uneven_replicas_bcc6-12_fcc5-10_T300-1600K",
    # reversible scaling of bcc 16^3 (8192 atoms), lambda 1 -> 1/16 from 100 K,
    # t_eq 10 ps, t_s 100 ps, four seeds in one batch (multi-kernel path)
    "rs16": "rs_bcc16x16x16_T0_100K_lambda_f_0.0625_4seeds_batched",
    # bcc 32^3 (65,536 atoms), 1 ps at lambda = 0 then a 20 ps FL switch at
    # 300 K, the backward pass (30,000 knot gradients) fused after every step
    "grad32": "fl_grad_bcc32x32x32_T300K_backward_every_step",
}
# schedule (t_eq, t_s), path, lambda_f and the runner of each workload
SCHEDULE = {"fl2": (T_EQ, T_S), "batched256": (T_EQ, 20000), "rs16": (10000, 100000), "grad32": (1000, 20000)}
ARGS = None


def workload():
    return ARGS.workload if ARGS is not None else "fl2"


def systems():
    """(lattice, n, a, seed, T) per replica of the workload."""
    out = []
    if workload() == "batched256":
        for r in W.batched_replicas(256, seed=1):
            a = W.A_BCC if r["lattice"] == W.BCC else W.A_FCC
            out.append((r["lattice"], r["n"], a, 1, r["T"]))
        return out
    if workload() == "rs16":
        return [(W.BCC, 16, W.A_BCC, 1 + s, 100.0) for s in range(4)]
    if workload() == "grad32":
        return [(W.BCC, 32, W.A_BCC, 1, 300.0)]
    for s in range(10):
        out.append((W.BCC, 10, W.A_BCC, 1 + s, T_K))
    for s in range(10):
        out.append((W.FCC, 8, W.A_FCC, 1 + s, T_K))
    return out


def build_batch(ne, np):
    x0s, offs, boxes, mds = [], [0], [], []
    mass = W.MASS_FE_AMU * 1.0364269656262175e-4
    t_eq, t_s = SCHEDULE[workload()]
    rs = workload() == "rs16"
    for r, (lat, n, a, seed, Tk) in enumerate(systems()):
        x0, box = ne.ne_create_crystal(lat, a, n, n, n)
        x0s.append(x0)
        offs.append(offs[-1] + len(x0))
        boxes.append(box)
        k = 4.0 if workload() == "grad32" else K_SPRING[lat]
        mds.append(ne.md_params(dt=1e-3, T=Tk, damp=0.1, mass=mass, k_spring=k,
                                skin=1.0 if workload() in ("rs16", "grad32") else SKIN,
                                lambda_fn=2, path=ne.NE_PATH_RS if rs else ne.NE_PATH_FL, lambda_f=0.0625,
                                t_eq=t_eq, t_s=t_s, seed=seed, replica=r, fix_cm=1))
    return np.concatenate(x0s), offs, boxes, mds


CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def clock_query():
    """One read-only nvidia-smi reading of this rank's GPU (a csv line or None)."""
    try:
        r = subprocess.run(["nvidia-smi", "--query-gpu=" + CLOCK_QUERY, "--format=csv,noheader,nounits",
                            "-i", str(os.environ.get("LOCAL_RANK", 0))],
                           capture_output=True, text=True, timeout=20)
        return r.stdout.strip().splitlines()[0] if r.returncode == 0 and r.stdout.strip() else None
    except (OSError, subprocess.TimeoutExpired):
        return None


class Clocks:
    """nvidia-smi samples (200 ms) during the timed region, plus one reading
    taken just before it starts and one just after it ends (a region of a
    few milliseconds sees no periodic sample)."""

    def __init__(self):
        self.proc = None
        self.lines = []
        self.edges = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + CLOCK_QUERY, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(os.environ.get("LOCAL_RANK", 0))],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def edge(self):
        ln = clock_query()
        if ln:
            self.edges.append(ln)

    def settle(self, timeout=5.0, quiet_s=0.05):
        """The reading before the timed region, taken once the periodic
        sampler is past its start-up (its first line is in): an nvidia-smi
        that is starting up or has just exited holds driver calls of this
        process back by tens of microseconds, so the region starts quiet_s
        after both."""
        t0 = time.time()
        while self.proc and not self.lines and time.time() - t0 < timeout:
            time.sleep(0.01)
        self.edge()
        time.sleep(quiet_s)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    @staticmethod
    def _parse(lines, reasons):
        sm, mx = [], []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return sm, mx

    def summary(self):
        """Median SM clock of the periodic samples, or of the two edge
        readings when the region was too short for any; throttle reasons
        seen in either."""
        reasons = set()
        sm_p, mx_p = self._parse(self.lines, reasons)
        sm_e, mx_e = self._parse(self.edges, reasons)
        sm = sm_p or sm_e
        mx = mx_p + mx_e
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm_p) + len(sm_e),
                "from": "periodic samples" if sm_p else ("readings just before and after the timed region"
                                                         if sm_e else None),
                "edge_sm_mhz": sm_e}


def measured_peak(key):
    """A peak from MEASURED_PEAKS.json at the repository root (None if absent)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key])
    except (OSError, KeyError, ValueError, TypeError):
        return None


def flush_l2(torch, buf):
    buf.add_(1.0)


def rank_replica_ids(n_rep, rank):
    """Philox replica indices of one rank's replicas: every rank runs its own
    copy of the workload, so the indices are shifted by n_rep per rank."""
    return [rank * n_rep + r for r in range(n_rep)]


def max_over_ranks(ms, dist, device):
    """The slowest rank's time (all_reduce MAX); the same value on every rank."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms):
    """Units per second of the whole job: all ranks' units over the slowest time."""
    return units_per_rank * world / (ms * 1e-3)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2201_04622_gb300 import ne

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ne.load()
    prec = ne.NE_MIXED if args.prec == "mixed" else ne.NE_FP64
    x0_np, offs, boxes, mds = build_batch(ne, np)
    for m, rid in zip(mds, rank_replica_ids(len(mds), rank)):
        m.prec = prec
        m.replica = rid
    n_rep, n_atoms = len(mds), int(offs[-1])
    ctx = ne.ne_ctx_create(ne.eam_params(**W.EAM_FE_LIKE), n_atoms, n_rep)
    ne.ne_ctx_set_tuning(ctx, args.tpa)
    x0 = torch.tensor(x0_np, dtype=torch.float64, device=dev)
    x = x0.clone()
    v = torch.zeros_like(x)
    for r, m in enumerate(mds):
        ne.ne_init_velocities(ctx, m, v[offs[r]:offs[r + 1]])
    Wd = torch.zeros((n_rep, 2), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    t_eq_w, t_s_w = SCHEDULE[args.workload]
    S_total = 2 * t_eq_w + 2 * t_s_w
    K, Wm = args.steps, args.warmup
    if Wm + K > S_total:
        raise SystemExit("warmup + steps exceeds the %d-step schedule" % S_total)
    l2 = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.float64, device=dev)  # > 129 MB L2
    path = args.path
    if path == "auto":
        # the crystal runners (cluster runner up to 4096 atoms a replica, brick
        # runner above) for the mixed crystal workloads; the gradient workload
        # needs the multi-kernel path's fused backward
        path = "crystal" if prec == ne.NE_MIXED and args.workload != "grad32" else "general"
    grad = args.workload == "grad32"
    if grad and path == "crystal":
        raise SystemExit("the gradient workload runs on the multi-kernel path")
    gth = torch.zeros(6 * W.EAM_FE_LIKE["n_knots"], dtype=torch.float64, device=dev) if grad else None
    crystals = [(lat, a, n, n, n) for (lat, n, a, seed, Tk) in systems()]

    # the crystal path runs through the library's BatchAdvancer: a replica that
    # leaves the crystal runner's range (a hop or melting at high T) continues
    # on the multi-kernel mixed path from its state before that chunk, next to
    # the crystal runner for the others; all of it inside the timed region
    adv = None
    if path == "crystal":
        from paper_2201_04622_gb300.workflow import BatchAdvancer
        adv = BatchAdvancer(ctx, mds, crystals, offs, boxes, x0,
                            chunk=5000 if args.workload == "batched256" else None)

    wts = {}

    def segment(xx, vv, x00, WW, s0, ns):
        if grad:
            # the backward after every step: weight 1 at each of the ns + 1
            # configurations of the segment (the gradient sums over them)
            if ns not in wts:
                wts[ns] = torch.ones(ns + 1, dtype=torch.float64, device=dev)
            ne.ne_switch_run_segment_grad(ctx, mds, offs, xx, vv, x00, boxes, WW, s0, ns, wts[ns], gth)
        elif path != "crystal":
            ne.ne_switch_run_segment(ctx, mds, offs, xx, vv, x00, boxes, WW, s0, ns)
        else:
            adv.advance(xx, vv, WW, s0, ns)
    if grad:
        segment(x.clone(), v.clone(), x0, Wd.clone(), 0, 2)  # weights and backward set-up, untimed

    tuned = None
    if path == "crystal" and not args.no_autotune and args.workload == "fl2":
        # CTAs per cluster, timed on the batch itself before the timed region
        from paper_2201_04622_gb300 import autotune
        best, table = autotune.tune_crystal(ctx, mds, crystals, x, v, Wd, 0, 200)
        tuned = {"best": best, "candidates": table,
                 "what": "crystal runner (cluster runner at 6-8 CTAs per cluster, or the brick runner)"}
    if path == "general" and args.autotune:
        from paper_2201_04622_gb300 import autotune
        best, table = autotune.tune(ctx, mds, offs, x, v, x0, boxes, Wd, 0, 60,
                                    skins=[1.0, 1.8, 2.6])
        tuned = {"best": {k: best[k] for k in ("tpa", "skin", "ms_per_step")}, "candidates": len(table)}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # torch creates an event at its first record (~20 us of host time): for e1
    # that would fall between the last kernel and the end stamp
    e0.record(stream)
    e1.record(stream)
    with Clocks() as clk:
        clk.settle()
        # warm-up steps (the start of the schedule) right before the timed
        # ones: after the host has idled, a single call carries ~50 us more
        # host latency than one that follows a call of the same path
        segment(x, v, x0, Wd, 0, Wm)
        x_w, v_w, W_w = x.clone(), v.clone(), Wd.clone()  # state after warm-up, for the e2e replay
        moved_w = list(adv.moved) if adv else []
        c0 = ne.ne_ctx_counters(ctx)
        n_log0 = len(adv.log) if adv else 0
        flush_l2(torch, l2)
        if world > 1:
            dist.barrier()
        gc.disable()  # no collection inside the timed call (as timeit does)
        torch.cuda.synchronize()
        e0.record(stream)
        segment(x, v, x0, Wd, Wm, K)
        e1.record(stream)
        torch.cuda.synchronize()
        gc.enable()
        clk.edge()
    ms = e0.elapsed_time(e1)
    # device time of the crystal runner's own launches in the timed call
    # (events the library records on the launching stream)
    kern_ms = ne.ne_ctx_last_run_ms(ctx) if path == "crystal" and not (adv and adv.moved) else None
    c1 = ne.ne_ctx_counters(ctx)
    timed_log = list(adv.log[n_log0:]) if adv else []
    moved_timed = list(adv.moved) if adv else []
    list_builds = c1[0] - c0[0]
    visits, pairs = c1[1] - c0[1], c1[2] - c0[2]
    if world > 1:
        ms = max_over_ranks(ms, dist, dev)
        dist.barrier()
    value = whole_job_rate(K * n_atoms, world, ms)

    # end to end: the same K steps again from the state after warm-up, through
    # the C ABI from pinned host buffers (copies in, K steps, state and work out)
    # x and v travel as one packed pinned buffer each way; the crystal runner
    # takes the sites from the crystal description, so x0 is an input of the
    # multi-kernel path only
    n3 = x_w.numel()
    sh = torch.cat([x_w.reshape(-1), v_w.reshape(-1)]).cpu().pin_memory()
    x0h = x0.cpu().pin_memory() if path != "crystal" else None
    Wh = W_w.cpu().pin_memory()
    del x_w, v_w, W_w
    K2 = K
    e2e = None
    if K2 > 0:
        # device buffers the copies land in, allocated before the timer starts
        sd = torch.empty_like(sh, device=dev)
        xd, vd = sd[:n3].view(-1, 3), sd[n3:].view(-1, 3)
        x0d = torch.empty_like(x0h, device=dev) if x0h is not None else x0
        Wd2 = torch.empty_like(Wh, device=dev)
        flush_l2(torch, l2)
        gc.disable()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sd.copy_(sh, non_blocking=True)
        if x0h is not None:
            x0d.copy_(x0h, non_blocking=True)
        Wd2.copy_(Wh, non_blocking=True)
        if adv:
            adv.moved = list(moved_w)
        segment(xd, vd, x0d, Wd2, Wm, K2)
        sh.copy_(sd, non_blocking=True)
        Wh.copy_(Wd2, non_blocking=True)
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        gc.enable()
        if world > 1:
            t_e2e = max_over_ranks(t_e2e * 1e3, dist, dev) * 1e-3
        h2d = (sh.numel() + (x0h.numel() if x0h is not None else 0) + Wh.numel()) * 8
        d2h = (sh.numel() + Wh.numel()) * 8
        e2e = {"value": whole_job_rate(K2 * n_atoms, world, t_e2e * 1e3), "unit": UNIT,
               "h2d_bytes_per_step": h2d / K2, "d2h_bytes_per_step": d2h / K2,
               "steps": K2, "note": "the timed K steps replayed through one ABI call from pinned host state: "
                                    "copies in, K steps, state and work out"}

    roof = None
    clk_sum = clk.summary()
    runner_kind, plan = None, None
    if path == "crystal":
        # the launch plan of the timed call (runner, threads per atom, CTAs)
        plan = ne.ne_ctx_crystal_plan(ctx)
        runner_kind = plan["runner"]
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    if path == "crystal" and kern_ms:
        # the timed call is one persistent launch per size class; its device
        # time is kern_ms.  Algorithmic work: 2,700 FP32 lane instructions and
        # 200 bytes per atom-step; peak lane rate = SMs x 128 FP32 lanes x the
        # median SM clock sampled around the timed region
        atom_steps = K * n_atoms
        sm_hz = (clk_sum["sm_mhz"] or clk_sum["sm_max_mhz"] or 2070.0) * 1e6
        peak = n_sm * FP32_LANES_PER_SM * sm_hz
        alg = ALG_LANE_OPS_PER_ATOM_STEP * atom_steps / (kern_ms * 1e-3)
        issued = (OPS_VISIT * visits + OPS_PAIR * pairs + OPS_ATOM * atom_steps) / (kern_ms * 1e-3)
        hbm_peak = measured_peak("hbm_gbs")
        hbm = ALG_BYTES_PER_ATOM_STEP * atom_steps / (kern_ms * 1e-3) / 1e9
        roof = {"bound": "alu", "kernel": "k_cluster (persistent cluster runner)" if runner_kind == "cluster"
                else "k_brick (persistent brick runner, grid barriers)",
                "achieved": alg / 1e12, "peak": peak / 1e12, "unit": "T lane-ops/s",
                "frac": alg / peak,
                # ncu DRAM read + write of one launch of this kernel on this
                # workload (k_cluster on fl2, a 200-step launch: 2.27 MB read, 0
                # written; k_brick on rs16, a 200-step launch: 1.86 MB read,
                # 0.07 MB written); the replicas live on chip or in L2, so the
                # figure does not grow with the steps; null elsewhere
                "traffic": (2.27e6 if args.workload == "fl2" and runner_kind == "cluster" else
                            1.91e6 if args.workload == "rs16" and runner_kind == "brick" else None),
                "kernel_ms": kern_ms, "us_per_step": kern_ms * 1e3 / K,
                "peak_note": "%d SMs x %d FP32 lanes x %.0f MHz (median SM clock sampled around the "
                             "timed region)" % (n_sm, FP32_LANES_PER_SM, sm_hz / 1e6),
                "algorithmic": "%d FP32 lane instructions per atom-step x %d atom-steps over the "
                               "launch's CUDA-event duration" % (ALG_LANE_OPS_PER_ATOM_STEP, atom_steps),
                "hbm": {"achieved_gbs": hbm, "peak_gbs": hbm_peak,
                        "frac": hbm / hbm_peak if hbm_peak else None,
                        "note": "%d B of state per atom-step; peak of measured copy bandwidth"
                                % ALG_BYTES_PER_ATOM_STEP},
                "issued": {"lane_ops_per_s": issued / 1e12, "ratio_to_algorithmic": issued / alg,
                           "note": "lane-ops the source issues: %d per stencil visit, %d per pair, %d per "
                                   "atom-step" % (OPS_VISIT, OPS_PAIR, OPS_ATOM)},
                "per_atom_step": {"stencil_visits": visits / atom_steps, "pairs": pairs / atom_steps}}
    # per-kernel durations (events around each launch) for the roofline
    xp, vp = x.clone(), v.clone()
    Wp = Wd.clone()
    n_prof = min(200, S_total - Wm - K) if S_total - Wm - K > 0 and path == "general" else 0
    prof = None
    if n_prof > 0:
        kms, cnt = ne.ne_profile_segment(ctx, mds, offs, xp, vp, x0, boxes, Wp, Wm + K, n_prof)
        prof = kms
    # multi-kernel path: the dominant kernel of ne_profile_segment's per-launch
    # times, against the algorithmic work of its pass: pass 1 ~16 and pass 2
    # ~30 FP32 lane instructions per neighbour inside r_c (58 in bcc, 54 in
    # fcc at these temperatures), the step kernel's ~164 B of state per atom
    if prof:
        pairs_per_atom = sum((58.0 if lat == W.BCC else 54.0) * ((2 if lat == W.BCC else 4) * n ** 3)
                             for (lat, n, a, seed, Tk) in systems()) / n_atoms
        peak = n_sm * FP32_LANES_PER_SM * (clk_sum["sm_mhz"] or clk_sum["sm_max_mhz"] or 2070.0) * 1e6
        per = {"nl_check": prof[0], "density": prof[1], "force": prof[2], "step": prof[3]}
        top = max(("density", "force", "step"), key=lambda q: per[q])
        if top == "step":
            hbm_peak = measured_peak("hbm_gbs")
            gbs = 164.0 * n_atoms / (per["step"] * 1e-3) / 1e9
            roof = {"bound": "hbm", "kernel": "k_step (fused blend, spring, work, BAOAB)", "achieved": gbs,
                    "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak if hbm_peak else None,
                    "traffic": None, "per_launch_ms": per}
        else:
            ops = (16.0 if top == "density" else 30.0) * pairs_per_atom * n_atoms
            ach = ops / (per[top] * 1e-3)
            roof = {"bound": "alu", "kernel": "k_density (pass 1)" if top == "density" else "k_force (pass 2)",
                    "achieved": ach / 1e12, "peak": peak / 1e12, "unit": "T lane-ops/s", "frac": ach / peak,
                    "traffic": None, "per_launch_ms": per,
                    "algorithmic": "%d FP32 lane instructions per pair inside r_c x %.1f pairs per atom"
                                   % (16 if top == "density" else 30, pairs_per_atom)}
        if grad:
            # the fused backward's own time per step: the timed step minus the
            # forward kernels (same launches without the backward)
            roof["backward_ms_per_step"] = ms / K - sum(per.values())
    steps_per_graph = 32
    general_launches = 6 * K + (K - 1) // steps_per_graph + 10  # list prep, bin, list, pass 1, pass 2, step
    if path == "crystal":
        launches = (c1[3] - c0[3]) + sum(6 * e[3] + e[3] // steps_per_graph + 10
                                         for e in timed_log if e[0] == "general")
    else:
        launches = general_launches + (2 * (K + 1) if grad else 0)  # backward: bins + reduction per step
    # the plain FP64 GPU path on the same batch (the comparison the metric names)
    fp64 = None
    if prec == ne.NE_MIXED and not args.no_fp64 and not grad:
        K64 = min(K, 2000, S_total - 1)
        m64 = [ne.md_params(dt=m.dt, T=m.T, damp=m.damp, mass=m.mass, k_spring=m.k_spring, skin=SKIN,
                            lambda_fn=m.lambda_fn, path=m.path, t_eq=m.t_eq, t_s=m.t_s, seed=m.seed,
                            replica=m.replica, fix_cm=m.fix_cm, prec=ne.NE_FP64) for m in mds]
        x64, v64 = x0.clone(), v.clone()
        W64 = torch.zeros_like(Wd)
        ne.ne_switch_run_segment(ctx, m64, offs, x64, v64, x0, boxes, W64, 0, 50)
        flush_l2(torch, l2)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        f1.record(stream)
        torch.cuda.synchronize()
        f0.record(stream)
        ne.ne_switch_run_segment(ctx, m64, offs, x64, v64, x0, boxes, W64, 50, K64)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1)
        if world > 1:
            ms64 = max_over_ranks(ms64, dist, dev)
        v64val = whole_job_rate(K64 * n_atoms, world, ms64)
        fp64 = {"value": v64val, "unit": UNIT, "ms_per_step": ms64 / K64, "steps": K64,
                "path": "multi-kernel, FP64 throughout", "speedup_of_mixed": value / v64val}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
           "warmup": Wm, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+f64" if prec == ne.NE_MIXED else "f64",
           "data": "synthetic (perfect bcc/fcc lattices, Philox Maxwell-Boltzmann velocities)",
           "config": {"workload": WORKLOADS[args.workload], "replicas": n_rep, "atoms": n_atoms,
                      "T_K": {"fl2": T_K, "batched256": "300-1600", "rs16": "100 -> 1600 (lambda 1 -> 0.0625)",
                              "grad32": 300.0}[args.workload],
                      "t_eq": t_eq_w, "t_s": t_s_w, "dt_fs": 1.0, "skin_A": mds[0].skin,
                      "precision": args.prec, "path": path, "runner": runner_kind,
                      "threads_per_atom": plan["threads_per_atom"] if plan else args.tpa,
                      "ctas": plan["ctas"] if plan else None,
                      "ctas_per_cluster": (plan["cluster_ctas"] or None) if plan else None,
                      "autotune": tuned,
                      "list_builds_per_replica_step": list_builds / (K * n_rep),
                      "moved_to_multikernel": {"replicas": moved_timed,
                                               "calls": [[e[1], e[2], e[3]] for e in timed_log
                                                         if e[0] == "general"]},
                      "parallelism": "replicas only" if world > 1 else "1 GPU",
                      "l2": "flushed before the timed segment; the 40k-atom state stays L2-resident "
                            "across MD steps by design"},
           "gpu_launches": launches, "clocks": clk_sum, "e2e": e2e, "roofline": roof,
           "fp64_gpu": fp64}
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_steps)
    ne.ne_ctx_destroy(ctx)
    if rank == 0:
        print(json.dumps(out))
    if adv:
        adv.close()
    if world > 1:
        dist.destroy_process_group()


def _oracle_replica(job):
    import oracle as O
    lat, n, a, seed, r, steps, Tk = job
    p = O.eam(**W.EAM_FE_LIKE)
    th = O.eam_theta(p)
    x0, box = O.create_crystal(lat, a, n, n, n)
    m = O.md(dt=1e-3, T=Tk, damp=0.1, mass=W.MASS_FE_AMU * O.amu(), k_spring=K_SPRING[lat],
             lambda_fn=2, path=O.PATH_FL, t_eq=0, t_s=max(1, steps // 2), seed=seed, replica=r,
             fix_cm=1)
    v = O.init_velocities(m, len(x0))
    t0 = time.perf_counter()
    O.switch_run(p, th, m, x0, v, x0, box)
    return len(x0) * 2 * max(1, steps // 2), time.perf_counter() - t0


def cpu_baseline(steps):
    """The FP64 oracle on the host cores: each of the 20 replicas of the
    workload runs `steps` switching steps, one replica per thread."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle as O
    O.lib()
    jobs = [(lat, n, a, seed, r, steps, Tk) for r, (lat, n, a, seed, Tk) in enumerate(systems())]
    cores = min(len(jobs), os.cpu_count() or 1)
    t0 = time.perf_counter()
    with ThreadPoolExecutor(cores) as ex:
        res = list(ex.map(_oracle_replica, jobs))
    wall = time.perf_counter() - t0
    total = sum(r[0] for r in res)
    return {"value": total / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d switching steps of each of the 20 replicas (%d atom-steps), FP64, "
                      "one replica per thread" % (2 * max(1, steps // 2), total)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # each reference step: one MD step of every replica of the workload by the
    # oracle (one replica per host thread); the run is a bounded sample of the
    # K requested steps
    n_atoms = sum((2 if lat == W.BCC else 4) * n ** 3 for (lat, n, a, seed, Tk) in systems())
    K = args.steps
    per_step_est = n_atoms / 2.0e6  # s, at ~2e6 atom-steps/s across the host cores
    k_run = max(2, min(K, int(90.0 / per_step_est)))
    w_run = max(1, min(args.warmup, 20))
    cpu_baseline(w_run)
    cb = cpu_baseline(k_run)
    out = {"metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": 0, "steps": k_run,
           "warmup": w_run, "ms_per_step": n_atoms / cb["value"] * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "impl": "reference",
           "data": "synthetic (perfect bcc/fcc lattices, Philox Maxwell-Boltzmann velocities)",
           "config": {"workload": WORKLOADS[args.workload], "replicas": len(systems()), "atoms": n_atoms},
           "cpu_baseline": cb,
           "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--tpa", type=int, default=4)
    ap.add_argument("--path", default="auto", choices=["auto", "crystal", "general"],
                    help="crystal: persistent cluster runner (mixed); general: multi-kernel path")
    ap.add_argument("--cpu-steps", type=int, default=80)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 GPU comparison")
    ap.add_argument("--autotune", action="store_true",
                    help="multi-kernel path: pick threads per atom and skin by timing the batch")
    ap.add_argument("--no-autotune", action="store_true",
                    help="crystal runner: keep the occupancy-based cluster size instead of timing 6-8 CTAs")
    ap.add_argument("--workload", default="fl2", choices=sorted(WORKLOADS),
                    help="fl2: FL switching of 20 crystals (crystal runner); batched256: 256 uneven replicas; "
                         "rs16: reversible scaling of bcc 16^3; grad32: bcc 32^3 with the backward every step")
    args = ap.parse_args()
    global ARGS
    ARGS = args
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
