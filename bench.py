"""Benchmark of the SiPO PDHG solve on GB300.

One step = one PDHG iteration of the restarted Halpern PDHG (projection with
fused primal update, backprojection with fused dual update, FP64 scalar step;
every check_every-th iteration also the KKT / restart evaluation).

Default workload: 256^3 voxels, 360 parallel-beam views over [0, pi), 256x256
detector, FP32 iterates, Case 2 (inhibition ratio 0.8), seeded CSG target in a
radius-120 vial (band width 10).  The working set (~1.5 GB) exceeds L2, so no
flush is needed between iterations.

`value` is PDHG iterations per second over all ranks with inputs resident in
HBM; `e2e` is the same through the C ABI with the target read from pinned host
memory and y* written back to pinned host memory, context creation included.
Extra keys: time to relative KKT 1e-4, the per-phase breakdown, the roofline
of the dominant kernel, the CPU oracle baseline, sampled SM clocks.

Multi-GPU (torchrun): every rank solves an independent replica (the LP does
not need an exchange across problems); value = total iterations / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PDHG iter/s and time-to-1e-4 KKT at 256³×360 views; projector GB/s vs HBM"
FP32_LANES_PER_SM = 128


def sm_count(device=None) -> int:
    """Streaming multiprocessors of the device (cudaDeviceProp.multiProcessorCount)."""
    import torch
    return int(torch.cuda.get_device_properties(device if device is not None else 0).multi_processor_count)


def sm_max_mhz(peaks: dict) -> float:
    """Maximum SM clock: the measured value, else the GB300 specification (2070 MHz)."""
    try:
        return float(peaks.get("sm_max_mhz", 2070.0))
    except (TypeError, ValueError):
        return 2070.0


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# two fused operator kernels, from one single-pass ncu capture of this
# workload.  It is reported only while the kernel sources (code, comments
# aside) still hash to the value they had at the capture; after any change to
# the code it is null until re-captured.
KERNEL_SOURCES = ["sipo_device.cuh", "sipo_solver.cuh", "sipo_ops.cuh", "sipo_launch.h",
                  "sipo_project.cu", "sipo_backproject.cu", "sipo_bp_tma.cuh"]
TRAFFIC = {("csg256", "f32"): {"sources_sha256_16": "b793cafb01817e69",
                               "project": 278965120, "backproject": 228099328}}


def _code_only(text: str) -> str:
    """Source text without comments and blank space (comments do not change a kernel)."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.strip() for line in text.splitlines() if line.strip())


def kernel_sources_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2604_08997_gb300", "csrc", f)) as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def captured_traffic(workload: str, storage: str, kernel: str):
    rec = TRAFFIC.get((workload, storage))
    if rec is None or rec["sources_sha256_16"] != kernel_sources_hash():
        return None
    return rec[kernel]


# ------------------------------------------------------------- distributed
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def init_dist(world, backend):
    if world <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend=backend)
    return dist


def max_over_ranks(x: float, dist, device=None) -> float:
    """Maximum of a per-rank float over all ranks (identity without a group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while active."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int = 0, period_ms: int = 200):
        self.index = index
        self.period_ms = period_ms
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", f"-lms={self.period_ms}"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- workload
def make_workload(name: str):
    from synthetic.targets import workload
    return workload(name)


def geometry_dict(wl):
    return dict(nx=wl.n, ny=wl.n, nz=wl.nz, angles=wl.angles, n_det=wl.n_det,
                vial_radius=wl.vial_radius, mu=wl.mu, psf_sigma=wl.psf_sigma,
                psf_trunc=wl.psf_trunc)


def case_dict(wl):
    return dict(kase=wl.case, w1=wl.w1, w2=wl.w2, tol_lo=wl.tol_lo, tol_hi=wl.tol_hi,
                inhibit_ratio=wl.inhibit_ratio, band_width=wl.band_width)


def workload_config(wl, storage_name):
    return {"workload": f"{wl.name}: {wl.n}x{wl.n}x{wl.nz} voxels, {wl.n_angles} views over [0,pi), "
                        f"{wl.n_det}x{wl.nz} detector, case {wl.case}, vial R={wl.vial_radius:g}, "
                        f"mu={wl.mu:g}, psf sigma={tuple(wl.psf_sigma)}",
            "n": wl.n, "n_angles": wl.n_angles, "storage": storage_name,
            "case": wl.case, "inhibit_ratio": wl.inhibit_ratio, "band_width": wl.band_width,
            "l2_policy": "working set > L2 (no flush)", "target": "seeded CSG (synthetic)"}


# ------------------------------------------------------------ CPU oracle
def _oracle_slab(args):
    """One oracle PDHG run on z-slices [z0, z0 + nz_sample) of the workload for
    `iters` iterations (no checks), after an untimed run of `warm` iterations
    when given; returns (setup seconds, solve seconds)."""
    name, case, delta, z0, nz_sample, iters = args[:6]
    warm = args[6] if len(args) > 6 else 0
    from oracle import pdhg
    from oracle.lp import CaseParams, build_lp
    from oracle.operators import Geometry
    wl = make_workload(name)
    _apply_case(wl, case, delta)
    tgt = np.ascontiguousarray(wl.target[:, :, z0:z0 + nz_sample])
    geo = Geometry(wl.n, wl.n, nz_sample, wl.angles, wl.n_det, vial_radius=wl.vial_radius,
                   mu=wl.mu, psf_sigma=wl.psf_sigma, psf_trunc=wl.psf_trunc)
    cp = CaseParams(case=wl.case, w1=wl.w1, w2=wl.w2, tol_lo=wl.tol_lo, tol_hi=wl.tol_hi,
                    inhibit_ratio=wl.inhibit_ratio, band_width=wl.band_width)
    t0 = time.perf_counter()
    lp, ops = build_lp(geo, tgt, cp)
    if warm > 0:
        pdhg.solve(lp, ops, kkt_tol=0.0, max_iter=warm, check_every=10 ** 9)
    t1 = time.perf_counter()
    pdhg.solve(lp, ops, kkt_tol=0.0, max_iter=iters, check_every=10 ** 9)
    return t1 - t0, time.perf_counter() - t1


def _apply_case(wl, case, delta):
    if case is not None:
        wl.case = case
        if case == 1:
            wl.tol_lo = wl.tol_hi = delta


def oracle_iteration_rate(wl, max_seconds: float = 20.0, nz_sample: int = 2, case=None, delta=0.05):
    """Oracle PDHG throughput on the host cores, extrapolated to the whole
    workload (the operator is slice-separable, so work scales with nz).

    Single thread: one process runs `nz_sample` middle z-slices, doubling the
    iteration count until about max_seconds / 2.  All cores: one spawned
    process per core, each on its own `nz_sample` slices for the same number
    of iterations, timed by the wall clock around the pool.  Returns
    (rate all cores, rate one thread, description, cores)."""
    import multiprocessing as mp
    nz_sample = min(nz_sample, wl.nz)
    z0 = wl.nz // 2 - nz_sample // 2
    iters = 2
    while True:
        setup, dt = _oracle_slab((wl.name, case, delta, z0, nz_sample, iters))
        if dt * 2 > max_seconds / 2 or iters >= 64:
            break
        iters *= 2
    single = 1.0 / (dt / iters * wl.nz / nz_sample)
    # slabs whose every slice holds part of the target, spread over the z range
    has = wl.target.reshape(-1, wl.nz).any(axis=0)
    cand = [z for z in range(wl.nz - nz_sample + 1) if has[z:z + nz_sample].all()]
    cores = max(1, min(os.cpu_count() or 1, len(cand)))
    rate, wall = single, dt
    if cores > 1:
        starts = [cand[(i * len(cand)) // cores] for i in range(cores)]
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores) as pool:
            t0 = time.perf_counter()
            out = pool.map(_oracle_slab, [(wl.name, case, delta, z, nz_sample, iters) for z in starts])
            wall = time.perf_counter() - t0
        solve = max(o[1] for o in out)
        # the pool's busiest process bounds the throughput of the cores
        rate = 1.0 / (solve / iters * wl.nz / (nz_sample * cores))
    desc = (f"oracle restarted Halpern PDHG (numpy/scipy FP64, explicit sparse P^T), {iters} iterations on "
            f"{nz_sample} of {wl.nz} z-slices per process, {cores} processes (one per host core, spawned) "
            f"and separately 1 process; per-iteration time scaled to nz = {wl.nz} (slice-separable); "
            f"single process {dt:.1f} s, pool wall {wall:.1f} s")
    return rate, single, desc, cores


REF_MAX_STEPS = 512


def oracle_steps_rate(wl, warmup: int, steps: int, nz_sample: int = 2, case=None, delta=0.05):
    """The reference arm: the oracle PDHG on the host cores, W untimed then K
    timed iterations in every process (one spawned process per core, each on
    its own `nz_sample` slices that hold part of the target); a step is one
    iteration of the whole volume, its time the busiest process's per-
    iteration time scaled to nz (slice-separable).  K is capped at
    REF_MAX_STEPS so that the run ends within minutes.  Returns (rate all
    cores, rate of one process in the pool, steps run, description, cores)."""
    import multiprocessing as mp
    nz_sample = min(nz_sample, wl.nz)
    steps = max(1, min(int(steps), REF_MAX_STEPS))
    has = wl.target.reshape(-1, wl.nz).any(axis=0)
    cand = [z for z in range(wl.nz - nz_sample + 1) if has[z:z + nz_sample].all()] or [0]
    cores = max(1, min(os.cpu_count() or 1, len(cand)))
    starts = [cand[(i * len(cand)) // cores] for i in range(cores)]
    jobs = [(wl.name, case, delta, z, nz_sample, steps, warmup) for z in starts]
    t0 = time.perf_counter()
    if cores > 1:
        with mp.get_context("spawn").Pool(cores) as pool:
            out = pool.map(_oracle_slab, jobs)
    else:
        out = [_oracle_slab(jobs[0])]
    wall = time.perf_counter() - t0
    solve = max(o[1] for o in out)
    rate = 1.0 / (solve / steps * wl.nz / (nz_sample * cores))
    single = 1.0 / (out[0][1] / steps * wl.nz / nz_sample)
    desc = (f"oracle restarted Halpern PDHG (numpy/scipy FP64, explicit sparse P^T): {warmup} untimed and "
            f"{steps} timed iterations on {nz_sample} of {wl.nz} z-slices per process, {cores} processes (one "
            f"per host core, spawned); step time = busiest process's iteration time scaled to nz = {wl.nz} "
            f"(slice-separable); pool wall {wall:.1f} s")
    return rate, single, steps, desc, cores


def cpu_baseline(wl, max_seconds=20.0, case=None, delta=0.05):
    rate, single, desc, cores = oracle_iteration_rate(wl, max_seconds, case=case, delta=delta)
    return {"value": rate, "unit": "iter/s", "cores": cores, "kind": "oracle", "sample": desc,
            "single_thread": {"value": single, "unit": "iter/s", "cores": 1}}


# ---------------------------------------------------------------- GPU arm
def needed_units(sipo, ctx, wl):
    """Columns the solver's kernels process: (y, x) columns with a band or gel
    voxel (backprojector) and (angle, bin) columns with an active ray (projector)."""
    lab = np.empty((wl.n, wl.n, wl.nz), np.uint8)
    act = np.empty((wl.n_angles, wl.n_det, wl.nz), np.uint8)
    sipo.sipo_get_array(ctx, 0, lab)
    sipo.sipo_get_array(ctx, 1, act)
    need = (lab != 0).any(axis=2)
    act_col = act.any(axis=2)
    return need, act_col


def tap_counts(wl, need, act_col):
    """Interpolation taps one launch of each fused kernel applies (per z value
    times nz): the backprojector's in-range taps of the needed columns, and the
    projector's non-zero taps from the needed columns into the active (angle,
    bin) columns.  Both kernels skip columns outside `need` (the input of the
    projector, the dual combination, is zero there), so neither count includes
    them."""
    n, nd = wl.n, wl.n_det
    c = np.arange(n) - (n - 1) / 2.0
    Y, X = np.meshgrid(c, c, indexing="ij")
    inside = np.ones((n, n), bool) if wl.vial_radius <= 0 else (X * X + Y * Y <= wl.vial_radius ** 2)
    bp_mask = need & inside
    xs_b, ys_b = X[bp_mask], Y[bp_mask]
    off = (nd - 1) / 2.0
    bp = fp = 0
    for k, th in enumerate(wl.angles):
        cth, sth = np.cos(th), np.sin(th)
        u = xs_b * cth + ys_b * sth + off
        i0 = np.floor(u)
        bp += int(np.count_nonzero((i0 >= 0) & (i0 < nd)) + np.count_nonzero((i0 + 1 >= 0) & (i0 + 1 < nd)))
        i0 = i0.astype(np.int64)
        w = u - i0
        hits = np.zeros(nd + 2, np.int64)
        ok = (i0 >= 0) & (i0 < nd)
        np.add.at(hits, i0[ok], 1)
        ok1 = (i0 + 1 >= 0) & (i0 + 1 < nd) & (w > 0)
        np.add.at(hits, i0[ok1] + 1, 1)
        fp += int(hits[:nd][act_col[k]].sum())
    return bp * wl.nz, fp * wl.nz


def deal_lps(work, world: int, rank: int) -> list[int]:
    """Indices of the independent LPs that `rank` solves: largest estimated
    work first, each to the rank with the least work so far (ties to the
    lower rank); the same on every rank, every LP to exactly one rank."""
    load = [0.0] * world
    owner = {}
    for i in sorted(range(len(work)), key=lambda i: (-work[i], i)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += work[i]
    return [i for i in range(len(work)) if owner[i] == rank]


def combine_sweep(elapsed: float, statuses: dict, iters: int, dist, device=None):
    """Whole-sweep figures from one rank's share: the slowest rank's seconds,
    the status counts and iteration totals summed over ranks."""
    names = ["optimal", "primal_infeasible", "dual_infeasible", "iteration_limit"]
    if dist is None:
        return float(elapsed), {k: v for k, v in statuses.items() if v}, int(iters)
    import torch
    t = torch.tensor([float(statuses.get(k, 0)) for k in names] + [float(iters)], dtype=torch.float64,
                     device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    counts = {k: int(v) for k, v in zip(names, t[:-1].tolist()) if v}
    return max_over_ranks(elapsed, dist, device), counts, int(t[-1].item())


def run_sweep(args, device, dist=None, rank=0, world=1):
    """The batched sweep (32 independent LPs, 64^3-192^3, 180-720 views, Case-1
    tolerances and Case-2 ratios): one sipo_solve_batched call to relative KKT
    1e-4 (or a certificate, or the iteration cap), timed on the host around the
    call with the device synchronised; per-LP sizes, statuses and iterations.
    With several ranks the LPs are dealt out whole (deal_lps) and each rank
    solves its share as one batch; nothing is exchanged but the timing and
    the status counts (the slowest rank's time is the sweep's)."""
    import torch
    import paper_2604_08997_gb300 as sipo
    from synthetic.targets import sweep_workloads
    sipo.build()
    storage = {"f32": sipo.SIPO_F32, "bf16": sipo.SIPO_BF16, "f64": sipo.SIPO_F64}[args.storage]
    wls_all = sweep_workloads()
    mine = deal_lps([w.n ** 3 * w.n_angles for w in wls_all], world, rank)
    wls = [wls_all[i] for i in mine]
    t0 = time.perf_counter()
    ctxs = []
    for wl in wls:
        tol = dict(storage=storage, kkt_tol=1e-4, max_iter=args.kkt_iters, check_every=args.check_every)
        ctxs.append(sipo.sipo_create(geometry_dict(wl), torch.from_numpy(wl.target).to(device), case_dict(wl), tol))
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0
    n0 = sipo.sipo_kernel_launch_count()
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clocks:
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = sipo.sipo_solve_batched(ctxs)
        torch.cuda.synchronize()
        elapsed = time.perf_counter() - t0
        if dist is not None:
            dist.barrier()
    launches = sipo.sipo_kernel_launch_count() - n0
    sequential = None
    if args.sweep_sequential:
        # the same LPs solved one after another (one graph per context), for
        # the batched form's comparison with the plain form
        for c in ctxs:
            sipo.sipo_destroy(c)
        ctxs = []
        for wl in wls:
            tol = dict(storage=storage, kkt_tol=1e-4, max_iter=args.kkt_iters, check_every=args.check_every)
            ctxs.append(sipo.sipo_create(geometry_dict(wl), torch.from_numpy(wl.target).to(device),
                                         case_dict(wl), tol))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        seq = [sipo.sipo_solve(c) for c in ctxs]
        torch.cuda.synchronize()
        seq_s = time.perf_counter() - t0
        same = sum(1 for a, b in zip(res, seq) if a["status"] == b["status"] and a["iters"] == b["iters"])
        sequential = {"seconds": seq_s, "same_status_and_iterations": same, "of": len(seq)}
    per_lp = [{"n": wl.n, "n_angles": wl.n_angles, "case": wl.case,
               "param": wl.tol_lo if wl.case == 1 else wl.inhibit_ratio,
               "status": r["status_name"], "iters": r["iters"], "kkt": r["kkt"], "objective": r["pobj"]}
              for wl, r in zip(wls, res)]
    for c in ctxs:
        sipo.sipo_destroy(c)
    statuses = {}
    for p in per_lp:
        statuses[p["status"]] = statuses.get(p["status"], 0) + 1
    local_iters = sum(p["iters"] for p in per_lp)
    t_max, statuses, total_iters = combine_sweep(elapsed, statuses, local_iters, dist, device)
    return {"metric": "batched sweep: seconds until every LP of the sweep has a status (KKT 1e-4, "
                      "infeasibility certificate or iteration cap)",
            "value": t_max, "unit": "s", "n_gpus": world, "steps": total_iters, "warmup": 0,
            "ms_per_step": t_max * 1e3 / max(1, total_iters), "higher_is_better": False,
            "scaling": "strong", "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
            "config": {"workload": f"sweep: {len(wls_all)} LPs, {min(w.n for w in wls_all)}^3-"
                                   f"{max(w.n for w in wls_all)}^3 voxels, {min(w.n_angles for w in wls_all)}-"
                                   f"{max(w.n_angles for w in wls_all)} views, Case 1 delta 0.02-0.20 and Case 2 "
                                   f"r 0.60-0.90, one batch per GPU",
                       "iteration_cap": args.kkt_iters, "storage": args.storage,
                       "parallelism": f"LPs dealt out whole over {world} GPU(s)"},
            "gpu_launches": int(launches), "create_seconds": t_create, "statuses": statuses,
            "iterations_per_second": total_iters / t_max, "sequential": sequential,
            "per_lp_rank0": per_lp, "clocks": clocks.summary()}


def run_gpu(args, dist, rank, world, device):
    import torch
    import paper_2604_08997_gb300 as sipo
    sipo.build()
    storage = {"f32": sipo.SIPO_F32, "bf16": sipo.SIPO_BF16, "f64": sipo.SIPO_F64}[args.storage]
    wl = make_workload(args.workload)
    _apply_case(wl, args.case, args.delta)
    geo, cp = geometry_dict(wl), case_dict(wl)
    tgt = torch.from_numpy(wl.target).to(device)
    tol = dict(storage=storage, kkt_tol=0.0, max_iter=args.warmup, check_every=args.check_every,
               tile_cfg=args.bp_tile)
    ctx = sipo.sipo_create(geo, tgt, cp, tol)
    sipo.sipo_solve(ctx)                      # W warm-up iterations (graph captured here)
    sipo.sipo_set_tolerances(ctx, 0.0, args.steps, args.check_every)
    torch.cuda.synchronize()
    n0 = sipo.sipo_kernel_launch_count()
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clocks:
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = sipo.sipo_solve(ctx)            # exactly K iterations (kkt_tol = 0)
        torch.cuda.synchronize()
        elapsed = time.perf_counter() - t0
        if dist is not None:
            dist.barrier()
    launches = sipo.sipo_kernel_launch_count() - n0
    t_max = max_over_ranks(elapsed, dist, device)
    iters_total = res["iters"] * world
    value = iters_total / t_max
    # per-phase breakdown with CUDA events on the solver stream
    phases = sipo.sipo_profile(ctx, args.profile_iters)
    normal = sum(v for k, v in phases.items() if k != "check_step")
    per_iter_ms = (normal * (args.check_every - 1) + phases["check_step"]) / args.check_every
    # roofline of the dominant kernel (work counted in taps: one FMA each)
    need, act_col = needed_units(sipo, ctx, wl)
    need_cols, act_cols = int(need.sum()), int(act_col.sum())
    bp_taps, fp_taps = tap_counts(wl, need, act_col)
    bp_ms = phases["backproject"]
    fp_ms = phases["project_primal"]
    tr_bp = captured_traffic(args.workload, args.storage, "backproject")
    tr_fp = captured_traffic(args.workload, args.storage, "project")
    bp_name = {0: "k_backproject", 1: "k_backproject", 2: "k_backproject", 3: "k_backproject2",
               4: "k_backproject2"}.get(res["tile_cfg"], "k_backproject3")
    fp_name = "k_project"
    if bp_ms >= fp_ms:
        dom, dom_ms, taps, traffic = f"{bp_name} (fused dual update)", bp_ms, bp_taps, tr_bp
    else:
        dom, dom_ms, taps, traffic = f"{fp_name} (fused primal update)", fp_ms, fp_taps, tr_fp
    # algorithmic HBM bytes: every input element once, every output once
    el = 2 if args.storage == "bf16" else (8 if args.storage == "f64" else 4)
    cw = 8 if args.storage == "f64" else 4
    S = wl.n_angles * wl.n_det * wl.nz
    bytes_bp = S * el + need_cols * wl.nz * (4 * el + 2 * cw + 1 + 2 * el + cw + el)
    bytes_fp = wl.n * wl.n * wl.nz * el + act_cols * wl.nz * (cw + 2 * el + 2 * el)
    clk = clocks.summary()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    n_sm, mhz = sm_count(device), sm_max_mhz(peaks)
    peak_tflops = n_sm * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    achieved = 2.0 * taps / (dom_ms * 1e-3) / 1e12
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak_tflops,
                "unit": "TFLOP/s", "frac": achieved / peak_tflops, "traffic": traffic,
                "traffic_unit": "bytes per launch (ncu dram read + write)",
                "peak_source": f"derived: {n_sm} SMs (cudaDeviceProp) x {FP32_LANES_PER_SM} FP32 lanes x "
                               f"2 FLOP x {mhz:.0f} MHz (no measured FP32 peak exists)",
                "units": "taps (one FMA = 2 FLOP per tap per z value)", "units_per_launch": taps,
                "avg_launch_ms": dom_ms,
                "l1_roof_frac": (taps / (dom_ms * 1e-3)) / (n_sm * 32 * mhz * 1e6),
                "backproject": {"ms": bp_ms, "taps": bp_taps,
                                "tflops": 2.0 * bp_taps / (bp_ms * 1e-3) / 1e12,
                                "alg_bytes": bytes_bp, "gbs": bytes_bp / (bp_ms * 1e-3) / 1e9,
                                "traffic": tr_bp,
                                "hbm_frac_of_measured": bytes_bp / (bp_ms * 1e-3) / 1e9 / hbm},
                "project": {"ms": fp_ms, "taps": fp_taps,
                            "tflops": 2.0 * fp_taps / (fp_ms * 1e-3) / 1e12,
                            "alg_bytes": bytes_fp, "gbs": bytes_fp / (fp_ms * 1e-3) / 1e9,
                            "traffic": tr_fp,
                            "hbm_frac_of_measured": bytes_fp / (fp_ms * 1e-3) / 1e9 / hbm},
                "hbm_peak_gbs": hbm}
    # time to relative KKT 1e-4: the requested instance, and the strictest
    # inhibition ratio of the sweep grid above it that converges (the requested
    # Case-2 instance may be infeasible, in which case its status is reported)
    kkt_info = None
    if args.kkt_iters > 0:
        kkt_info = {}
        runs = [("requested_plain_case2" if wl.case == 2 else "requested", cp)]
        if wl.case == 2 and args.feasible_ratio > 0:
            runs.append(("feasible_ratio_%.2f" % args.feasible_ratio,
                         dict(cp, inhibit_ratio=args.feasible_ratio)))
        for label, cpk in runs:
            ctx_k = ctx if cpk is cp else sipo.sipo_create(geo, tgt, cpk, tol)
            sipo.sipo_set_tolerances(ctx_k, 1e-4, args.kkt_iters, args.check_every)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rk = sipo.sipo_solve(ctx_k)
            torch.cuda.synchronize()
            tk = time.perf_counter() - t0
            kkt_info[label] = {"inhibit_ratio": cpk.get("inhibit_ratio"), "seconds": tk,
                               "iters": rk["iters"], "status": rk["status_name"], "kkt": rk["kkt"],
                               "rel_primal": rk["rel_primal"], "rel_dual": rk["rel_dual"],
                               "rel_gap": rk["rel_gap"], "objective": rk["pobj"],
                               "restarts": rk["restarts"], "dtvr_f": rk["dtvr_f"], "psr_f": rk["psr_f"],
                               "alpha": rk["alpha"]}
            if ctx_k is not ctx:
                sipo.sipo_destroy(ctx_k)
        if wl.case == 2:
            # Case 2 with its feasibility settled: the separation LP (Case 1
            # of the part, tol_lo = 0) gives the best band-to-gel ratio and
            # its dual is probed as a Farkas ray of Case 2 during the solve;
            # the concurrent form solves Case 2 beside it on its own stream,
            # the sequential one starts Case 2 after it
            sep_runs = [("requested", cp, True)]
            if args.feasible_ratio > 0:
                sep_runs.append(("separation_feasible_ratio_%.2f" % args.feasible_ratio,
                                 dict(cp, inhibit_ratio=args.feasible_ratio), True))
            if args.separation_sequential:
                sep_runs += [(lab + "_sequential", c, False) for lab, c, _ in list(sep_runs)]
            for label, cpk, race in sep_runs:
                tol_k = dict(tol, kkt_tol=1e-4, max_iter=args.kkt_iters)
                # the separation LP runs in FP32 storage (BF16 iterates stall
                # above the accuracy its certificate needs)
                tol_s = dict(tol, kkt_tol=1e-4, max_iter=args.separation_iters,
                             storage=sipo.SIPO_F64 if tol["storage"] == sipo.SIPO_F64 else sipo.SIPO_F32,
                             primal_weight=args.separation_omega)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ws = sipo.case2_with_separation(geo, tgt, cpk["inhibit_ratio"], band_width=cpk["band_width"],
                                                tolerances=tol_k, separation_tolerances=tol_s,
                                                probe_every=args.probe_every, race=race)
                torch.cuda.synchronize()
                tk = time.perf_counter() - t0
                sep, c2 = ws["separation"], ws["case2"]
                status = {sipo.SIPO_OPTIMAL: "optimal", sipo.SIPO_PRIMAL_INFEASIBLE: "primal_infeasible",
                          sipo.SIPO_ITER_LIMIT: "iteration_limit"}.get(ws["status"], str(ws["status"]))
                kkt_info[label] = {
                    "inhibit_ratio": cpk["inhibit_ratio"], "seconds": tk, "status": status,
                    "certified": ws["certified"], "cert_slice": ws["cert_slice"],
                    "ratio_bound": ws["ratio_bound"], "separation_status": sep["status_name"],
                    "separation_iters": sep["iters"], "separation_kkt": sep["kkt"],
                    "separation_dobj": sep["dobj"], "form": "concurrent" if race else "sequential",
                    "case2_iters": c2["iters"] if c2 else 0, "case2_kkt": c2["kkt"] if c2 else None,
                    "objective": c2["pobj"] if c2 else None,
                    "separation_form": "Case 1 with tol_lo = 0, tol_hi = 10 (minimum band dose over gel dose >= target)",
                    "includes": ("context creation of the separation LP and two Case-2 contexts (probe target, "
                                 "solve), separation solve with Farkas probes and Case-2 solve on two streams at "
                                 "once" if race else
                                 "context creation of both LPs, separation solve with Farkas probes, Case-2 solve")}
        if args.escalate > 0:
            # precision escalation: BF16 storage for at most N iterations, then
            # FP32 warm-started from its last check (both contexts created first)
            for label, cpk in runs:
                lo = sipo.sipo_create(geo, tgt, cpk, dict(tol, storage=sipo.SIPO_BF16, kkt_tol=1e-4,
                                                          max_iter=args.escalate))
                hi = sipo.sipo_create(geo, tgt, cpk, dict(tol, storage=sipo.SIPO_F32, kkt_tol=1e-4,
                                                          max_iter=args.kkt_iters))
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rl = sipo.sipo_solve(lo)
                if rl["status"] != sipo.SIPO_OPTIMAL and rl["status"] != sipo.SIPO_PRIMAL_INFEASIBLE:
                    sipo.sipo_warm_start(hi, lo)
                    rh = sipo.sipo_solve(hi)
                else:
                    rh = rl
                torch.cuda.synchronize()
                tk = time.perf_counter() - t0
                kkt_info["bf16_%d_then_f32_%s" % (args.escalate, label)] = {
                    "inhibit_ratio": cpk.get("inhibit_ratio"), "seconds": tk,
                    "iters_bf16": rl["iters"], "kkt_bf16": rl["kkt"],
                    "iters_f32": rh["iters"] if rh is not rl else 0, "status": rh["status_name"],
                    "kkt": rh["kkt"], "objective": rh["pobj"]}
                sipo.sipo_destroy(lo)
                sipo.sipo_destroy(hi)
    # end to end through the C ABI from pinned host memory
    tgt_h = torch.from_numpy(wl.target).pin_memory()
    y_h = torch.empty((wl.n_angles, wl.n_det, wl.nz), dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx_e = sipo.sipo_create(geo, tgt_h, cp, dict(tol, max_iter=args.steps))
    re = sipo.sipo_solve(ctx_e, y_h)
    sipo.sipo_destroy(ctx_e)
    torch.cuda.synchronize()
    te = time.perf_counter() - t0
    te_max = max_over_ranks(te, dist, device)
    e2e = {"value": re["iters"] * world / te_max, "unit": "iter/s",
           "h2d_bytes_per_step": int(wl.target.nbytes) // max(1, re["iters"]),
           "d2h_bytes_per_step": int(y_h.numel() * 4) // max(1, re["iters"]),
           "includes": "sipo_create (H2D target + device setup) + sipo_solve + D2H y*"}
    out = {"metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world,
           "steps": int(res["iters"]), "warmup": args.warmup,
           "ms_per_step": t_max * 1e3 / max(1, res["iters"]), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
           "config": workload_config(wl, args.storage), "e2e": e2e, "gpu_launches": int(launches),
           "roofline": roofline, "clocks": clk, "time_to_kkt_1e-4": kkt_info,
           "phases_ms": phases, "model_iter_ms": per_iter_ms,
           "solver": {"status": res["status_name"], "kkt": res["kkt"], "restarts": res["restarts"],
                      "bp_tile_cfg": res["tile_cfg"],
                      "check_every": args.check_every, "need_columns": need_cols,
                      "active_columns": act_cols}}
    sipo.sipo_destroy(ctx)
    return out, wl


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=256)
    p.add_argument("--warmup", type=int, default=16)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--workload", default="csg256")
    p.add_argument("--storage", default="f32", choices=["f32", "bf16", "f64"])
    p.add_argument("--check-every", type=int, default=64)
    p.add_argument("--case", type=int, default=None, choices=[0, 1, 2],
                   help="override the workload's LP case (1: tolerance band, 2: inhibition)")
    p.add_argument("--delta", type=float, default=0.05, help="case-1 dose tolerance")
    p.add_argument("--bp-tile", type=int, default=-1,
                   help="backprojector tile table entry (-1: autotuned at creation)")
    p.add_argument("--profile-iters", type=int, default=8)
    p.add_argument("--kkt-iters", type=int, default=2048)
    p.add_argument("--feasible-ratio", type=float, default=0.85)
    p.add_argument("--separation-omega", type=float, default=0.0,
                   help="initial primal weight of the separation LP (0: the library's rule)")
    p.add_argument("--separation-iters", type=int, default=16384,
                   help="iteration cap of the separation LP that settles Case-2 feasibility")
    p.add_argument("--probe-every", type=int, default=128,
                   help="iterations between Farkas probes of the Case-2 LP during the separation solve")
    p.add_argument("--separation-sequential", action="store_true",
                   help="also time the sequential form of the separation workflow (separation LP first)")
    p.add_argument("--escalate", type=int, default=0,
                   help="also time BF16 storage for N iterations, then FP32 warm-started from it")
    p.add_argument("--sweep-sequential", action="store_true",
                   help="--workload sweep: also solve the LPs one after another and time that")
    p.add_argument("--cpu-seconds", type=float, default=20.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    args = p.parse_args(argv)
    if args.warmup < 3:
        p.error("--warmup must be >= 3")
    world, rank, local = dist_env()

    if args.impl == "reference":
        # the CPU oracle is the reference implementation of this path
        if rank != 0:
            return 0
        wl = make_workload(args.workload)
        _apply_case(wl, args.case, args.delta)
        t0 = time.perf_counter()
        rate, single, steps, desc, cores = oracle_steps_rate(wl, args.warmup, args.steps, case=args.case,
                                                             delta=args.delta)
        out = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "iter/s",
               "n_gpus": world, "steps": steps, "warmup": args.warmup,
               "ms_per_step": 1e3 / rate, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": workload_config(wl, "f64"),
               "cpu_baseline": {"value": rate, "unit": "iter/s", "cores": cores, "kind": "oracle",
                                "sample": desc,
                                "single_process_in_pool": {"value": single, "unit": "iter/s", "cores": 1}},
               "e2e": {"value": rate, "unit": "iter/s", "h2d_bytes_per_step": 0,
                       "d2h_bytes_per_step": 0},
               "wall_s": time.perf_counter() - t0}
        print(json.dumps(out), flush=True)
        return 0

    import torch
    if not torch.cuda.is_available():
        print(json.dumps({"metric": METRIC, "error": "no CUDA device"}))
        return 1
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    dist = init_dist(world, "nccl")
    if args.workload == "sweep":
        out = run_sweep(args, device, dist, rank, world)
        if rank == 0:
            print(json.dumps(out), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return 0
    out, wl = run_gpu(args, dist, rank, world, device)
    if rank == 0:
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds, case=args.case, delta=args.delta)
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
