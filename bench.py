#!/usr/bin/env python
"""Benchmark of the two-scale Eikonal solver (one JSON line on rank 0).

A step is one complete solve through the C ABI of the largest single-grid
workload: a 4097 x 4097 grid with a 64 x 64 checkerboard of speeds F in
{1, 2} and a seeded maze of F = 0 walls one node thick with random gaps, 4
seeded point sources (the paper's checkerboard and comb-maze examples at the
single-GPU size): the double-float cell solves on the FP32 pipe and the FP64
residual certificate (precision "fp32ref", the default), or the plain FP64
solve (--precision fp64).  --workload sin1025 times the 1025 x 1025 grid with
F = 1 + 0.5 sin(20 pi x) sin(20 pi y) and a centre source instead.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own replica on its own GPU (the single
grid does not shard without an exchange step; instances are independent), so
scaling is weak and value = total points solved by all ranks / max rank time.
--impl reference times the CPU FP64 oracle (Fast Marching) on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "converged Mpts/s at max|err| vs FP64 oracle"
UNIT = "Mpts/s"
FALLBACK_HBM_GBS = 6800.0
WORKLOADS = {
    "checker_maze4097": "single solve FP32+FP64-refinement: 4097x4097 grid, piecewise-constant speed: 64x64 "
                        "checkerboard of F in {1,2} plus seeded maze of axis-aligned barrier walls 1 gridpoint "
                        "thick with F=0 leaving random gaps, 4 seeded random point sources",
    "sin1025": "single solve, 1025x1025 grid on [0,1]^2, F=1+0.5 sin(20 pi x) sin(20 pi y), point source at centre",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32ref", "fp64"], default="fp32ref")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="checker_maze4097")
    ap.add_argument("--k", type=int, default=0, help="cell size (0: the tuned default)")
    ap.add_argument("--bucket-width", type=float, default=0.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-grid batch measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the Poisson serving measurement")
    ap.add_argument("--no-sweep", action="store_true", help="skip the cell-size sweep")
    ap.add_argument("--no-configs", action="store_true", help="skip the C1 / C2-FP64 / C3 solves")
    ap.add_argument("--serving-requests", type=int, default=128)
    ap.add_argument("--batch-count", type=int, default=512,
                    help="grids in the batch measurement (512: the 512-grid workload; fewer for profiling)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload(name="checker_maze4097"):
    from paper_1110_6220_gb300 import workloads as W
    if name == "sin1025":
        return W.sin_point(1025, omega=20.0, amp=0.5)
    return W.checker_maze(4097)


def config_dict(args, k, precision, I=None):
    d = {"workload": WORKLOADS[args.workload], "grid": f"{I.nx}x{I.ny}" if I is not None else None,
         "precision": precision, "cell_k": k,
         "bucket_width": "library choice per pass" if args.bucket_width == 0 else args.bucket_width,
         "parallelism": "replicas (one independent grid per GPU)",
         "l2": "flushed between timed steps (256 MiB write)"}
    return d


# ------------------------------------------------------------------ CPU side
def cpu_baseline(I, seconds):
    """The oracle FMM, as it stands, on one host core: whole solves of the
    same grid until `seconds` have passed (at least one)."""
    import oracle
    oracle.build()
    n, t0 = 0, time.perf_counter()
    while True:
        oracle.fmm(I.F, I.h, I.si, I.sj, I.sq)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return {"value": n * I.npts / el / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} full {I.nx}x{I.ny} solves with the FP64 Fast Marching oracle "
                      f"(binary heap), 1 thread, {el:.1f} s"}


def _oracle_solve(args):
    """One grid with the oracle FMM (a worker of oracle_parallel)."""
    F, h, si, sj, sq = args
    import oracle
    oracle.fmm(F, h, si, sj, sq)
    return int(F.size)


def oracle_parallel(insts, seconds, cores=8):
    """The oracle FMM, as it stands, one grid per process on up to `cores`
    host cores (a pool started by spawn: the parent has initialised CUDA),
    each process taking the next grid when it is free.  The sample is the
    workload's first grids, as many as make about `seconds` of work per core
    at the oracle's single-core rate (~7 Mpts/s)."""
    import multiprocessing as mp
    import oracle
    from paper_1110_6220_gb300 import workloads as W
    oracle.build()
    cores = max(1, min(cores, os.cpu_count() or 1))
    sample, pts = [], 0
    for I in insts:
        sample.append(I)
        pts += I.npts
        if pts >= seconds * cores * 7e6:
            break
    tiny = W.const_point(17)
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_solve, [(tiny.F, tiny.h, tiny.si, tiny.sj, tiny.sq)] * cores)  # start and load
        t0 = time.perf_counter()
        done = sum(pool.imap_unordered(_oracle_solve, [(I.F, I.h, I.si, I.sj, I.sq) for I in sample]))
        el = time.perf_counter() - t0
    return {"value": done / el / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"the first {len(sample)} grids of the workload ({done} points), FP64 Fast Marching "
                      f"oracle, one grid per process on {cores} cores, {el:.1f} s"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    I = workload(args.workload)
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        oracle.fmm(I.F, I.h, I.si, I.sj, I.sq)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.fmm(I.F, I.h, I.si, I.sj, I.sq)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = args.steps * I.npts / tot / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(args, 0, "fp64 (CPU oracle)", I),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} full {I.nx}x{I.ny} FMM solves, 1 thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU side
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""

    def summary(self):
        rows = [r.split(",") for r in (self.out or "").strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows]
        smax = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[5 + i].strip().lower() == "active"})
        busy = [s for s in sm if s > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows)}


def measured_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return float(json.load(fh)["hbm_gbs"]), "of measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "of fallback"


# the sources the persistent solver kernels are compiled from (their
# instantiation units, the templates and the shared header, and the C API
# header it includes): a change elsewhere (host code, the node-wise kernels)
# leaves a committed DRAM-traffic figure of these kernels valid
SOLVER_SOURCES = ("paper_1110_6220_gb300/csrc/eik_common.cuh", "paper_1110_6220_gb300/csrc/eik_solver.cuh",
                  "paper_1110_6220_gb300/csrc/eik_solver_modes.cuh", "paper_1110_6220_gb300/csrc/eik_solver_df.cu",
                  "paper_1110_6220_gb300/csrc/eik_solver_f32.cu", "paper_1110_6220_gb300/csrc/eik_solver_f64.cu",
                  "include/eik.h")


def kernel_source_hash():
    h = hashlib.sha256()
    for f in SOLVER_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, k):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as fh:
            t = json.load(fh)
    except (OSError, ValueError):
        return None
    e = t.get(f"{kernel}/k{k}")
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return e.get("dram_bytes_per_launch")


def kernel_name(sched, prec, first):
    """The persistent kernel a pass ran, from eik_stats.schedule (bit 0: FP32
    pass round-free, bit 1: main pass round-free, bit 5: value order)."""
    if first:
        base, mode = ("k_solve_async" if sched & 1 else "k_solve"), "F32"
    else:
        base, mode = ("k_solve_async" if sched & 2 else "k_solve"), ("DF" if prec else "F64")
    order = ",ordered" if (sched & 32) and base == "k_solve_async" else ""
    return f"{base}<{mode}{order}>"


def roofline(stats, k, prec, npts, p32, p64):
    """Roofline of the dominant kernel (the longer persistent pass).
    Algorithmic bytes per grid point (each point read and written once, plus
    the halo of every cell): FP32 pass 4 B f + 2 x 4 B U, double-float and
    FP64 passes 8 B f + 2 x 8 B U, each times (1 + 4/k).  The pass's device
    time comes from events the library records around the launch on its
    stream (eik_stats.pass_ms)."""
    sched = stats[-1].schedule
    if p32 > p64:
        kname, kms, bpp = kernel_name(sched, prec, True), p32, 12.0 * (1 + 4.0 / k)
    else:
        kname, kms, bpp = kernel_name(sched, prec, False), p64, 24.0 * (1 + 4.0 / k)
    peak, peak_src = measured_hbm()
    achieved = bpp * npts / (kms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": ncu_traffic(kname, k), "peak_source": peak_src,
            "kernel": kname, "cell_k": k, "kernel_ms": kms, "algorithmic_bytes_per_pt": bpp,
            "algorithmic_bytes_per_launch": bpp * npts}


def k_sweep(eik, torch, I, reps=3):
    """The single 1025^2 solve at every cell size, both precisions: device
    time of whole solves (median of reps) and the error against the oracle."""
    import oracle
    F = torch.from_numpy(I.F).cuda()
    src = torch.from_numpy(I.src_ij).cuda()
    q = torch.from_numpy(np.ascontiguousarray(I.sq)).cuda()
    V = oracle.fmm(I.F, I.h, I.si, I.sj, I.sq)
    fin = np.isfinite(V)
    out = []
    for prec, pname in ((eik.EIK_FP64, "fp64"), (eik.EIK_FP32_REFINE, "fp32ref")):
        for k in (4, 8, 16, 32, 64):
            U = torch.empty_like(F)
            with eik.Plan(I.nx, I.ny, I.h, k, prec) as p:
                ms = []
                for r in range(reps + 1):
                    rc, st = p.solve(F, src, q, U)
                    if rc:
                        raise RuntimeError(f"eik_solve k={k}: {eik.eik_strerror(rc)}")
                    if r:
                        ms.append(st.ms)
            Ug = U.cpu().numpy()
            err = float(np.abs(Ug[fin] - V[fin]).max() / np.abs(V[fin]).max())
            med = statistics.median(ms)
            out.append({"precision": pname, "cell_k": k, "ms": med, "value": I.npts / med / 1e3,
                        "unit": UNIT, "max_rel_err": err, "rounds": st.rounds, "avhr": st.avhr,
                        "pass_ms": list(st.pass_ms), "value_ordered": bool(st.schedule & 32)})
    return out


def config_measure(eik, torch, I, prec, steps=5, k=0):
    """One more configuration: device-resident inputs, median device time of
    whole solves through a plan, and the error against the oracle."""
    import oracle
    F = torch.from_numpy(I.F).cuda()
    src = torch.from_numpy(I.src_ij).cuda()
    q = torch.from_numpy(np.ascontiguousarray(I.sq)).cuda()
    U = torch.empty_like(F)
    ms, sts = [], []
    with eik.Plan(I.nx, I.ny, I.h, k, prec) as p:
        for r in range(steps + 2):
            rc, st = p.solve(F, src, q, U)
            if rc:
                raise RuntimeError(f"eik_solve {I.name}: {eik.eik_strerror(rc)}")
            if r >= 2:
                ms.append(st.ms)
                sts.append(st)
    V = oracle.fmm(I.F, I.h, I.si, I.sj, I.sq)
    Ug = U.cpu().numpy()
    fin = np.isfinite(V)
    err = float(np.abs(Ug[fin] - V[fin]).max() / np.abs(V[fin]).max())
    med = statistics.median(ms)
    out = {"grid": f"{I.nx}x{I.ny}", "precision": "fp64" if prec == eik.EIK_FP64 else "fp32ref",
           "cell_k": st.cell_k, "ms": med, "value": I.npts / med / 1e3, "unit": UNIT,
           "max_rel_err": err, "inf_pattern_exact": bool((np.isfinite(Ug) == fin).all()),
           "err_bound": st.err_bound, "avhr": st.avhr, "avs": st.avs, "buckets": st.buckets,
           "schedule": st.schedule, "value_ordered": bool(st.schedule & 32),
           "roofline": roofline(sts, st.cell_k, prec, I.npts, statistics.mean(x.pass_ms[0] for x in sts),
                                statistics.mean(x.pass_ms[1] for x in sts))}
    if prec == eik.EIK_FP64:
        # the FP64 pipe: three FP64 adds per node evaluation (the library's
        # count of evaluations, lock-step passes included) against GB300's
        # nominal FP64 rate, 1.25 TFLOP/s = 0.625 T instructions/s
        adds = 3.0 * st.updates_per_pt * I.npts
        out["fp64_pipe"] = {"bound": "alu", "achieved": adds / (med / 1e3) / 1e9, "peak": 625.0,
                            "unit": "G FP64 instructions/s", "frac": adds / (med / 1e3) / 625e9,
                            "peak_source": "of nominal", "updates_per_pt": st.updates_per_pt}
    return out


def fhcm_measure(eik, torch, I, steps=5):
    """The heap-cell variants on the single 1025^2 grid, FP64: the Fast
    Heap-Cell Method (Sec. 4.3) beside the exact one (HCM) and HCM with
    locking inside cells (Remark locking_FSM; exact, fewer local updates),
    and the Fast Marching-Sweeping Method (Sec. 4.1) at three cell sizes;
    device times and Sec. 5's error ratios against Fast Marching on an h/4
    grid, beside the oracle's serial FHCM / FMSM and the paper's Tab. sinu_1
    rows for the closest cell size.  Returns (fhcm, fmsm) dictionaries."""
    import oracle
    from paper_1110_6220_gb300 import workloads as W
    F = torch.from_numpy(I.F).cuda()
    src = torch.from_numpy(I.src_ij).cuda()
    q = torch.from_numpy(np.ascontiguousarray(I.sq)).cuda()
    U = torch.empty_like(F)
    out = {}
    for name, method in (("hcm", eik.EIK_METHOD_HCM), ("fhcm", eik.EIK_METHOD_FHCM),
                         ("hcm_lsm", eik.EIK_METHOD_HCM_LSM)):
        ms = []
        with eik.Plan(I.nx, I.ny, I.h, 0, eik.EIK_FP64, method=method) as p:
            for r in range(steps + 2):
                rc, st = p.solve(F, src, q, U)
                if rc:
                    raise RuntimeError(f"eik_solve ({name}): {eik.eik_strerror(rc)}")
                if r >= 2:
                    ms.append(st.ms)
        med = statistics.median(ms)
        out[name] = {"ms": med, "value": I.npts / med / 1e3, "unit": UNIT, "cell_k": st.cell_k,
                     "avhr": st.avhr, "avs": st.avs, "updates_per_pt": st.updates_per_pt}
        if method == eik.EIK_METHOD_FHCM:
            out[name]["mono_pct"] = st.mono_pct
            Ug = U.cpu().numpy()
        if method == eik.EIK_METHOD_HCM_LSM:
            Ul = U.cpu().numpy()
    n = I.nx
    J = W.sin_point(4 * (n - 1) + 1)
    orc = oracle.default()
    V = orc.fmm(I.F, I.h, I.si, I.sj, I.sq)
    truth = orc.fmm(J.F, J.h, J.si, J.sj, J.sq)[::4, ::4]
    e = np.abs(V - truth)
    m = e > 0

    def ratios(X):
        E = np.abs(X - truth)
        return {"R": float((E[m] / e[m]).max()), "rho": float((E[m] / e[m]).mean()),
                "R_max_errors": float(E.max() / e.max())}
    out["fhcm"].update(ratios(Ug))
    fin = np.isfinite(V)
    out["hcm_lsm"]["max_rel_err_vs_oracle_fmm"] = float(np.abs(Ul[fin] - V[fin]).max() / np.abs(V[fin]).max())
    out["fhcm"]["below_exact"] = int((Ug < V - 1e-12 * V.max()).sum())
    Uo, so = orc.cells(I.F, I.h, I.si, I.sj, I.sq, out["fhcm"]["cell_k"], fast=True)
    out["oracle_serial_fhcm"] = dict(ratios(Uo), avhr=so["avhr"], avs=so["avs"], mono_pct=so["mon_pct"])
    out["paper_tab_sinu_1_fhcm_176_cells"] = {"R": 1.0560, "rho": 1.0022, "R_max_errors": 1.0000,
                                               "avhr": 1.125, "avs": 1.262, "mono_pct": 94.5,
                                               "note": "1408^2 grid, 8-node cells; context"}
    fm = {}
    for k in (8, 16, 32):
        ms, coarse, main = [], [], []
        with eik.Plan(I.nx, I.ny, I.h, k, eik.EIK_FP64, method=eik.EIK_METHOD_FMSM) as p:
            for r in range(steps + 2):
                rc, st = p.solve(F, src, q, U)
                if rc:
                    raise RuntimeError(f"eik_solve (fmsm): {eik.eik_strerror(rc)}")
                if r >= 2:
                    ms.append(st.ms)
                    coarse.append(st.pass_ms[0])
                    main.append(st.pass_ms[1])
        med = statistics.median(ms)
        Ug = U.cpu().numpy()
        Uo, so = orc.fmsm(I.F, I.h, I.si, I.sj, I.sq, k)
        fm[f"k{k}"] = dict({"ms": med, "value": I.npts / med / 1e3, "unit": UNIT,
                            "coarse_solve_ms": statistics.median(coarse), "cell_pass_ms": statistics.median(main),
                            "avs": st.avs, "launches": st.launches,
                            "max_rel_diff_vs_oracle_fmsm": float(np.abs(Ug - Uo)[np.isfinite(Uo)].max() /
                                                                 np.abs(Uo[np.isfinite(Uo)]).max()),
                            "oracle_avs": so["avs"]}, **ratios(Ug))
    fm["paper_tab_sinu_1_fmsm"] = {
        "k8_176_cells": {"R": 3.4828, "rho": 1.0074, "R_max_errors": 1.3705, "avs": 1.126},
        "k16_88_cells": {"R": 4.6801, "rho": 1.0515, "R_max_errors": 1.9504, "avs": 1.213},
        "k32_44_cells": {"R": 6.0892, "rho": 1.3657, "R_max_errors": 2.2889, "avs": 1.200},
        "note": "1408^2 grid; context"}
    return out, fm


def batch_measure(eik, torch, steps=5, warmup=2, k=0, count=512, cpu_seconds=0.0):
    """The batched workload: 512 grids with side lengths log-uniform in
    [65, 1025] (sin-product or random-block speeds, 1-8 sources), FP32 +
    refinement, inputs resident on the device.  Timed as a fixed batch
    (eik_batch_create once, then eik_batch_run: the captured launch sequence
    replayed), wall clock per run including the result read-back; the one-off
    eik_solve_batch call (which builds the job each time) is timed beside it."""
    from paper_1110_6220_gb300 import workloads as W
    insts = W.batch_mix(count, seed=1)
    npts = sum(I.npts for I in insts)
    dev = []
    for I in insts:
        F = torch.from_numpy(I.F).cuda()
        dev.append((F, torch.from_numpy(I.src_ij).cuda(), torch.from_numpy(I.sq).cuda(), torch.empty_like(F)))
    descs = [eik.make_desc(I.nx, I.ny, I.h, k, eik.EIK_FP32_REFINE) for I in insts]
    ins = [eik.make_instance(*d) for d in dev]
    torch.cuda.synchronize()
    batch = eik.eik_batch_create(descs, ins)
    try:
        for _ in range(warmup):
            eik.eik_batch_run(batch)
        wall, dms = [], []
        for _ in range(steps):
            t0 = time.perf_counter()
            rc, st = eik.eik_batch_run(batch)
            wall.append(1e3 * (time.perf_counter() - t0))
            if rc:
                raise RuntimeError(f"eik_batch_run: {eik.eik_strerror(rc)}")
            dms.append(st[0].ms)
    finally:
        eik.eik_batch_destroy(batch)
    one_off = []
    for r in range(3):
        t0 = time.perf_counter()
        rc, st1 = eik.eik_solve_batch(descs, ins)
        if rc:
            raise RuntimeError(f"eik_solve_batch: {eik.eik_strerror(rc)}")
        if r:
            one_off.append(1e3 * (time.perf_counter() - t0))
    med = statistics.median(wall)
    # the dominant kernel is the persistent pass over all grids: its time from
    # the kernel's own start and end stamps (events do not time inside a
    # replayed graph), its bytes those of every grid's points
    pk = st[0].pass_ms[1]
    kb = st[0].cell_k
    bpp = 24.0 * (1 + 4.0 / kb)
    peak, peak_src = measured_hbm()
    kname = kernel_name(st[0].schedule, 1, False)
    roof = {"bound": "hbm", "achieved": bpp * npts / (pk / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
            "frac": bpp * npts / (pk / 1e3) / 1e9 / peak, "traffic": ncu_traffic(kname + "/batch", kb),
            "peak_source": peak_src, "kernel": kname, "cell_k": kb, "kernel_ms": pk,
            "algorithmic_bytes_per_pt": bpp, "algorithmic_bytes_per_launch": bpp * npts}
    out = {"workload": f"{count} grids, n log-uniform in [65, 1025], sin-product or random-block F, "
                       "1-8 sources, seed 1", "precision": "fp32ref", "cell_k_used": st[0].cell_k,
           "roofline": roof,
           "points": npts, "ms_per_batch": med, "value": npts / (med / 1e3) / 1e6, "unit": UNIT,
           "timing": "wall clock per eik_batch_run (graph replay + read-back), median of 5",
           "device_ms": statistics.median(dms), "pass_ms": list(st[0].pass_ms),
           "graph_replay": bool(st[0].schedule & 8),
           "max_err_bound": max(s.err_bound for s in st), "launches_per_batch": st[0].launches,
           "one_off_eik_solve_batch_ms": statistics.median(one_off),
           "one_off_value": npts / (statistics.median(one_off) / 1e3) / 1e6}
    if cpu_seconds > 0:
        out["cpu_baseline_parallel"] = oracle_parallel(insts, cpu_seconds)
    return out

def _pct(xs, p):
    xs = sorted(xs)
    if not xs:
        return None
    i = min(len(xs) - 1, max(0, int(math.ceil(p / 100.0 * len(xs))) - 1))
    return xs[i]


def serving_measure(eik, torch, count=128, seed=5, budget=64 << 30, cpu_seconds=0.0):
    """The serving workload: a seeded Poisson stream of FP32 + refinement
    solves, side lengths log-uniform in [129, 2049], sin-product, random-block
    and checkerboard+maze speeds in equal shares, served through
    eik_submit / eik_poll with a 64 GB admission budget.  Reports the
    saturated throughput (all requests submitted at once) and p50/p99
    latency at 0.5x and 0.9x of that rate, beside the same stream solved as
    serial plain solves (one eik_solve per request in arrival order; their
    latency follows from the measured service times and the arrival times)."""
    from paper_1110_6220_gb300 import workloads as W
    stream = W.poisson_stream(count, 1.0, seed=seed)
    insts = [I for _, I in stream]
    unit_arrivals = [t for t, _ in stream]  # rate 1 per second; rescaled below
    npts = sum(I.npts for I in insts)
    dev = []
    for I in insts:
        F = torch.from_numpy(I.F).cuda()
        dev.append((F, torch.from_numpy(I.src_ij).cuda(), torch.from_numpy(I.sq).cuda(),
                    torch.empty_like(F)))
    descs = [eik.make_desc(I.nx, I.ny, I.h, 0, eik.EIK_FP32_REFINE) for I in insts]
    ins = [eik.make_instance(*d) for d in dev]
    torch.cuda.synchronize()

    # serial plain solves, back to back, one plan per request shape
    plans = {}
    for I in insts:
        if (I.nx, I.ny) not in plans:
            plans[(I.nx, I.ny)] = eik.Plan(I.nx, I.ny, I.h, 0, eik.EIK_FP32_REFINE)
    for e in range(min(4, count)):  # warm-up
        plans[(insts[e].nx, insts[e].ny)].solve(*dev[e])
    service = []
    t0 = time.perf_counter()
    for I, d in zip(insts, dev):
        a = time.perf_counter()
        rc, _ = plans[(I.nx, I.ny)].solve(*d)
        if rc:
            raise RuntimeError(f"eik_solve: {eik.eik_strerror(rc)}")
        service.append(time.perf_counter() - a)
    serial_s = time.perf_counter() - t0
    for p in plans.values():
        p.close()

    def serial_latency(arr):
        lat, free = [], 0.0
        for a, s in zip(arr, service):
            start = max(a, free)
            free = start + s
            lat.append(free - a)
        return lat

    srv = eik.eik_server_create(budget, count)
    try:
        def run(arrivals):
            """Submit each request at its arrival time (None: all at once);
            returns (makespan s, latencies s, stats)."""
            pending, lat, sts = {}, [0.0] * count, [None] * count
            nxt = 0
            t0 = time.perf_counter()
            while nxt < count or pending:
                now = time.perf_counter() - t0
                while nxt < count and (arrivals is None or arrivals[nxt] <= now):
                    rc, t = eik.eik_submit(srv, descs[nxt], ins[nxt])
                    if rc:
                        raise RuntimeError(f"eik_submit: {eik.eik_strerror(rc)}")
                    pending[t] = (nxt, now if arrivals is not None else 0.0)
                    nxt += 1
                for t in list(pending):
                    rc, st = eik.eik_poll(srv, t)
                    if rc == eik.EIK_EAGAIN:
                        continue
                    e, arr = pending.pop(t)
                    if rc:
                        raise RuntimeError(f"eik_poll: {eik.eik_strerror(rc)}")
                    lat[e] = time.perf_counter() - t0 - arr
                    sts[e] = st
                time.sleep(5e-5)
            return time.perf_counter() - t0, lat, sts

        run(None)  # warm-up
        sat_s, sat_lat, sts = run(None)
        rate = count / sat_s
        out = {"workload": f"{count} requests, Poisson arrivals (seed {seed}), n log-uniform in "
                           "[129, 2049], sin-product / random-block / checkerboard+maze F, "
                           "1-8 sources, 64 GB admission budget",
               "precision": "fp32ref", "requests": count, "points": npts,
               "saturated": {"req_per_s": rate, "value": npts / sat_s / 1e6, "unit": UNIT,
                             "makespan_s": sat_s},
               "serial_plain": {"req_per_s": count / serial_s, "value": npts / serial_s / 1e6,
                                "unit": UNIT, "p50_service_ms": 1e3 * _pct(service, 50),
                                "p99_service_ms": 1e3 * _pct(service, 99)},
               "max_err_bound": max(s.err_bound for s in sts), "load": []}
        for frac in (0.5, 0.9):
            lam = frac * rate
            arr = [t / lam for t in unit_arrivals]
            span, lat, _ = run(arr)
            sl = serial_latency(arr)
            out["load"].append({
                "rate_frac_of_saturated": frac, "req_per_s": lam,
                "p50_ms": 1e3 * _pct(lat, 50), "p99_ms": 1e3 * _pct(lat, 99),
                "serial_p50_ms": 1e3 * _pct(sl, 50), "serial_p99_ms": 1e3 * _pct(sl, 99),
                "value": npts / span / 1e6, "unit": UNIT})
        if cpu_seconds > 0:
            out["cpu_baseline_parallel"] = oracle_parallel(insts, cpu_seconds)
        return out
    finally:
        eik.eik_server_destroy(srv)


def replica_rate(local_ms, npts, steps, world, device):
    """Replicas: every rank solved `steps` grids of `npts` points in local_ms.
    The job took the slowest rank's time (max over ranks); the rate is all
    ranks' points over it, in Mpts/s.  Returns (max ms, rate)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        local_ms = float(t.item())
    return local_ms, world * steps * npts / (local_ms / 1e3) / 1e6


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the solver has no CPU path)")
    torch.cuda.set_device(local)
    from paper_1110_6220_gb300 import build
    build.build()
    from paper_1110_6220_gb300 import eik

    I = workload(args.workload)
    prec = eik.EIK_FP32_REFINE if args.precision == "fp32ref" else eik.EIK_FP64
    k = args.k  # 0: the library's choice (tuned table or built-in)
    stream = torch.cuda.current_stream()
    dev = torch.device("cuda", local)
    F = torch.from_numpy(I.F).to(dev)
    src = torch.from_numpy(I.src_ij).to(dev)
    q = torch.from_numpy(I.sq).to(dev)
    U = torch.empty_like(F)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2
    plan = eik.Plan(I.nx, I.ny, I.h, k, prec, bucket_width=args.bucket_width, stream=stream)

    def step():
        rc, st = plan.solve(F, src, q, U)
        if rc:
            raise RuntimeError(f"eik_solve: {eik.eik_strerror(rc)}")
        return st

    for _ in range(max(args.warmup, 3)):
        k = step().cell_k
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    stats = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for e0, e1 in ev:
            flush.zero_()
            e0.record(stream)
            stats.append(step())
            e1.record(stream)
        torch.cuda.synchronize()
    step_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    tot_ms, value = replica_rate(sum(step_ms), I.npts, args.steps, world, dev)
    if world > 1:
        dist.barrier()

    # ---- end to end through the public API with host (pinned) buffers
    Fh = torch.from_numpy(I.F).pin_memory()
    srch = torch.from_numpy(I.src_ij).pin_memory()
    qh = torch.from_numpy(I.sq).pin_memory()
    Uh = torch.empty(I.F.shape, dtype=torch.float64).pin_memory()
    for _ in range(2):
        plan.solve(Fh, srch, qh, Uh)
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rc, _ = plan.solve(Fh, srch, qh, Uh)
        b.record(stream)
        b.synchronize()
        if rc:
            raise RuntimeError(f"eik_solve (host buffers): {eik.eik_strerror(rc)}")
        e2e_ms.append(a.elapsed_time(b))
    e2e_tot, e2e_value = replica_rate(sum(e2e_ms), I.npts, args.steps, world, dev)

    if rank == 0:
        Ug = U.cpu().numpy()
        import oracle
        V = oracle.fmm(I.F, I.h, I.si, I.sj, I.sq)
        fin = np.isfinite(V)
        rel_err = float(np.abs(Ug[fin] - V[fin]).max() / np.abs(V[fin]).max())
        same_inf = bool((np.isfinite(Ug) == fin).all())

        # ---- roofline of the dominant kernel (the longer persistent pass).
        # Algorithmic bytes per grid point (each point read and written once,
        # plus the halo): FP32 pass 4 B f + 2 x 4 B U, double-float refinement
        # and FP64 passes 8 B f + 2 x 8 B U, each times (1 + 4/k).
        p32 = statistics.mean(s.pass_ms[0] for s in stats)
        p64 = statistics.mean(s.pass_ms[1] for s in stats)
        roof = roofline(stats, k, prec, I.npts, p32, p64)
        s0 = stats[-1]
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64" if prec else "f64", "data": "synthetic",
                "config": config_dict(args, k, args.precision, I),
                "max_rel_err": rel_err, "inf_pattern_exact": same_inf,
                "err_bound": s0.err_bound, "status": eik.eik_strerror(s0.status),
                "roofline": roof,
                "e2e": {"value": e2e_value, "unit": UNIT,
                        "h2d_bytes_per_step": int(I.F.nbytes + I.src_ij.nbytes + I.sq.nbytes),
                        "d2h_bytes_per_step": int(I.F.nbytes)},
                "gpu_launches": int(sum(s.launches for s in stats)),
                "clocks": clk.summary(),
                "solver": {"avhr": s0.avhr, "avs": s0.avs, "updates_per_pt": s0.updates_per_pt,
                           "rounds": s0.rounds, "buckets": s0.buckets,
                           "pass_ms": [p32, p64], "solve_ms_device": statistics.mean(s.ms for s in stats),
                           "paper_hcm_k8_1408": {"avhr": 1.117, "avs": 4.350,
                                                 "cite": "Tab. sinu_1, HCM 176x176 cells"}}}
        line["solver"]["bucket_width_main"] = s0.bucket_width
        line["solver"]["schedule"] = {"fp32_pass_round_free": bool(s0.schedule & 1),
                                      "main_pass_round_free": bool(s0.schedule & 2),
                                      "one_double_float_pass": bool(s0.schedule & 4),
                                      "value_ordered": bool(s0.schedule & 32)}
        from paper_1110_6220_gb300 import workloads as W
        C2 = I if args.workload == "sin1025" else W.sin_point(1025)
        if not args.no_sweep:
            line["k_sweep"] = k_sweep(eik, torch, C2)
        if not args.no_configs:
            line["configs"] = {
                "c1_const129_fp64": config_measure(eik, torch, W.const_point(129), eik.EIK_FP64),
                "c2_sin1025_fp32ref": config_measure(eik, torch, C2, eik.EIK_FP32_REFINE),
                "c2_sin1025_fp64": config_measure(eik, torch, C2, eik.EIK_FP64),
                "c3_checker_maze4097_fp64": config_measure(eik, torch, W.checker_maze(4097), eik.EIK_FP64),
                "q_boundary_sin1025_fp32ref": config_measure(eik, torch, W.sin_boundary(1025), eik.EIK_FP32_REFINE),
                "q_boundary_sin1025_fp64": config_measure(eik, torch, W.sin_boundary(1025), eik.EIK_FP64),
            }
            if args.workload == "sin1025":
                line["configs"]["c3_checker_maze4097_fp32ref"] = config_measure(
                    eik, torch, W.checker_maze(4097), eik.EIK_FP32_REFINE)
        if not args.no_configs:
            line["fhcm"], line["fmsm"] = fhcm_measure(eik, torch, C2)
        if not args.no_batch:
            line["batch"] = batch_measure(eik, torch, count=args.batch_count,
                                          cpu_seconds=0.0 if args.no_cpu_baseline else 10.0)
        if not args.no_serving:
            line["serving"] = serving_measure(eik, torch, count=args.serving_requests,
                                              cpu_seconds=0.0 if args.no_cpu_baseline else 10.0)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(I, args.cpu_seconds)
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
