"""Benchmark of the cut-cell step on GB300 (one JSON line on rank 0).

Workloads (synthetic, seeded; the paper's hills sampled at grid corners):
  ensemble   64 independent single-level domains of uneven sizes (64^3 ..
             192x192x96), seed 1509, bell or half-ellipsoid hills; all
             instances advance together in one launch per stage in the FP32
             perturbation form; the plain FP64 form loops over the instances.
  hemisphere the 128x128x64 grid of 50 m cells over the 1 km hemisphere (FP64).
  bell512    the 512x512x128 grid (100 m, dz 50 m) over the 400 m / 2 km bell,
             FP32 against its FP64 run (--error-steps for long comparisons).
  refined    three block-structured levels (200 m over 64x32x16 km, 100 m and
             50 m boxes around the 1 km hemisphere), FP32 perturbation form;
             a step is one cycle of level 0 (2 steps of level 1, 4 of level 2).
The default run (ensemble) also measures the refined workload and adds it as
the "refined" object of the line.

A step is one leapfrog step of every domain of the workload (all stages:
full-cell stencil, cut-cell groups, velocity diagnosis, and for the refined
workload the flux register, restriction and prolongation).
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
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1509_02572_gb300 import workloads as W  # noqa: E402

METRIC = "cell-updates/s"
BYTES_PER_CELL = {"f32": 80, "f64": 160}  # 5 fields x (read n-1, read n, write n+1, write filtered n)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ensemble",
                    choices=["ensemble", "hemisphere", "bell512", "refined", "refined-blocks", "convergence",
                             "refined-vs-uniform"])
    ap.add_argument("--seconds", type=float, default=3600.0,
                    help="simulated time of each run of the convergence workload")
    ap.add_argument("--error-steps", type=int, default=0,
                    help="extra untimed steps of the FP32 and FP64 runs before their difference is taken")
    ap.add_argument("--no-refined", action="store_true", help="skip the refined object of the default run")
    ap.add_argument("--instances", type=int, default=64)
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the FP32-against-FP64 precision run of the 512 x 512 x 128 bell")
    ap.add_argument("--precision-steps", type=int, default=5000)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--schedule", default=None,
                    help="TILE_Y,ITEMS[,ROLES]: fixed full-cell schedule (and FP32 warp roles, 1 or 2) instead "
                         "of the autotuner (profiling runs)")
    return ap.parse_args()


def workload_configs(args):
    if args.workload == "ensemble":
        cfgs = W.ensemble_configs(args.instances, 1509)
        name = f"ensemble-{len(cfgs)}x(64^3..192x192x96)-seed1509"
    elif args.workload == "bell512":
        cfgs = [W.C3_BELL]
        name = W.C3_BELL.name
    else:
        cfgs = [W.C2_HEMI]
        name = W.C2_HEMI.name
    return name, cfgs


def kfull_source_hash(dtype="f64"):
    """Hash of the full-cell stencil's source (the kernel, its shared-memory
    layout and tile shape): the counters recorded under profiles/ apply only
    while it is unchanged.  FP64 runs the one-cell kernel of step.cu, FP32 the
    two-cell kernel of pair.cuh with the helpers of step.cu it calls (the
    copies and the equation of state)."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1509_02572_gb300", "csrc")
    hdr = open(os.path.join(csrc, "cc_internal.h")).read()
    tiles = [ln for ln in hdr.splitlines() if "TILE_" in ln or "SCHED_" in ln or "constexpr int GX" in ln]
    if dtype == "f32":
        src = open(os.path.join(csrc, "step.cu")).read()
        body = src[:src.index("struct FullCfg")] + open(os.path.join(csrc, "pair.cuh")).read()
    else:
        src = open(os.path.join(csrc, "step.cu")).read()
        a = src.index("struct FullCfg")
        body = src[a:src.index('#include "pair.cuh"', a)]
    return hashlib.sha256((body + "\n".join(tiles)).encode()).hexdigest()[:16]


def kfull_traffic(dtype, cells, schedule, roles=1):
    """DRAM bytes of one k_full launch over `cells` interior cells, scaled
    from the committed ncu capture (per interior cell) of the same tile height
    and warp roles, or None when the kernel changed since the capture or the
    precision differs."""
    try:
        with open(os.path.join(ROOT, "profiles", "k_full_traffic.json")) as f:
            t = json.load(f)
    except Exception:
        return None
    if t.get("source_hash") != kfull_source_hash(dtype) or t.get("precision") != {"f32": "fp32", "f64": "fp64"}[dtype]:
        return None
    per = t.get("dram_bytes_per_interior_cell_by_schedule", {}).get(f"{schedule[0]}x{roles}")
    if per is None and roles == 1:
        per = t.get("dram_bytes_per_interior_cell_by_tile_y", {}).get(str(schedule[0]))
    return None if per is None else per * cells


def refined_kfull_traffic(dtype, workload, schedules):
    """DRAM bytes of the full-cell stencil per launch, averaged over the
    launches of one cycle (as the refined roofline averages its algorithmic
    bytes), from the committed ncu capture of the refined workload; None when
    the kernel, the precision, the workload or the tile heights of the levels
    differ (the items per launch only split the z-columns)."""
    try:
        with open(os.path.join(ROOT, "profiles", "k_full_traffic.json")) as f:
            t = json.load(f)
    except Exception:
        return None
    r = t.get("refined")
    if (r is None or t.get("source_hash") != kfull_source_hash("f32") or dtype != "f32"
            or r.get("workload") != workload or [(x[0], (x + [1, 1])[2]) for x in r.get("schedule", [])]
            != [(x[0], (x + [1, 1])[2]) for x in schedules]):
        return None
    return r["cycle_dram_bytes"] / r["cycle_launches"]


def job_time_and_rate(ms, units_per_rank, world, dist=None, device="cuda"):
    """Whole-job timing over the ranks: the slowest rank's time (max over
    ranks) and the units all ranks processed divided by it."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    msmax = float(t.item())
    return msmax, units_per_rank * world / (msmax / 1e3)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.p = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", delete=False, suffix=".csv")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if "Active" in v and "Not" not in v:
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def fluid_cells(model, cfgs):
    n = 0
    for d in range(len(cfgs)):
        g = model.geometry(d)
        n += int((g["cls"] != 0).sum())
    return n


SCHEDULE = None  # fixed (tile_y, items[, warp roles]) from --schedule


def make_model(cc, cfgs, prec, tune=True):
    m = cc.Model(cfgs, prec)
    for d, c in enumerate(cfgs):
        m.set_terrain(d, c.heights())
    m.build_geometry()
    m.init_state()
    if SCHEDULE:
        m.set_schedule(0, *SCHEDULE[:2])
        if len(SCHEDULE) > 2 and prec == cc.CC_FP32:
            m.set_warp_roles(0, SCHEDULE[2])
    elif tune:
        m.autotune(3)
    return m


def time_steps(torch, model, steps, warmup):
    """W untimed steps, then K steps between events on the model's stream
    (Python's garbage collector paused while the steps are issued)."""
    for _ in range(warmup):
        model.step(1)
    model.synchronize()
    gc.collect()
    gc.disable()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    e0.record(st)
    for _ in range(steps):
        model.step(1)
        launches += model.last_launch_count
    e1.record(st)
    e1.synchronize()
    gc.enable()
    return e0.elapsed_time(e1), launches


def time_graphs(torch, model, steps):
    """The same steps replayed from CUDA graphs, without per-stage events."""
    model.profile(False)
    model.graphs(True)
    model.step(4)  # capture the four arrangements of the time levels
    model.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    model.step(steps)
    e1.record(st)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def cpu_baseline(cfgs, seconds):
    """The FP64 oracle as it stands on the host cores, on a bounded sample of
    the workload: whole instances, stepped until about `seconds` of CPU work."""
    import oracle
    t_used, cells_done, steps_done, inst = 0.0, 0, 0, []
    for c in cfgs:
        m = oracle.Model(c)
        nf = int((m.geometry()["cls"] != 0).sum())
        m.init_state()
        m.step(1)  # forward-Euler start, not timed
        s = 0
        t0 = time.perf_counter()
        while True:
            m.step(1)
            s += 1
            if time.perf_counter() - t0 >= seconds / 2 or s >= 50:
                break
        dt = time.perf_counter() - t0
        t_used += dt
        cells_done += nf * s
        steps_done += s
        inst.append(f"{c.name} x {s} steps")
        del m
        if t_used >= seconds:
            break
    return {"value": cells_done / t_used, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": "; ".join(inst) + f" ({t_used:.1f} s, single-threaded FP64 oracle)"}


def _allcore_worker(cfg, seconds, barrier, q):
    """One core: build the oracle instance, one untimed forward-Euler step,
    then (after every worker is ready) step it for about `seconds`."""
    import oracle
    m = oracle.Model(cfg)
    nf = int((m.geometry()["cls"] != 0).sum())
    m.init_state()
    m.step(1)
    barrier.wait()
    s, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        m.step(1)
        s += 1
    q.put((cfg.name, nf * s, s, time.perf_counter() - t0))


def cpu_baseline_allcores(cfgs, seconds):
    """The FP64 oracle as it stands on every host core at once: one spawned
    process per core, each stepping its own instance of the workload (the
    smallest ones, so that the memory stays bounded) from a common start; the
    rate is the sum of the processes' rates."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    ncores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    pick = sorted(cfgs, key=lambda c: c.cells)
    pick = [pick[w % len(pick)] for w in range(ncores)]
    ctx = mp.get_context("spawn")
    barrier, q = ctx.Barrier(ncores), ctx.Queue()
    procs = [ctx.Process(target=_allcore_worker, args=(c, seconds, barrier, q)) for c in pick]
    for p in procs:
        p.start()
    res = []
    try:
        import queue as _queue
        for _ in procs:
            res.append(q.get(timeout=seconds + 600.0))  # set-up and stepping; a dead worker ends the wait
    except _queue.Empty:
        pass
    for p in procs:
        p.join(timeout=5.0)
        if p.is_alive():
            p.terminate()
            p.join()
    if len(res) < ncores:
        return {"value": None, "unit": METRIC, "cores": ncores, "kind": "oracle",
                "error": f"{ncores - len(res)} of {ncores} oracle processes did not finish"}
    rate = sum(r[1] / r[3] for r in res)
    names = sorted({r[0] for r in res})
    return {"value": rate, "unit": METRIC, "cores": ncores, "kind": "oracle",
            "sample": f"{ncores} processes, one per host core, each stepping one instance for {seconds:.0f} s "
                      f"({', '.join(names)}); single-threaded FP64 oracle in each"}


def fp64_flops_per_cell(tile_y):
    """Executed FP64 flops of the FP64 full-cell stencil per interior cell
    (2 per fused multiply-add) for tiles of height tile_y, from the committed
    ncu count, or None when the kernel changed since the count."""
    try:
        with open(os.path.join(ROOT, "profiles", "k_full_fp64_flops.json")) as f:
            t = json.load(f)
    except Exception:
        return None
    if t.get("source_hash") != kfull_source_hash("f64"):
        return None
    return t.get("flops_per_interior_cell_by_tile_y", {}).get(str(tile_y))


FIELDS5 = (("rho'", "RHOP"), ("p'", "PP"), ("rho u", "MX"), ("rho v", "MY"), ("rho w", "MZ"))


def precision_columns(cfg):
    """Sampled columns (J, I) of the precision check: a 6 x 6 lattice over the
    domain and rings at 5, 10 and 20 cells around the hill centre."""
    cols = set()
    for a in range(6):
        for b in range(6):
            cols.add(((cfg.ny * (2 * a + 1)) // 12, (cfg.nx * (2 * b + 1)) // 12))
    cj, ci = cfg.ny // 2, cfg.nx // 2
    for r in (5, 10, 20):
        for dj, di in ((0, r), (0, -r), (r, 0), (-r, 0)):
            cols.add((cj + dj, ci + di))
    cols = sorted(cols)
    return np.array([c[0] for c in cols]), np.array([c[1] for c in cols])


def _oracle_columns_worker(cfg, steps, q):
    """The oracle alone on the host: `steps` steps of the whole domain, then
    every field on the sampled columns."""
    import oracle
    om = oracle.Model(cfg)
    om.init_state()
    om.step(steps)
    J, I = precision_columns(cfg)
    q.put({name: om.field(getattr(oracle, "F_" + f), 1)[:, J, I] for name, f in FIELDS5})


def bench_precision(cc, torch, steps):
    """FP32 perturbation form against the plain FP64 form on the 512 x 512 x
    128 bell (100 m / 50 m cells, h0 = 400 m, a = 2 km) after `steps` steps,
    per field over the whole domain; and both forms against the oracle on
    sampled columns after two steps (the oracle runs the whole domain on the
    host meanwhile, in a spawned process)."""
    import multiprocessing as mp
    import queue as _queue
    import oracle
    oracle.build()
    cfg = W.C3_BELL
    ostep = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    proc = ctx.Process(target=_oracle_columns_worker, args=(cfg, ostep, q))
    proc.start()
    J, I = precision_columns(cfg)
    t0 = time.perf_counter()
    fields, early = {}, {}
    for prec, tag in ((cc.CC_FP32, "fp32"), (cc.CC_FP64, "fp64")):
        m = make_model(cc, [cfg], prec)
        m.step(ostep)
        early[tag] = {name: m.download(0, getattr(cc, "CC_" + f))[:, J, I] for name, f in FIELDS5}
        m.step(steps - ostep)
        fields[tag] = {name: m.download(0, getattr(cc, "CC_" + f)) for name, f in FIELDS5}
        nf = m.diagnostics(0, check=False)["nonfinite"]
        m.close()
        if nf:
            fields[tag] = None
    gpu_s = time.perf_counter() - t0
    try:
        ref = q.get(timeout=1800.0)
    except _queue.Empty:
        ref = None
    proc.join(timeout=10.0)
    if proc.is_alive():
        proc.terminate()
        proc.join()

    def rel(a, b):
        den = float(np.sqrt(np.sum(b * b)))
        sc = float(np.abs(b).max())
        return {"rel_l2": float(np.sqrt(np.sum((a - b) ** 2))) / den if den > 0 else float(np.abs(a).max()),
                "rel_linf": float(np.abs(a - b).max()) / sc if sc > 0 else float(np.abs(a).max())}
    out = {"workload": cfg.name, "cells": cfg.cells, "steps": steps, "gpu_seconds": round(gpu_s, 1)}
    if fields["fp32"] is not None and fields["fp64"] is not None:
        out["fp32_vs_fp64_gpu"] = {name: rel(fields["fp32"][name], fields["fp64"][name]) for name, _ in FIELDS5}
    else:
        out["fp32_vs_fp64_gpu"] = None
    if ref is not None:
        out["vs_oracle"] = {"after_steps": ostep, "columns": int(len(J)),
                            "fp32": {n: rel(early["fp32"][n], ref[n]) for n, _ in FIELDS5},
                            "fp64": {n: rel(early["fp64"][n], ref[n]) for n, _ in FIELDS5}}
    else:
        out["vs_oracle"] = None
    return out


def bench_inflow(cc):
    """The open defect of the refined runs (Sec 3.2 set-up): the 1 km
    hemisphere on the paper's 64 x 32 x 16 km domain at 400 m with a 200 m box
    (and a 100 m box), FP32, one hour; the largest |w| below 3.2 km in the 6 km
    behind each fine level's inflow face at 1,200, 2,400 and 3,600 s, and the
    uniform 200 m run's at the same points."""
    base = W.RunConfig("hemisphere-400m", 160, 80, 40, 400.0, 400.0, 400.0, 0.3, 1, "hemisphere", 1000.0, 1000.0,
                       theta0=300.0)
    regions = {1: (16000.0, 22000.0, 8000.0, 24000.0), 2: (24000.0, 30000.0, 12000.0, 20000.0)}

    def max_w(w, dx, dz, ox, oy, reg):
        xa, xb, ya, yb = reg
        nk, ny, nx = w.shape
        X, Y, Z = ox + np.arange(nx) * dx, oy + np.arange(ny) * dx, np.arange(nk) * dz
        return float(np.abs(w[np.ix_(Z < 3200.0, (Y >= ya) & (Y <= yb), (X >= xa) & (X < xb))]).max())
    out = {}
    for nbox in (1, 2):
        boxes = [(160, 80, 40, 80, 40)] * nbox
        rc = W.RefinedConfig("paper-domain", base, boxes)
        m = cc.RefinedModel(base, boxes, cc.CC_FP32)
        for l, c in enumerate(m.cfgs):
            m.set_terrain(l, rc.finest_heights() if l == m.nlev - 1 else np.zeros((c.ny, c.nx)))
        m.build_geometry()
        m.init_state()
        rec = {}
        for T in (1200, 2400, 3600):
            m.step(4000)
            rec[T] = [round(max_w(m.derived(l, cc.CC_W), m.cfgs[l].dx, m.cfgs[l].dz, *rc.level_origin(l), regions[l]), 4)
                      for l in range(1, m.nlev)]
        m.close()
        out[f"{nbox + 1}_levels"] = rec
    u = base.replace(nx=320, ny=160, nz=80, dx=200.0, dy=200.0, dz=200.0, dt=0.15)
    m = cc.Model([u], cc.CC_FP32)
    m.set_terrain(0, u.heights())
    m.build_geometry()
    m.init_state()
    rec = {}
    for T in (1200, 2400, 3600):
        m.step(8000)
        w = m.derived(0, cc.CC_W)
        rec[T] = [round(max_w(w, 200.0, 200.0, 0.0, 0.0, regions[l]), 4) for l in (1, 2)]
    m.close()
    out["uniform_200m"] = rec
    out["how"] = ("largest |w| (m/s) below 3.2 km in the 6 km behind the inflow face of each fine level "
                  "(200 m level, then 100 m box), at 1200 / 2400 / 3600 s; uniform_200m: the same regions of the "
                  "uniform 200 m run")
    return out


def make_refined(cc, rc, prec):
    m = cc.RefinedModel(rc.base, rc.boxes, prec, xcuts=rc.xcuts, ycuts=rc.ycuts)
    for l in range(m.nlev):
        if l == m.nlev - 1:
            m.set_level_terrain(l, rc.finest_heights())
        else:
            c = m.cfgs[l]
            m.set_terrain(l, np.zeros((c.ny, c.nx)))
    m.build_geometry()
    m.init_state()
    m.autotune(3)
    return m


def refined_cell_updates(model):
    """Cell updates of one cycle of level 0: the fluid cells of level l that
    the next finer level does not cover, times its 2^l substeps (the covered
    cells are computed too, but the finer level's values stand for them)."""
    n = 0
    for d in range(model.ndom):
        l = model.blocks[d][0]
        fluid = model.geometry(d)["cls"] != 0
        if l + 1 < model.nlev:
            nx, ny, nz, ox, oy = model.boxes[l]
            fluid[:nz // 2, oy // 2:(oy + ny) // 2, ox // 2:(ox + nx) // 2] = False
        n += int(fluid.sum()) * 2 ** l
    return n


def refined_kfull_bytes(model, dtype):
    """Algorithmic bytes of the full-cell stencil over one cycle (interior
    cells of every level times its substeps)."""
    return sum(BYTES_PER_CELL[dtype] * c.nx * c.ny * c.nz * 2 ** model.blocks[d][0] for d, c in enumerate(model.cfgs))


def bench_refined(cc, torch, args, hbm, peak_kind, barrier, world, rc=None, fp64=True):
    """The refined workload: FP32 cycles timed on the device, k_full roofline
    over all levels, the plain FP64 form and the FP32 error against it (the
    finest level cut into sibling blocks when rc has cuts)."""
    rc = W.C4_REFINED if rc is None else rc
    m = make_refined(cc, rc, cc.CC_FP32)
    upd = refined_cell_updates(m)
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    barrier()
    m.profile(True)
    m.profile_reset()
    clocks.start()
    ms, launches = time_steps(torch, m, args.steps, args.warmup)
    clk = clocks.stop()
    barrier()
    kms, kn = m.profile_read(cc.CC_K_FULL)
    stages = {cc.KERNEL_NAMES[k]: dict(zip(("ms_total", "launches"), m.profile_read(k))) for k in cc.KERNEL_NAMES}
    m.profile(False)
    gms = time_graphs(torch, m, args.steps)
    # per launch, averaged over the launches of a cycle (the profiled launches
    # include the warm-up cycles): one k_full launch per level and substep
    per_cycle = sum(2 ** l for l in range(m.nlev))
    kavg = kms / max(1, kn)
    # algorithmic bytes: the cell updates the metric counts (fluid cells no
    # finer level covers, times the substeps); the stencil also computes the
    # covered and underground cells of its boxes (frac_computed)
    achieved = BYTES_PER_CELL["f32"] * upd / per_cycle / (kavg / 1e3) / 1e9
    computed = refined_kfull_bytes(m, "f32") / per_cycle / (kavg / 1e3) / 1e9
    # per level: tile height, items per launch, warp roles
    schedules = [list(m.schedule(m.level_domains(l)[0])) + [m.warp_roles(m.level_domains(l)[0])]
                 for l in range(m.nlev)]
    out = {"workload": rc.name, "levels": [list(b) for b in rc.boxes], "value": upd * args.steps * world / (ms / 1e3),
           "schedule": schedules,
           "unit": METRIC, "ms_per_step": ms / args.steps, "cell_updates_per_step": upd, "dtype": "f32",
           "gpu_launches": launches, "clocks": clk, "stages": stages,
           "graphs": {"ms_per_step": gms, "value": upd * world / (gms / 1e3), "unit": METRIC,
                      "how": "the same cycles replayed from CUDA graphs, no per-stage events"},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                        "traffic": refined_kfull_traffic("f32", rc.name, schedules),
                        "traffic_unit": "bytes per launch, averaged over a cycle",
                        "kernel": "k_full", "kernel_ms": kavg, "launches": kn,
                        "peak_kind": f"{peak_kind} hbm_gbs",
                        "bytes_per_cell": BYTES_PER_CELL["f32"], "frac_computed": computed / hbm,
                        "how": "80 B per cell update of a cycle (uncovered fluid cells of every level times its "
                               "substeps), per launch averaged over the cycle's launches"}}
    if rc.xcuts or rc.ycuts:
        out["blocks"] = {"xcuts": list(rc.xcuts), "ycuts": list(rc.ycuts), "finest_level_blocks": len(m.level_domains(m.nlev - 1)),
                         "how": "the 50 m level as sibling blocks of uneven sizes, each with its own ghost shell filled "
                                "by same-level copies after every step; all blocks in one launch per stage"}
    if fp64 and not args.no_fp64:
        m64 = make_refined(cc, rc, cc.CC_FP64)
        ks = max(2, min(args.steps, 5))
        m64.step(args.warmup)
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        m64.step(ks)
        e1.record(st)
        e1.synchronize()
        ms64 = e0.elapsed_time(e1)
        n32 = int(m.diagnostics(0, check=False)["steps"])  # steps the FP32 model has taken
        m64.step(n32 - args.warmup - ks)
        errs = {}
        for fname, f in (("rho'", cc.CC_RHOP), ("p'", cc.CC_PP), ("rho u", cc.CC_MX), ("rho v", cc.CC_MY),
                         ("rho w", cc.CC_MZ)):
            num = den = linf = scale = 0.0
            for l in range(m.ndom):
                a, b = m.download(l, f), m64.download(l, f)
                num += float(((a - b) ** 2).sum())
                den += float((b ** 2).sum())
                linf = max(linf, float(np.abs(a - b).max()))
                scale = max(scale, float(np.abs(b).max()))
            errs[fname] = {"rel_l2": (num / den) ** 0.5 if den > 0 else 0.0,
                           "rel_linf": linf / scale if scale > 0 else 0.0}
        out["fp64_plain"] = {"value": upd * ks / (ms64 / 1e3), "unit": METRIC, "dtype": "f64",
                             "ms_per_step": ms64 / ks, "steps": ks}
        out["l2_error"] = {"vs": "plain FP64 GPU form", "after_steps": n32, "fields": errs}
        m64.close()
    m.close()
    return out


def cpu_baseline_refined(seconds):
    """The FP64 oracle's refinement driver as it stands, on a bounded sample:
    the three-level 32x32x16 hemisphere (400/200/100 m), cycles of level 0
    until about `seconds` of CPU work."""
    import oracle
    rc = W.SMALL_REFINED
    R = oracle.Refine(rc.base, rc.boxes, rc.finest_heights(pad=4))
    upd = 0
    for l, lev in enumerate(R.levels):
        fluid = lev.geometry()["cls"] != 0
        if l + 1 < len(R.levels):
            nx, ny, nz, ox, oy = rc.boxes[l]
            fluid[:nz // 2, oy // 2:(oy + ny) // 2, ox // 2:(ox + nx) // 2] = False
        upd += int(fluid.sum()) * 2 ** l
    R.init_state()
    R.step(1)
    s = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds and s < 200:
        R.step(1)
        s += 1
    dt = time.perf_counter() - t0
    return {"value": upd * s / dt, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"{rc.name} x {s} cycles ({dt:.1f} s, single-threaded FP64 oracle)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    # each step: a bounded sample of the workload on the oracle
    per = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    vals = []
    if args.workload == "refined":
        name, ninst = W.C4_REFINED.name, 1
        for s in range(args.warmup + args.steps):
            r = cpu_baseline_refined(per)
            if s >= args.warmup:
                vals.append(r)
    else:
        name, cfgs = workload_configs(args)
        ninst = len(cfgs)
        for s in range(args.warmup + args.steps):
            r = cpu_baseline(cfgs[s % len(cfgs):] + cfgs[:s % len(cfgs)], per)
            if s >= args.warmup:
                vals.append(r)
    v = statistics.median(x["value"] for x in vals)
    line = {"metric": METRIC, "value": v, "unit": METRIC, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "instances": ninst},
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": 1, "kind": "oracle",
                             "sample": vals[-1]["sample"]},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_convergence(cc, torch, args):
    """The appendix accuracy experiment on the paper's domain: flow over the
    cosine hill (h_m = 400 m, a = 2 km, centred at (32, 16) km) on a periodic
    64 x 32 x 16 km domain with equal spacing 400, 250, 200 and 100 m, U = 10
    m/s, N = 0.01 1/s, Theta = 300 K, sponge above 10 km, FP32, for the same
    simulated time; the L1 and L2 errors of u and w above the hill top against
    the 100 m run, at the corners the grids share, and the orders between
    successive spacings. One JSON line."""
    h0, a = 400.0, 2000.0
    res = [100.0, 400.0, 250.0, 200.0]  # the reference run first

    def run(d):
        nx, ny, nz = int(round(64000 / d)), int(round(32000 / d)), int(round(16000 / d))
        cfg = W.RunConfig(f"cosine-{d:g}m", nx, ny, nz, d, d, d, 0.15 * d / 200.0, 1, "cosine", h0, a,
                          theta0=300.0)
        m = cc.Model([cfg], cc.CC_FP32)
        m.set_terrain_analytic(0, "cosine", h0, a)
        m.build_geometry()
        m.init_state()
        n = int(round(args.seconds / cfg.dt))
        t0 = time.perf_counter()
        m.step(n)
        m.synchronize()
        dg = m.diagnostics(0)
        return m, cfg, n, time.perf_counter() - t0, dg

    fine, fcfg, fn, fsec, fdg = run(res[0])
    runs = {res[0]: {"grid": [fcfg.nx, fcfg.ny, fcfg.nz], "steps": fn, "wall_s": round(fsec, 2),
                     "max_w": fdg["max_w"]}}
    for d in res[1:]:
        m, cfg, n, sec, dg = run(d)
        e = {"grid": [cfg.nx, cfg.ny, cfg.nz], "steps": n, "wall_s": round(sec, 2), "max_w": dg["max_w"]}
        for nm, w in (("u", cc.CC_U), ("w", cc.CC_W)):
            l1, l2, cnt = cc.error_norms(m, 0, fine, 0, w, h0)
            e[nm] = {"L1": l1, "L2": l2, "points": cnt}
        runs[d] = e
        m.close()
    fine.close()
    coarse = sorted(res[1:], reverse=True)
    orders = {}
    for nm in ("u", "w"):
        for norm in ("L1", "L2"):
            orders[f"{nm}_{norm}"] = [math.log(runs[x][nm][norm] / runs[y][nm][norm]) / math.log(x / y)
                                      for x, y in zip(coarse, coarse[1:])]
    line = {"metric": "global error of u and w against the 100 m run (L1, L2)", "unit": "m/s",
            "workload": "convergence-cosine-64x32x16km", "seconds": args.seconds, "dtype": "f32",
            "data": "synthetic", "n_gpus": 1, "zmin": h0,
            "runs": {f"{k:g}m": v for k, v in runs.items()}, "orders": orders,
            "how": "orders between successive spacings 400-250-200 m, log(e1/e2)/log(d1/d2); the paper's "
                   "appendix reports second order"}
    print(json.dumps(line), flush=True)


def run_refined_vs_uniform(cc, torch, args):
    """The paper's refined-grid test (Sec 3.2) with nested boxes in place of
    its cube sets: flow over the 1 km hemisphere on the 64 x 32 x 16 km domain
    (Theta = 300 K) for the same simulated time on a uniform 400 m grid, with
    a 200 m box (x 16-48 km, y 8-24 km, z 0-8 km), and with a further 100 m
    box (x 24-40 km, y 12-20 km, z 0-4 km); each against a uniform 100 m run.
    The root-mean-square difference of w at z = 1200 m is taken at the points
    of the 400 m lattice, from the finest level covering each point, in three
    regions: inside the 100 m box, inside the 200 m box only, and outside
    both (1 km margins). One JSON line."""
    base = W.RunConfig("hemisphere-400m", 160, 80, 40, 400.0, 400.0, 400.0, 0.3, 1, "hemisphere", 1000.0, 1000.0,
                       theta0=300.0)
    box1, box2 = (160, 80, 40, 80, 40), (160, 80, 40, 80, 40)
    z = 1200.0
    t0 = time.perf_counter()

    def finish(m, n):
        m.step(n)
        m.synchronize()

    # the uniform runs
    def uniform(d):
        cfg = base.replace(name=f"hemisphere-{d:g}m", nx=int(64000 / d), ny=int(32000 / d), nz=int(16000 / d),
                           dx=d, dy=d, dz=d, dt=0.15 * d / 200.0)
        m = cc.Model([cfg], cc.CC_FP32)
        m.set_terrain(0, cfg.heights())
        m.build_geometry()
        m.init_state()
        finish(m, int(round(args.seconds / cfg.dt)))
        w = m.derived(0, cc.CC_W)[int(round(z / d))]
        m.close()
        return w

    ref = uniform(100.0)
    lat = {"400m": [(0.0, 0.0, 400.0, uniform(400.0))]}  # (origin x, origin y, spacing, w plane) finest last
    for name, boxes in (("400/200m", [box1]), ("400/200/100m", [box1, box2])):
        rc = W.RefinedConfig(name, base, boxes)
        m = cc.RefinedModel(base, boxes, cc.CC_FP32)
        for l, c in enumerate(m.cfgs):
            m.set_terrain(l, rc.finest_heights() if l == m.nlev - 1 else np.zeros((c.ny, c.nx)))
        m.build_geometry()
        m.init_state()
        finish(m, int(round(args.seconds / base.dt)))
        planes = []
        for l, c in enumerate(m.cfgs):
            ox, oy = rc.level_origin(l)
            planes.append((ox, oy, c.dx, m.derived(l, cc.CC_W)[int(round(z / c.dx))]))
        lat[name] = planes
        m.close()

    def value(planes, x, y):
        """w at (x, y) from the finest level whose interior holds the point."""
        for ox, oy, d, w in reversed(planes):
            i, j = (x - ox) / d, (y - oy) / d
            if 0 <= i < w.shape[1] and 0 <= j < w.shape[0] and abs(i - round(i)) < 1e-9:
                return float(w[int(round(j)), int(round(i))])
        raise AssertionError((x, y))

    def region(x, y):
        if 25000 <= x <= 39000 and 13000 <= y <= 19000:
            return "inside the 100 m box"
        if 17000 <= x <= 47000 and 9000 <= y <= 23000 and not (23000 <= x <= 41000 and 11000 <= y <= 21000):
            return "inside the 200 m box only"
        if x < 15000 or x > 49000 or y < 7000 or y > 25000:
            return "outside both boxes"
        return None

    acc = {}
    for b in range(80):
        for a in range(160):
            x, y = 400.0 * a, 400.0 * b
            r = region(x, y)
            if r is None:
                continue
            wr = float(ref[4 * b, 4 * a])
            for name, planes in lat.items():
                e = acc.setdefault(r, {}).setdefault(name, [0.0, 0])
                e[0] += (value(planes, x, y) - wr) ** 2
                e[1] += 1
    out = {r: {name: {"rms": math.sqrt(v[0] / v[1]), "points": v[1]} for name, v in d.items()}
           for r, d in acc.items()}
    line = {"metric": "rms difference of w at z = 1200 m from the uniform 100 m run", "unit": "m/s",
            "workload": "refined-vs-uniform-hemisphere-64x32x16km", "seconds": args.seconds, "dtype": "f32",
            "data": "synthetic", "n_gpus": 1, "regions": out, "wall_s": round(time.perf_counter() - t0, 1),
            "how": "grids 400 m; 400 m + 200 m box; 400 m + 200 m + 100 m boxes (nested boxes standing for the "
                   "paper's cube sets); w at the 400 m lattice points, from the finest level holding each point"}
    print(json.dumps(line), flush=True)


def main():
    global SCHEDULE
    args = parse()
    if args.schedule:
        SCHEDULE = tuple(int(x) for x in args.schedule.split(","))
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1509_02572_gb300 import build as B
    B.build()
    from paper_1509_02572_gb300 import cutcell as cc

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    hbm, peak_kind = peaks()
    if args.workload in ("convergence", "refined-vs-uniform"):
        if rank == 0:
            (run_convergence if args.workload == "convergence" else run_refined_vs_uniform)(cc, torch, args)
        if world > 1:
            dist.destroy_process_group()
        return
    if args.workload in ("refined", "refined-blocks"):
        r = bench_refined(cc, torch, args, hbm, peak_kind, barrier, world,
                          rc=W.C4_BLOCKED if args.workload == "refined-blocks" else W.C4_REFINED)
        msps, rate = job_time_and_rate(r["ms_per_step"], r["cell_updates_per_step"], world, dist)
        line = {"metric": METRIC, "value": rate, "unit": METRIC,
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": msps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": r["workload"], "levels": r["levels"], "schedule": r["schedule"],
                           **({"blocks": r["blocks"]} if "blocks" in r else {}),
                           "cell_updates_per_step": r["cell_updates_per_step"],
                           "precision": "fp32 perturbations, fp64 geometry and base state",
                           "l2": "inputs larger than L2 (state of all levels)"},
                "gpu_launches": r["gpu_launches"], "roofline": r["roofline"], "stages": r["stages"],
                "clocks": r["clocks"]}
        for k in ("fp64_plain", "l2_error", "graphs"):
            if k in r:
                line[k] = r[k]
        if rank == 0 and world == 1 and not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline_refined(args.cpu_seconds)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    name, cfgs = workload_configs(args)
    prec_main = cc.CC_FP64 if args.workload == "hemisphere" else cc.CC_FP32
    dtype = "f32" if prec_main == cc.CC_FP32 else "f64"
    model = make_model(cc, cfgs, prec_main)
    nfluid = fluid_cells(model, cfgs)
    ninterior = sum(c.cells for c in cfgs)

    # ---- timed region (device time, CUDA events on the model's stream)
    clocks = Clocks(local)
    barrier()
    model.profile(True)
    model.profile_reset()
    clocks.start()
    ms, launches = time_steps(torch, model, args.steps, args.warmup)
    clk = clocks.stop()
    barrier()
    kfull_ms, kfull_n = model.profile_read(cc.CC_K_FULL)
    stage = {cc.KERNEL_NAMES[k]: model.profile_read(k) for k in cc.KERNEL_NAMES}
    model.profile(False)
    gms = time_graphs(torch, model, args.steps)
    ms, value = job_time_and_rate(ms, nfluid * args.steps, world, dist)

    kavg = kfull_ms / max(1, kfull_n)
    # algorithmic bytes: the fluid cells the metric counts (the stencil also
    # runs over the underground cells of its tiles: frac_computed)
    achieved = BYTES_PER_CELL[dtype] * nfluid / (kavg / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": kfull_traffic(dtype, ninterior, model.schedule(0), model.warp_roles(0)),
            "traffic_unit": "bytes per launch",
            "kernel": "k_full", "kernel_ms": kavg, "peak_kind": f"{peak_kind} hbm_gbs",
            "bytes_per_cell": BYTES_PER_CELL[dtype], "cells_per_launch": nfluid,
            "frac_computed": BYTES_PER_CELL[dtype] * ninterior / (kavg / 1e3) / 1e9 / hbm,
            "how": "80 B (FP32) per fluid cell of the step / the stencil's mean launch time (CUDA events)"}
    stages = {k: {"ms_total": v[0], "launches": v[1]} for k, v in stage.items()}
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": name, "instances": len(cfgs), "interior_cells": ninterior,
                       "schedule": list(model.schedule(0)), "warp_roles": model.warp_roles(0),
                       "fluid_cells": nfluid, "precision": ("fp32 perturbations, fp64 geometry and base state"
                                                            if dtype == "f32" else "fp64"),
                       "l2": "inputs larger than L2 (state of all domains)" if ninterior * 80 > 129e6 else
                       "working set may fit in L2"},
            "gpu_launches": launches, "roofline": roof, "stages": stages, "clocks": clk,
            "graphs": {"ms_per_step": gms, "value": nfluid * world / (gms / 1e3), "unit": METRIC,
                       "how": "the same steps replayed from CUDA graphs, no per-stage events"}}

    # ---- plain FP64 form on the same workload, one domain at a time
    if not args.no_fp64 and prec_main == cc.CC_FP32:
        singles = [make_model(cc, [c], cc.CC_FP64) for c in cfgs]
        ksteps = max(2, min(args.steps, 5))
        for s in singles:
            s.step(args.warmup)
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(ksteps):
            for s in singles:
                s.step(1)
        e1.record(st)
        e1.synchronize()
        ms64 = e0.elapsed_time(e1)
        v64 = nfluid * ksteps / (ms64 / 1e3)
        # error of the FP32 batched state against the FP64 runs after the same
        # number of steps (both started from the same initial state)
        if args.error_steps > 0:
            model.step(args.error_steps)
        n32 = int(model.diagnostics(0, check=False)["steps"])  # steps the FP32 model has taken
        n64 = args.warmup + ksteps
        for s in singles:
            s.step(n32 - n64)
        errs = {}
        for fname, f in (("rho'", cc.CC_RHOP), ("p'", cc.CC_PP), ("rho u", cc.CC_MX), ("rho v", cc.CC_MY),
                         ("rho w", cc.CC_MZ)):
            num = den = 0.0
            linf = scale = 0.0
            for d, s in enumerate(singles):
                a = model.download(d, f)
                b = s.download(0, f)
                num += float(((a - b) ** 2).sum())
                den += float((b ** 2).sum())
                linf = max(linf, float(np.abs(a - b).max()))
                scale = max(scale, float(np.abs(b).max()))
            errs[fname] = {"rel_l2": (num / den) ** 0.5 if den > 0 else 0.0,
                           "rel_linf": linf / scale if scale > 0 else 0.0}
        line["fp64_plain"] = {"value": v64, "unit": METRIC, "dtype": "f64", "ms_per_step": ms64 / ksteps,
                              "steps": ksteps, "how": "each domain stepped alone in FP64, looped over domains"}
        # its roofline: the FP64 pipe, not HBM, bounds it (160 B per cell at
        # 1e9 cells/s is a few per cent of HBM); per-launch time of its
        # full-cell stencil from events on one profiled step of every domain
        for s in singles:
            s.profile(True)
            s.profile_reset()
        for s in singles:
            s.step(1)
        torch.cuda.synchronize()
        k64_ms = sum(s.profile_read(cc.CC_K_FULL)[0] for s in singles)
        for s in singles:
            s.profile(False)
        peak64 = cc.fma_peak(cc.CC_FP64)
        per = [fp64_flops_per_cell(s.schedule(0)[0]) for s in singles]
        fpc = None if any(x is None for x in per) else sum(x * c.cells for x, c in zip(per, cfgs)) / ninterior
        ach64 = None if fpc is None else fpc * ninterior / (k64_ms / 1e3)
        line["fp64_plain"]["roofline"] = {
            "bound": "alu", "achieved": None if ach64 is None else ach64 / 1e12, "peak": peak64 / 1e12,
            "unit": "TFLOP/s", "frac": None if ach64 is None else ach64 / peak64, "kernel": "k_full (FP64)",
            "kernel_ms_per_step": k64_ms, "flops_per_cell": fpc,
            "peak_kind": "measured FP64 fused multiply-add rate (cc_fma_peak, this run)",
            "how": "executed FP64 flops per interior cell (ncu: 2 dfma + dadd + dmul, profiles/"
                   "k_full_fp64_flops.json) x interior cells / the stencil's event time over one step"}
        line["l2_error"] = {"vs": "plain FP64 GPU form", "after_steps": n32, "fields": errs}
        for s in singles:
            s.close()

    # ---- end to end through the C ABI with host buffers
    if not args.no_e2e:
        fields = (cc.CC_RHOP, cc.CC_PP, cc.CC_MX, cc.CC_MY, cc.CC_MZ)

        def e2e_run(f32):
            """Pinned host buffers in FP32 (the model's own precision, copied
            unchanged) or FP64; per step: upload, one step, download p'."""
            np_dt, t_dt, es = (np.float32, torch.float32, 4) if f32 else (np.float64, torch.float64, 8)
            # the whole state in one pinned buffer, in the order of cc_upload_all_*
            host = torch.from_numpy(np.concatenate([model.download(d, f, lev, dtype=np_dt).ravel()
                                                    for d in range(len(cfgs)) for f in fields
                                                    for lev in (0, 1)])).pin_memory()
            assert host.numel() == model.state_elems()
            outs = [torch.empty(tuple(model._shape(d, cc.CC_PP)), dtype=t_dt).pin_memory() for d in range(len(cfgs))]
            h2d = host.numel() * es
            d2h = sum(o.numel() * es for o in outs)
            # as many steps as the device-timed loop (up to 24): the host link
            # shows rare one-off stalls of 50-120 ms, which a short window
            # would over- or under-weight
            ke = max(3, min(args.steps, 24))

            def e2e_step():
                model.upload_all_ptr(host.data_ptr(), f32=f32)
                model.step(1)
                for d in range(len(cfgs)):
                    model.download_ptr(d, cc.CC_PP, 1, outs[d].data_ptr(), wait=False, f32=f32)
                model.synchronize()  # the step's result is on the host

            for _ in range(max(1, min(args.warmup, 3))):  # untimed, as for the device-timed steps
                e2e_step()
            gc.collect()
            gc.disable()  # no collection pause inside the timed host loop
            barrier()
            t0 = time.perf_counter()
            iter_ms = []
            for _ in range(ke):
                ti = time.perf_counter()
                e2e_step()
                iter_ms.append(round(1e3 * (time.perf_counter() - ti), 2))
            barrier()
            te = time.perf_counter() - t0
            gc.enable()
            del host, outs
            gc.collect()
            return {"value": nfluid * ke * world / te, "unit": METRIC, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": ke, "iter_ms": iter_ms}

        f32 = prec_main == cc.CC_FP32
        line["e2e"] = e2e_run(f32)
        line["e2e"]["how"] = ("per step: upload both time levels of every prognostic field of every domain from "
                              "one pinned host buffer (cc_upload_all_*, one copy per domain) in "
                              + ("FP32 (the model's precision, copied unchanged)" if f32 else "FP64")
                              + ", one step, download p' of every domain, then wait for it (transfers queued on "
                                "the model's stream, one host wait per step); untimed warm-up steps first")
        if f32:
            r = e2e_run(False)
            line["e2e"]["fp64_host"] = {k: r[k] for k in ("value", "h2d_bytes_per_step", "d2h_bytes_per_step",
                                                          "iter_ms")}

    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(cfgs, args.cpu_seconds)
        line["cpu_baseline"]["all_cores"] = cpu_baseline_allcores(cfgs, args.cpu_seconds)
    model.close()
    if args.workload == "ensemble" and not args.no_precision and rank == 0 and world == 1:
        line["precision"] = bench_precision(cc, torch, args.precision_steps)
    if args.workload == "ensemble" and not args.no_refined:
        line["refined"] = bench_refined(cc, torch, args, hbm, peak_kind, barrier, world)
        if rank == 0 and world == 1:
            line["refined"]["inflow_face_w"] = bench_inflow(cc)
        line["refined_blocks"] = bench_refined(cc, torch, args, hbm, peak_kind, barrier, world, rc=W.C4_BLOCKED,
                                               fp64=False)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
