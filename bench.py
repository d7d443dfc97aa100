"""Throughput of the free-surface LBM step on GB300: MLUPS and HBM-roofline
fraction of the bulk stream-collide kernel, FP32 / FP16-shifted storage next
to the plain FP64 path, on the 768 x 384 x 256 wave tank with 16 free boxes.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

One JSON line on stdout (rank 0).  'value' is the FP32-storage MLUPS (all
cells, whole job); the FP16 and FP64 runs of the same workload are reported
under 'variants'.
"""
from __future__ import annotations

import argparse
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

METRIC = "MLUPS & % of HBM roofline, FP32/FP16-stored vs FP64 plain at stated error"
BYTES_PER_FLUID = {"f64": 38 * 8, "f32": 38 * 4, "f16s": 80}
C_BODY_BYTES = 8 * (3 + 3 + 1 + 3 + 4 + 3 + 3)  # one lbm_fs_body_state_t
DTYPE = {"f64": "f64", "f32": "f32", "f16s": "f16s/f32"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


def strip_comments(src: str) -> str:
    """C/C++ source without its comments, trailing blanks and empty lines
    (string and character literals are kept as they are)."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            while i < n and src[i] != "\n":
                i += 1
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    lines = (line.rstrip() for line in "".join(out).split("\n"))
    return "\n".join(line for line in lines if line)


def kernel_source_hash() -> str:
    """sha256 of the kernel sources without their comments, to tie a stored
    ncu capture to the code."""
    import hashlib

    h = hashlib.sha256()
    for f in ("lbmfs_kernels.cuh", "lbmfs_internal.h"):
        with open(os.path.join(ROOT, "paper_1201_0351_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(strip_comments(fh.read()).encode("utf-8"))
    return h.hexdigest()


def stored_traffic(storage: str, algorithmic_bytes: float):
    """DRAM bytes per launch of the bulk kernel, scaled from the committed ncu
    capture of a smaller case of the same kernel (traffic grows in proportion
    to the liquid cells); None when the kernel sources changed since."""
    try:
        with open(os.path.join(ROOT, "profiles", "k_liquid_traffic.json")) as fh:
            rec = json.load(fh)
    except Exception:
        return None
    r = rec.get(storage)
    if not r or rec.get("kernel_source_sha256") != kernel_source_hash():
        return None
    return r["dram_bytes"] / r["algorithmic_bytes"] * algorithmic_bytes


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.out,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        self.out.flush()
        rows = []
        try:
            with open(self.out.name) as fh:
                for line in fh:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def fluid_counts(sim):
    f = sim.fields()
    fl = f["flags"]
    return int(((fl == 1) | (fl == 2)).sum()), int((fl == 1).sum()), int((fl == 2).sum())


def whole_job(ms_local: float, cells: int, steps: int, world: int, device: str = "cpu"):
    """Replicas (one tank per rank, no data-path collective): the job's time is
    the slowest rank's, and the job's throughput counts every rank's cells.
    Returns (max milliseconds over ranks, whole-job MLUPS)."""
    ms = ms_local
    if world > 1:
        import torch
        import torch.distributed as dist

        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * cells * steps / (ms * 1e-3) / 1e6


def stored_fp64_ops():
    """Double-precision operations per liquid cell of the double-storage bulk
    kernel, from the committed ncu capture; None when the kernel sources
    changed since."""
    try:
        with open(os.path.join(ROOT, "profiles", "k_liquid_traffic.json")) as fh:
            rec = json.load(fh)
    except Exception:
        return None
    r = rec.get("f64")
    if not r or rec.get("kernel_source_sha256") != kernel_source_hash() or "dp_ops_per_liquid_cell" not in r:
        return None
    return r["dp_ops_per_liquid_cell"]


def run_storage(sc, storage, steps, warmup, kernel_steps, clocks=None, barrier=None, late=(0, 0)):
    """Time `steps` steps after `warmup`; with late = (advance, k), also k
    steps after advancing `advance` more (a window later in the job, when the
    bodies move and the surface has folded)."""
    import torch

    from paper_1201_0351_gb300 import lbm_fs

    sim = lbm_fs.Simulation(sc, storage=storage, use_graphs=True)
    sim.step(warmup)
    sim.sync()
    n_fluid0, n_liq0, n_if0 = fluid_counts(sim)
    st0 = sim.stats()
    launches0, n_gen0 = st0["kernel_launches"], st0["n_general"]
    stream = sim.stream
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if barrier:
        barrier()
    torch.cuda.synchronize()
    ctx = clocks if clocks is not None else _Null()
    with ctx:
        start.record(stream)
        sim.step(steps)
        end.record(stream)
        end.synchronize()
    torch.cuda.synchronize()
    if barrier:
        barrier()
    ms = start.elapsed_time(end)
    st = sim.stats()
    launches = st["kernel_launches"] - launches0
    n_fluid1, n_liq1, n_if1 = fluid_counts(sim)
    late_window = None
    if late[0] > 0 and late[1] > 0:
        sim.step(late[0])
        sim.sync()
        start.record(stream)
        sim.step(late[1])
        end.record(stream)
        end.synchronize()
        ml = start.elapsed_time(end)
        n_all = sc.nx * sc.ny * sc.nz
        late_window = dict(after_steps=warmup + steps + late[0], steps=late[1], ms_per_step=ml / late[1],
                           mlups=n_all * late[1] / (ml * 1e-3) / 1e6, status=sim.stats()["status"])
    kt = sim.kernel_times(kernel_steps)
    sim.close()
    del sim
    torch.cuda.empty_cache()
    n = sc.nx * sc.ny * sc.nz
    n_liq = 0.5 * (n_liq0 + n_liq1)
    n_if = 0.5 * (n_if0 + n_if1)
    n_gen = 0.5 * (n_gen0 + st["n_general"])  # liquid cells stepped by the general-gather kernel
    b_fluid = BYTES_PER_FLUID[storage]
    # one flag byte per fluid cell (tiles of gas above the fluid are never read)
    step_bytes = (n_liq + n_if) * (b_fluid + 1) + n_if * 24
    liquid_bytes = (n_liq - n_gen) * b_fluid + (n_liq + n_if) * 1
    total_k = sum(kt.values())
    return dict(storage=storage, ms_total=ms, ms_per_step=ms / steps, mlups=n * steps / (ms * 1e-3) / 1e6,
                fluid_mlups=(n_liq + n_if) * steps / (ms * 1e-3) / 1e6, step_gbs=step_bytes / (ms / steps * 1e-3) / 1e9,
                liquid_ms=kt.get("liquid", float("nan")) / kernel_steps, liquid_bytes=liquid_bytes,
                liquid_gbs=liquid_bytes / (kt.get("liquid", float("nan")) / kernel_steps * 1e-3) / 1e9,
                kernel_share={k: v / total_k for k, v in kt.items() if total_k > 0},
                launches=launches, status=st["status"], n_fluid=(n_liq + n_if), n_interface=n_if, n_liquid=n_liq,
                n_general=n_gen, late_window=late_window,
                mass_resid=(st["liquid_mass"] - st["mass0"] - (st["uncovered"] - st["covered"] - st["lost_excess"]
                                                               + st["wall_source"])) / st["mass0"])


def run_batch(scenes, storage, steps, warmup, kernel_steps, separate_steps=20, barrier=None):
    """The batched form on many tanks (one launch per kernel for all tanks):
    autotuned tiling, CUDA-event time of `steps` steps on the batch's stream,
    bytes from the fluid cells of every tank; for comparison, the same tanks
    as separate handles stepped one after another on the same stream."""
    import torch

    from paper_1201_0351_gb300 import lbm_fs

    bt = lbm_fs.Batch(scenes, storage=storage, use_graphs=True)
    bt.step(warmup)
    bt.sync()
    cfg = bt.autotune()
    bt.step(2)
    bt.sync()

    def counts():
        liq = itf = gen = 0
        for t in bt.tanks:
            fl = t.flags()
            liq += int((fl == 1).sum())
            itf += int((fl == 2).sum())
            gen += int(t.stats()["n_general"])
        return liq, itf, gen

    liq0, if0, gen0 = counts()
    launches0, _ = bt.launches()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if barrier:
        barrier()
    torch.cuda.synchronize()
    start.record(bt.stream)
    bt.step(steps)
    end.record(bt.stream)
    end.synchronize()
    if barrier:
        barrier()
    ms = start.elapsed_time(end)
    launches = bt.launches()[0] - launches0
    liq1, if1, gen1 = counts()
    kt = bt.kernel_times(kernel_steps)
    bt.sync()
    cells = bt.cells
    bt.close()
    del bt
    torch.cuda.empty_cache()
    n_liq, n_if, n_gen = 0.5 * (liq0 + liq1), 0.5 * (if0 + if1), 0.5 * (gen0 + gen1)
    b_fluid = BYTES_PER_FLUID[storage]
    step_bytes = (n_liq + n_if) * (b_fluid + 1) + n_if * 24
    liquid_bytes = (n_liq - n_gen) * b_fluid + (n_liq + n_if) * 1
    liquid_ms = kt["liquid"] / kernel_steps
    # the same tanks as separate handles (each with its own captured graphs)
    ms_sep = None
    if separate_steps > 0:
        sims = [lbm_fs.Simulation(sc, storage=storage) for sc in scenes]
        for sim in sims:
            sim.step(2)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        start.record(stream)
        for _ in range(separate_steps):
            for sim in sims:
                sim.step(1)
        end.record(stream)
        end.synchronize()
        ms_sep = start.elapsed_time(end) / separate_steps
        for sim in sims:
            sim.close()
        del sims
        torch.cuda.empty_cache()
    total_k = sum(kt.values())
    return dict(storage=storage, tanks=len(scenes), cells=cells, ms_total=ms, ms_per_step=ms / steps,
                mlups=cells * steps / (ms * 1e-3) / 1e6, step_gbs=step_bytes / (ms / steps * 1e-3) / 1e9,
                liquid_ms=liquid_ms, liquid_bytes=liquid_bytes, liquid_gbs=liquid_bytes / (liquid_ms * 1e-3) / 1e9,
                kernel_share={k: v / total_k for k, v in kt.items() if total_k > 0}, launches=launches,
                autotune=cfg, separate_ms_per_step=ms_sep, mass_resid=None)


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def e2e_run(sc, storage, steps):
    """Through the public API with host buffers: create (uploads the initial
    state from pinned host arrays), then every step lbm_fs_step + lbm_fs_body_states of all
    bodies (device -> host read of the step's forces, torques and poses, as a
    host-side rigid-body coupling would do), timed on the host clock."""
    import dataclasses

    import torch

    from paper_1201_0351_gb300 import lbm_fs

    # the job's inputs (the initial state) wait in pinned host memory, filled
    # before the timed region; their host-to-device copy is timed
    pinned = {}
    for key in ("flags", "fill", "rho"):
        a = np.ascontiguousarray(getattr(sc, key))
        t = torch.empty(a.shape, dtype=torch.from_numpy(a[:1].copy()).dtype, pin_memory=True)
        t.numpy()[...] = a
        pinned[key] = t.numpy()
    sc = dataclasses.replace(sc, **pinned)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim = lbm_fs.Simulation(sc, storage=storage, use_graphs=True, host_init=True)
    states = (lbm_fs.lbm_fs_body_state_t * max(sim.nbodies, 1))()
    for _ in range(steps):
        sim.step(1)
        lbm_fs.lbm_fs_body_states(sim.h, 0, sim.nbodies, states)
    sim.sync()
    t1 = time.perf_counter()
    sim.close()
    n = sc.nx * sc.ny * sc.nz
    h2d = sc.flags.nbytes + sc.fill.nbytes + sc.rho.nbytes
    d2h = sim.nbodies * C_BODY_BYTES
    return dict(value=n * steps / (t1 - t0) / 1e6, unit="MLUPS", h2d_bytes_per_step=h2d // steps,
                d2h_bytes_per_step=d2h, steps=steps,
                covers="create from pinned host arrays, then every step lbm_fs_step + lbm_fs_body_states")


def cpu_baseline(sc_full, target_s=15.0):
    """The oracle as it stands, single-threaded, on a bounded sample of the
    workload: a 192 x 96 column window of the tank centred on its first box
    (full depth, walls on the cut), as many steps as fit in about target_s
    seconds."""
    import oracle
    from paper_1201_0351_gb300 import inputs

    wx, wy = min(192, sc_full.nx), min(96, sc_full.ny)
    b0 = sc_full.boxes[0] if sc_full.boxes else None
    x0 = 0 if b0 is None else int(min(max(b0.center[0] - wx / 2, 0), sc_full.nx - wx))
    y0 = 0 if b0 is None else int(min(max(b0.center[1] - wy / 2, 0), sc_full.ny - wy))
    sc = inputs.crop(sc_full, wx, wy, x0=x0, y0=y0)
    t0 = time.perf_counter()
    sim = oracle.OracleSim(sc)
    t_setup = time.perf_counter() - t0
    steps = 0
    t0 = time.perf_counter()
    while True:
        sim.step(1)
        steps += 1
        if time.perf_counter() - t0 > target_s or steps >= 50:
            break
    dt = time.perf_counter() - t0
    n = sc.nx * sc.ny * sc.nz
    return dict(value=n * steps / dt / 1e6, unit="MLUPS", cores=1, kind="oracle",
                sample="%dx%dx%d crop of the wave tank, %d boxes, %d steps, %.1f s (setup %.1f s)" % (
                    sc.nx, sc.ny, sc.nz, len(sc.boxes), steps, dt, t_setup))


def workload(args):
    from paper_1201_0351_gb300 import inputs

    return inputs.wave_tank(args.nx, args.ny, args.nz, nboxes=args.boxes)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nx", type=int, default=768)
    ap.add_argument("--ny", type=int, default=384)
    ap.add_argument("--nz", type=int, default=256)
    ap.add_argument("--boxes", type=int, default=16)
    ap.add_argument("--f64-steps", type=int, default=0, help="steps of the FP64 variant (default steps // 10)")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched 64-tank sweep")
    ap.add_argument("--batch-tanks", type=int, default=64, help="tanks of the batched sweep (small profiling cases)")
    ap.add_argument("--e2e-steps", type=int, default=0, help="steps of the end-to-end run (default: the workload's job length)")
    ap.add_argument("--late-advance", type=int, default=1000, help="steps run before the late timed window (0: none)")
    ap.add_argument("--late-steps", type=int, default=20, help="steps of the late timed window")
    args = ap.parse_args()
    ws, rank, local = dist_info()
    config = {"workload": "wave tank %dx%dx%d, %d free boxes 24x12x8, tau 0.52, g 1e-5" % (
        args.nx, args.ny, args.nz, args.boxes), "grid": [args.nx, args.ny, args.nz], "cells": args.nx * args.ny * args.nz,
        "l2": "inputs larger than L2 (>= 5.7 GB per population grid)", "parallelism": "replicas" if ws > 1 else "1 GPU"}

    if args.impl == "reference":
        if rank != 0:
            return 0
        sc = workload(args)
        cb = cpu_baseline(sc, target_s=max(5.0, min(60.0, 2.0 * (args.steps + args.warmup))))
        # the oracle steps a bounded sample: its time per step of the whole
        # workload follows from the measured rate
        ms_full = sc.nx * sc.ny * sc.nz / (cb["value"] * 1e6) * 1e3 if cb["value"] > 0 else None
        line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "MLUPS", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_full,
                "ms_per_step_from": "the sample's rate over the workload's cells", "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
                "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                                             "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import torch

    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        barrier = dist.barrier
    else:
        torch.cuda.set_device(0)
        barrier = None
    peaks, peak_src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    sc = workload(args)
    clocks = ClockSampler(local)
    main_run = run_storage(sc, "f32", args.steps, max(args.warmup, 3), 5, clocks=clocks, barrier=barrier,
                           late=(args.late_advance, args.late_steps))
    variants = {}
    if not args.no_variants:
        variants["f16s"] = run_storage(sc, "f16s", args.steps, max(args.warmup, 3), 5, barrier=barrier)
        f64_steps = args.f64_steps or max(3, args.steps // 10)
        variants["f64"] = run_storage(sc, "f64", f64_steps, 3, 2, barrier=barrier)
        from paper_1201_0351_gb300 import lbm_fs

        fp64_rates = {name: lbm_fs.lbm_fs_fp64_rate(op) for op, name in ((0, "fma"), (1, "add"), (2, "mul"))}
    batch = None
    if not args.no_variants and not args.no_batch:
        from paper_1201_0351_gb300 import inputs

        batch = run_batch(inputs.batched_sweep_tanks(args.batch_tanks), "f16s", args.steps, max(args.warmup, 3), 5,
                          barrier=barrier)
        # the FP32-stored batched form on the same tanks (no separate-handle comparison)
        batch32 = run_batch(inputs.batched_sweep_tanks(args.batch_tanks), "f32", args.steps, max(args.warmup, 3), 5,
                            separate_steps=0, barrier=barrier)
    n = sc.nx * sc.ny * sc.nz
    ms, value = whole_job(main_run["ms_total"], n, args.steps, ws, "cuda")
    e2e = e2e_run(sc, "f32", args.e2e_steps or sc.steps)
    e2e["value"] *= ws
    if rank != 0:
        return 0
    cb = None if args.no_cpu else cpu_baseline(sc)
    frac = main_run["liquid_gbs"] / hbm
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config,
        "roofline": {"bound": "hbm", "kernel": "k_liquid (stream + collide of liquid cells)",
                     "achieved": main_run["liquid_gbs"], "peak": hbm, "unit": "GB/s", "frac": frac,
                     "peak_source": peak_src, "traffic": stored_traffic("f32", main_run["liquid_bytes"]),
                     "algorithmic_bytes_per_launch": main_run["liquid_bytes"],
                     "step_achieved_gbs": main_run["step_gbs"], "step_frac": main_run["step_gbs"] / hbm},
        "cpu_baseline": cb, "e2e": e2e, "gpu_launches": main_run["launches"], "clocks": clocks.summary(),
        "fluid_mlups": main_run["fluid_mlups"], "kernel_share": main_run["kernel_share"],
        "mass_drift_per_step": main_run["mass_resid"] / (args.steps + max(args.warmup, 3)),
        "variants": {k: {kk: v[kk] for kk in ("mlups", "ms_per_step", "liquid_gbs", "step_gbs", "launches",
                                               "mass_resid", "liquid_ms", "liquid_bytes", "n_liquid", "n_general")}
                     | {"frac": v["liquid_gbs"] / hbm, "dtype": DTYPE[k],
                        "traffic": stored_traffic(k, v["liquid_bytes"])}
                     for k, v in variants.items()},
    }
    if main_run["late_window"] is not None:
        line["late_window"] = main_run["late_window"]
    if "f64" in variants:
        # the double path is bound by double arithmetic (GB300's FP64 rate is
        # 1/64 of its FP32 rate), not by memory: its bulk kernel's FP64
        # operations per second against this GPU's measured add rate (the
        # unit is built without fused multiply-add: adds and multiplies)
        v = variants["f64"]
        ops = stored_fp64_ops()
        achieved = None if ops is None else ops * (v["n_liquid"] - v["n_general"]) / (v["liquid_ms"] * 1e-3)
        line["variants"]["f64"]["roofline"] = {
            "bound": "alu", "kernel": "k_liquid<0>", "unit": "FP64 op/s", "achieved": achieved,
            "peak": fp64_rates["add"], "frac": None if achieved is None else achieved / fp64_rates["add"],
            "peak_source": "measured in this run: lbm_fs_fp64_rate (independent add chains on every SM)",
            "rates_measured": fp64_rates, "ops_per_liquid_cell": ops,
            "ops_source": "ncu sass thread instructions dadd + dmul + dfma of one launch (profiles/k_liquid_traffic.json)"}
    if batch is not None:
        line["batch"] = {
            "workload": "%d tanks of edge 48..112 (seeded), heeled boxes, FP16-shifted storage, one launch per " % batch["tanks"] +
                        "kernel for all tanks", "dtype": DTYPE["f16s"], "cells": batch["cells"],
            "mlups": batch["mlups"], "ms_per_step": batch["ms_per_step"], "launches": batch["launches"],
            "roofline": {"bound": "hbm", "kernel": "batched k_liquid", "achieved": batch["liquid_gbs"], "peak": hbm,
                         "unit": "GB/s", "frac": batch["liquid_gbs"] / hbm,
                         "algorithmic_bytes_per_launch": batch["liquid_bytes"],
                         "step_achieved_gbs": batch["step_gbs"], "step_frac": batch["step_gbs"] / hbm},
            "kernel_share": batch["kernel_share"], "autotune": batch["autotune"],
            "separate_handles_ms_per_step": batch["separate_ms_per_step"],
            "f32": {"dtype": DTYPE["f32"], "mlups": batch32["mlups"], "ms_per_step": batch32["ms_per_step"],
                    "launches": batch32["launches"], "autotune": batch32["autotune"],
                    "roofline": {"bound": "hbm", "kernel": "batched k_liquid", "achieved": batch32["liquid_gbs"],
                                 "peak": hbm, "unit": "GB/s", "frac": batch32["liquid_gbs"] / hbm,
                                 "algorithmic_bytes_per_launch": batch32["liquid_bytes"],
                                 "step_achieved_gbs": batch32["step_gbs"], "step_frac": batch32["step_gbs"] / hbm}}}
    print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
