#!/usr/bin/env python3
"""Benchmark of the GB300 persistent-homology path.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Workloads (seeded synthetic fields shaped like the paper's images/volumes):
  grf1024          one 2D 1024x1024 GRF (sigma 4), H0+H1        -- default; metric cells/s
  uniform64        one 2D 64x64 U[0,1) image, H0+H1             -- metric cells/s
  grf256cube_salt  one 3D 256^3 GRF (sigma 3) + 1% salt, H0-H2  -- metric cells/s
  grf512cube       one 3D 512^3 GRF (sigma 4), H0-H2            -- metric cells/s
  batch4096        4096 2D GRFs of sides 28..256, batched forward + backward of
                   sum_H1 lifetime^2                            -- metric images/s

A step is one pass of the whole path over one input resident in HBM.  Between
timed steps a 256 MiB buffer is written to flush L2 (inputs of the 2D
workloads fit in L2).  Each step is bracketed by CUDA events on the stream the
library launches on; the JSON line reports the mean.  ``--impl reference``
times the CPU oracle on the host cores instead (a bounded sample of the same
workload per step).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    "uniform64": dict(kind="single", shape=(64, 64), maxdim=1, steps=500),
    "grf1024": dict(kind="single", shape=(1024, 1024), maxdim=1, steps=200),
    "grf256cube_salt": dict(kind="single", shape=(256, 256, 256), maxdim=2, steps=10),
    "grf512cube": dict(kind="single", shape=(512, 512, 512), maxdim=2, steps=5),
    "batch4096": dict(kind="batch", n=4096, maxdim=1, steps=10),
}


def make_input(name, size=None):
    from paper_2005_12692_gb300 import synth
    if name == "uniform64":
        return synth.uniform64()
    if name == "grf1024":
        return synth.grf1024(size or 1024)
    if name == "grf256cube_salt":
        return synth.grf256cube_salt(size or 256)
    if name == "grf512cube":
        return synth.grf512cube(size or 512)
    if name == "batch4096":
        return synth.batch_images(4096)
    raise ValueError(name)


def num_cells(shape):
    n = 1
    for s in shape:
        n *= 2 * int(s) - 1
    return n


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi sampling (every 20 ms) from before the warm-up to the end of
    the timed region.  Samples carry nvidia-smi's own timestamps; the report
    uses those inside the timed region, or, when the region is shorter than
    the sampling period, the nearest sample on each side of it (the GPU is
    running the same steps then: warm-up and the profiled pass precede it)."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0:  # sampler live before the GPU work starts
                time.sleep(0.01)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    @staticmethod
    def _ts(text):
        from datetime import datetime
        try:
            return datetime.strptime(text.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def stop(self, region):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.05)  # one more sample after the region
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 10:
                continue
            try:
                rows.append((self._ts(parts[0]), float(parts[2]), float(parts[3]),
                             {nm for nm, v in zip(names, parts[6:10]) if v.lower() == "active"}))
            except ValueError:
                continue
        t0, t1 = region
        inside = [r for r in rows if r[0] is not None and t0 <= r[0] <= t1]
        window = "timed region"
        use = inside
        if not use:
            before = [r for r in rows if r[0] is not None and r[0] < t0]
            after = [r for r in rows if r[0] is not None and r[0] > t1]
            use = before[-1:] + after[:1]
            window = "nearest sample on each side of the timed region (%.1f ms, shorter than the 20 ms sampling)" \
                % ((t1 - t0) * 1e3)
        reasons = set()
        for r in use:
            reasons |= r[3]
        return {"sm_mhz": statistics.median(r[1] for r in use) if use else None,
                "sm_max_mhz": max(r[2] for r in use) if use else None,
                "reasons": sorted(reasons), "samples": len(use), "window": window}


# ---------------------------------------------------------------------------
# stage profile read from the library
# ---------------------------------------------------------------------------
def read_profile(cr):
    import ctypes
    L = cr.lib()
    out = {}
    name = ctypes.c_char_p()
    ms = ctypes.c_double()
    cnt = ctypes.c_int64()
    by = ctypes.c_double()
    for s in range(64):
        if L.cr_profile_read(s, ctypes.byref(name), ctypes.byref(ms), ctypes.byref(cnt), ctypes.byref(by)) != 0:
            break
        if cnt.value:
            out[name.value.decode()] = {"ms": ms.value, "launches": cnt.value, "bytes": by.value}
    return out


# stages that are one kernel launch per call (the roofline is quoted per kernel)
SINGLE_KERNEL_STAGES = ("h0_stencil", "h0_cross", "dual_stencil", "dual_cross", "h1_scan", "h1_reduce", "uf_round")


# what bounds each kernel in practice (the roofline denominator is HBM for all)
LIMITER = {"uf_round": "latency: grid barriers and dependent loads per phase",
           "h1_reduce": "latency: serial chain of the longest column",
           "h0_cross": "latency: scattered neighbour label loads",
           "dual_cross": "latency: scattered neighbour label loads"}


def dominant_stage(stages):
    best = None
    for k in SINGLE_KERNEL_STAGES:
        if k in stages and (best is None or stages[k]["ms"] > stages[best]["ms"]):
            best = k
    return best


def stage_index(cr, name):
    import ctypes
    L = cr.lib()
    nm = ctypes.c_char_p()
    for s in range(64):
        if L.cr_profile_read(s, ctypes.byref(nm), None, None, None) != 0:
            break
        if nm.value.decode() == name:
            return s
    raise KeyError(name)


def roofline_from(stages, peaks, sustained=True):
    best = None
    for k in SINGLE_KERNEL_STAGES:
        s = stages.get(k)
        if s and (best is None or s["ms"] > stages[best]["ms"]):
            best = k
    if best is None:
        return None
    s = stages[best]
    per_launch_s = s["ms"] / 1e3 / s["launches"]
    per_launch_bytes = s["bytes"] / s["launches"]
    achieved = per_launch_bytes / per_launch_s / 1e9
    peak = peaks.get("hbm_gbs")
    src = "measured"
    if not peak:
        peak, src = 6800.0, "fallback"
    return {"kernel": best, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_source": src, "traffic": None,
            "bytes_per_launch": per_launch_bytes, "ms_per_launch": per_launch_s * 1e3,
            "limiter": LIMITER.get(best, "hbm")}


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest x over all ranks: a replicated job's time is its slowest rank's."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: float, world: int, ms_per_step: float) -> float:
    """Whole-job throughput: every rank processes units_per_rank per step (weak scaling)."""
    return units_per_rank * world / (ms_per_step / 1e3)


def tune_candidates(W, data):
    """Knob values the autotuner tries for a workload (knobs that cannot change its launches are left out:
    a batch or a volume always fills every SM with union-find blocks; only volumes run the reduction)."""
    if W["kind"] == "batch":
        return {"uf_compact": [1, 2, 4, 8]}
    if len(data.shape) == 3 and min(data.shape) > 1:
        return {"red_warps": [8, 16], "uf_compact": [1, 4]}
    return {"uf_items": [2, 4, 8, 16, 32], "uf_compact": [1, 2, 4, 8]}


def workload_config(args, W, data, world):
    """The config object of the JSON line (the same for both arms)."""
    return {"workload": args.workload,
            "shape": list(data.shape) if W["kind"] == "single" else "4096 x U{28..256}^2",
            "maxdim": W["maxdim"], "cells": num_cells(data.shape) if W["kind"] == "single" else None,
            "size_override": args.size,
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "flushed between steps (256 MiB write)"}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f)
    except Exception:
        return {}


# ---------------------------------------------------------------------------
# oracle (CPU baseline / reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(name, data):
    """A bounded sample of the workload for the CPU oracle: (array(s), cells, description)."""
    from paper_2005_12692_gb300 import synth
    if name in ("uniform64", "grf1024"):
        return [data], num_cells(data.shape), "the full %s image" % "x".join(map(str, data.shape))
    if name == "grf256cube_salt":
        sub = np.ascontiguousarray(data[:48, :48, :48])
        return [sub], num_cells(sub.shape), "a 48^3 corner crop of the 256^3 volume"
    if name == "grf512cube":
        sub = np.ascontiguousarray(data[:48, :48, :48])
        return [sub], num_cells(sub.shape), "a 48^3 corner crop of the 512^3 volume"
    if name == "batch4096":
        imgs = data[:16]
        return imgs, len(imgs), "the first 16 of the 4096 images (forward only), scaled to images/s"
    raise ValueError(name)


def run_oracle(name, data):
    import oracle
    oracle.build()
    arrs, units, desc = oracle_sample(name, data)
    t0 = time.perf_counter()
    for a in arrs:
        oracle.persistence(a)
    dt = time.perf_counter() - t0
    return units / dt, dt, desc


# ---------------------------------------------------------------------------
# main
# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default per workload: enough for a timed region of ~0.1 s or more)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="grf1024", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end loop (profiling runs)")
    ap.add_argument("--autotune", default="on", choices=["on", "off"],
                    help="pick the library's launch knobs by timing candidates before the warm-up (not timed)")
    ap.add_argument("--size", type=int, default=None,
                    help="side length override of a single-image workload (same recipe; profiling on smaller cases)")
    args = ap.parse_args()
    W = WORKLOADS[args.workload]
    if args.steps is None:
        # the oracle arm times seconds-long CPU samples: a handful of steps
        args.steps = 5 if args.impl == "reference" else W["steps"]

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    metric = "images/s batched fwd+bwd" if W["kind"] == "batch" else "cells/s full PH"

    if args.impl == "reference":
        if rank != 0:
            return 0
        data = make_input(args.workload, args.size)
        import oracle  # noqa: F401
        cores = 1
        vals = []
        for i in range(args.warmup + args.steps):
            v, dt, desc = run_oracle(args.workload, data)
            if i >= args.warmup:
                vals.append((v, dt))
        value = statistics.mean(v for v, _ in vals)
        line = {"metric": metric, "value": value, "unit": metric.split()[0], "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * statistics.mean(dt for _, dt in vals),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "impl": "reference",
                "config": workload_config(args, W, data, 1),
                "cpu_baseline": {"value": value, "unit": metric.split()[0], "cores": cores, "kind": "oracle",
                                 "sample": desc},
                "e2e": {"value": value, "unit": metric.split()[0], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import torch
    import paper_2005_12692_gb300 as cr

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cr.build()
    L = cr.lib()

    data = make_input(args.workload, args.size)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    # -------- the step --------
    if W["kind"] == "single":
        img = torch.from_numpy(data).to(dev)
        units = num_cells(data.shape)

        def step():
            return cr.cr_persistence(img, maxdim=W["maxdim"])
    else:
        shapes = [tuple(a.shape) for a in data]
        offs = [0]
        for a in data:
            offs.append(offs[-1] + a.size)
        flat = torch.from_numpy(np.concatenate([a.reshape(-1) for a in data])).to(dev)
        units = len(data)

        def step():
            bp = cr.cr_persistence_batched(flat, maxdim=1, shapes=shapes, offsets=offs)
            p = bp.pairs
            sel = (p.dim == 1) & torch.isfinite(p.death)
            life = torch.where(sel, p.death - p.birth, torch.zeros_like(p.birth))
            g = cr.cr_backward_batched(flat, shapes, offs, bp, -2 * life, 2 * life)
            return g

    # -------- launch knobs: tuned offline, before the warm-up, outside every timed region --------
    tuning = None
    if args.autotune == "on":
        from paper_2005_12692_gb300 import autotune as at
        t0 = time.time()
        try:
            res = at.autotune(step, tune_candidates(W, data), warmup=2, repeats=3)
            tuning = {"best": res.best, "seconds": round(time.time() - t0, 2), "table": res.as_dict()["table"]}
        except cr.CRError as e:  # keep the default launch shapes
            at.apply(at.DEFAULTS)
            tuning = {"error": str(e)[:200], "best": at.current()}

    clocks = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    clocks.start()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    # -------- stage breakdown (separate pass: its events would perturb the timing) --------
    prof_steps = max(2, min(args.steps, 5))
    L.cr_profile_select(0xFFFFFFFF)
    L.cr_profile_reset()
    L.cr_profile_enable(1)
    for _ in range(prof_steps):
        flush.fill_(1)
        step()
    torch.cuda.synchronize(dev)
    L.cr_profile_enable(0)
    stages = read_profile(cr)
    roof_stage = dominant_stage(stages)

    # -------- timed region (device-resident input) --------
    # only the dominant kernel's launches are bracketed by events, for the roofline
    L.cr_profile_reset()
    if roof_stage is not None:
        L.cr_profile_select(1 << stage_index(cr, roof_stage))
        L.cr_profile_enable(1)
    launches0 = int(L.cr_launch_count())
    step_ms = []
    barrier()
    t_region0 = time.time()
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize(dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        b.synchronize()
        step_ms.append(a.elapsed_time(b))
    barrier()
    t_region1 = time.time()
    clk = clocks.stop((t_region0, t_region1))
    L.cr_profile_enable(0)
    L.cr_profile_select(0xFFFFFFFF)
    launches = int(L.cr_launch_count()) - launches0
    timed_stages = read_profile(cr)
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    ms_per_step = total_ms / args.steps
    value = job_value(units, world, ms_per_step)

    # -------- end to end through host buffers --------
    e2e_ms = []
    if args.no_e2e:
        h2d = d2h = 0
    elif W["kind"] == "single":
        host = torch.from_numpy(data).pin_memory()
        h2d = host.numel() * 4
        d2h = 0
        for i in range(args.warmup + max(3, args.steps // 2)):
            flush.fill_(1)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            dimg = host.to(dev, non_blocking=True)
            p = cr.cr_persistence(dimg, maxdim=W["maxdim"])
            out = p.raw.cpu()
            torch.cuda.synchronize(dev)
            if i >= args.warmup:
                e2e_ms.append((time.perf_counter() - t0) * 1e3)
            d2h = out.numel()
    else:
        hflat = flat.cpu().pin_memory()
        h2d = hflat.numel() * 4
        d2h = 0
        for i in range(args.warmup + max(2, args.steps // 2)):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            dflat = hflat.to(dev, non_blocking=True)
            bp = cr.cr_persistence_batched(dflat, maxdim=1, shapes=shapes, offsets=offs)
            p = bp.pairs
            sel = (p.dim == 1) & torch.isfinite(p.death)
            life = torch.where(sel, p.death - p.birth, torch.zeros_like(p.birth))
            g = cr.cr_backward_batched(dflat, shapes, offs, bp, -2 * life, 2 * life)
            gh = g.cpu()
            torch.cuda.synchronize(dev)
            if i >= args.warmup:
                e2e_ms.append((time.perf_counter() - t0) * 1e3)
            d2h = gh.numel() * 4
    e2e_value = job_value(units, world, max_over_ranks(statistics.mean(e2e_ms), world, dev)) if e2e_ms else None

    # the plain per-image path on the same GPU (a subset, scaled to images/s)
    plain = None
    if W["kind"] == "batch" and not args.no_e2e:
        sub = 512
        imgs_dev = [torch.from_numpy(a).to(dev) for a in data[:sub]]

        def plain_step():
            for im in imgs_dev:
                p = cr.cr_persistence(im, maxdim=1)
                sel = (p.dim == 1) & torch.isfinite(p.death)
                life = torch.where(sel, p.death - p.birth, torch.zeros_like(p.birth))
                cr.cr_backward(im, p, -2 * life, 2 * life)

        plain_step()
        torch.cuda.synchronize(dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plain_step()
        b.record(stream)
        b.synchronize()
        pms = a.elapsed_time(b)
        plain = {"images_per_s": sub / (pms / 1e3), "sample": "first %d images, same loss" % sub,
                 "batched_over_plain": value / (sub / (pms / 1e3))}

    # the localised-feature images (Sec. 4) from one call's pairs, timed alone
    images = None
    if W["kind"] == "single":
        pr = step()
        shp = tuple(data.shape)
        nd = len(shp)
        vox = int(np.prod(shp))
        lo, hi = float(data.min()), float(data.max())
        for _ in range(3):
            cr.lifetime_image(shp, pr)
            cr.persistent_histogram_image(shp, pr, 8, (lo, hi), 8, hi - lo)
        reps = 20
        res = {}
        for name, fn, nbytes in (
                ("lifetime_image", lambda: cr.lifetime_image(shp, pr), 4.0 * nd * vox + 32.0 * pr.n),
                ("histogram_image_8x8", lambda: cr.persistent_histogram_image(shp, pr, 8, (lo, hi), 8, hi - lo),
                 4.0 * nd * 64 * vox + 32.0 * pr.n)):
            torch.cuda.synchronize(dev)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
            b.synchronize()
            ms = a.elapsed_time(b) / reps
            res[name] = {"ms": ms, "algorithmic_bytes": nbytes, "gbs": nbytes / (ms / 1e3) / 1e9}
        images = {"pairs": pr.n, **res,
                  "note": "output zero-fill + one scatter per pair; inputs in HBM; not part of the timed step"}

    # the float64 input path on the same field (Sec. 3's precision), timed alone after everything else
    f64 = None
    if W["kind"] == "single" and not args.no_e2e:
        try:
            img64 = torch.from_numpy(data.astype(np.float64)).to(dev)
            reps = max(3, min(args.steps, 20)) if len(data.shape) < 3 else 2
            for _ in range(3):
                cr.cr_persistence_f64(img64, maxdim=W["maxdim"])
            f64_ms = []
            for _ in range(reps):
                flush.fill_(1)
                torch.cuda.synchronize(dev)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                cr.cr_persistence_f64(img64, maxdim=W["maxdim"])
                b.record(stream)
                b.synchronize()
                f64_ms.append(a.elapsed_time(b))
            ms64 = statistics.mean(f64_ms)
            f64 = {"value": units / (ms64 / 1e3), "unit": metric.split()[0], "ms_per_call": ms64, "calls": reps,
                   "note": "cr_persistence_f64 on the same field cast to float64, device-resident, L2 flushed"}
        except Exception as e:  # reported, never fatal to the headline numbers
            f64 = {"error": str(e)[:200]}

    peaks = load_peaks()
    roof = roofline_from({roof_stage: timed_stages[roof_stage]} if roof_stage in timed_stages else stages, peaks)

    line = {"metric": metric, "value": value, "unit": metric.split()[0], "n_gpus": args.gpus * 0 + world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(args, W, data, world),
            "clocks": clk, "gpu_launches": launches,
            "e2e": {"value": e2e_value, "unit": metric.split()[0], "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "roofline": roof,
            "tuning": tuning,
            "plain_path": plain,
            "localised_images": images,
            "f64_path": f64,
            "stages": {k: {"ms_per_step": v["ms"] / prof_steps, "launches_per_step": v["launches"] / prof_steps}
                       for k, v in stages.items()},
            "stages_note": "separate profiled pass of %d steps (events around every stage)" % prof_steps}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, dt, desc = run_oracle(args.workload, data)
        line["cpu_baseline"] = {"value": v, "unit": metric.split()[0], "cores": 1, "kind": "oracle",
                                "sample": desc, "seconds": dt}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
