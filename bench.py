#!/usr/bin/env python3
"""Benchmark of the GB300 persistent-homology path.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Workloads (seeded synthetic fields shaped like the paper's images/volumes):
  grf512cube       one 3D 512^3 GRF (sigma 4), H0-H2, forward; the backward of
                   sum over H1 and H2 of lifetime^2 is timed beside it
                                                                -- default; metric cells/s
  grf256cube_salt  one 3D 256^3 GRF (sigma 3) + 1% salt, H0-H2  -- metric cells/s
  grf1024          one 2D 1024x1024 GRF (sigma 4), H0+H1        -- metric cells/s
  batch4096        4096 2D GRFs of sides 28..256, batched forward + backward of
                   sum_H1 lifetime^2                            -- metric images/s
  uniform64        one 2D 64x64 U[0,1) image, H0+H1             -- metric cells/s

A step is one pass of the whole path over one input resident in HBM.  Between
timed steps a 256 MiB buffer is written to flush L2.  Each step is bracketed by
CUDA events on the stream the library launches on; the JSON line reports the
mean.  With the default workload the other three configurations (1024^2,
256^3 + salt, the 4096-image batch beside the plain per-image path) are
measured after it and reported as extra keys.  ``--impl reference`` times the
CPU oracle on the host cores instead (a bounded sample of the same workload
per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
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
    "grf512cube": dict(kind="single", shape=(512, 512, 512), maxdim=2, steps=5, backward=True),
    "batch4096": dict(kind="batch", n=4096, maxdim=1, steps=10),
}
DEFAULT_WORKLOAD = "grf512cube"
# measured after the default workload and reported as extra keys
EXTRA_WORKLOADS = ("grf1024", "grf256cube_salt", "batch4096")

# kernels whose bound is HBM bandwidth (one launch per call; algorithmic bytes
# per launch are counted by the library, cr_profile_read) and kernels bound by
# latency (dependent loads, grid barriers): reported as time and path length
HBM_STAGES = ("h0_stencil", "dual_stencil", "h1_scan", "h0_cross", "dual_cross")
LATENCY_STAGES = ("h1_reduce", "uf_round", "jump")
ROOFLINE_KERNEL = {"single3": "h1_scan", "single2": "h0_stencil", "batch": "h0_stencil"}


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


def stage_mask(cr, names):
    import ctypes
    L = cr.lib()
    nm = ctypes.c_char_p()
    mask = 0
    for s in range(64):
        if L.cr_profile_read(s, ctypes.byref(nm), None, None, None) != 0:
            break
        if nm.value.decode() in names:
            mask |= 1 << s
    return mask


def kernel_source_sha(kernel):
    """SHA-256 of the source file that holds a stage's kernel (the traffic
    counters of a kernel are valid only for the source they were taken on)."""
    f = {"h1_scan": "cr_h1.cu", "h1_reduce": "cr_h1.cu"}.get(kernel, "cr_uf.cu")
    with open(os.path.join(ROOT, "paper_2005_12692_gb300", "csrc", f), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()


def measured_traffic(kernel, workload):
    """DRAM bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)
    from the summary under profiles/, if it was taken on the current source of
    the kernel; None otherwise."""
    path = os.path.join(ROOT, "profiles", "dram_traffic_%s.md" % workload)
    try:
        text = open(path).read()
    except OSError:
        return None, None
    sha = kernel_source_sha(kernel)
    for m in re.finditer(r"^traffic (\w+) (\d+) bytes per launch, source sha256 ([0-9a-f]{64})", text, re.M):
        if m.group(1) == kernel:
            if m.group(3) == sha:
                return int(m.group(2)), "profiles/dram_traffic_%s.md" % workload
            return None, "stale: %s changed since the capture" % kernel
    return None, None


def roofline_entry(kernel, s, peaks, workload):
    per_launch_s = s["ms"] / 1e3 / s["launches"]
    per_launch_bytes = s["bytes"] / s["launches"]
    achieved = per_launch_bytes / per_launch_s / 1e9
    peak = peaks.get("hbm_gbs")
    src = "measured (MEASURED_PEAKS.json hbm_gbs, copy bandwidth)"
    if not peak:
        peak, src = 6800.0, "fallback"
    traffic, tsrc = measured_traffic(kernel, workload)
    return {"kernel": kernel, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_source": src, "traffic": traffic, "traffic_source": tsrc,
            "algorithmic_bytes_per_launch": per_launch_bytes, "ms_per_launch": per_launch_s * 1e3,
            "traffic_over_algorithmic": round(traffic / per_launch_bytes, 3) if traffic else None}


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
        return {"batch_threads": [0, 1, 2, 3], "uf_compact": [1, 4]}
    if len(data.shape) == 3 and min(data.shape) > 1:
        return {"red_warps": [8, 16], "uf_compact": [1, 4], "red_budget": [512, 1024, 2048]}
    return {"uf_items": [2, 4, 8, 16, 32], "uf_compact": [1, 2, 4, 8]}


def workload_config(name, W, data, world, size=None):
    """The config object of the JSON line (the same for both arms)."""
    return {"workload": name,
            "shape": list(data.shape) if W["kind"] == "single" else "4096 x U{28..256}^2",
            "maxdim": W["maxdim"], "cells": num_cells(data.shape) if W["kind"] == "single" else None,
            "size_override": size,
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
VOLUME_SAMPLE = 144  # corner crop side: about 10 s of the oracle on one core


def volume_sample_side(calls):
    """Crop side for an oracle run repeated `calls` times: about 150 s in all at the oracle's ~1.8 M cells/s on
    one core of the box (8 cells per voxel), never above VOLUME_SAMPLE."""
    per_call = 150.0 / max(1, calls)
    side = int((per_call * 1.8e6 / 8.0) ** (1.0 / 3.0))
    return max(32, min(VOLUME_SAMPLE, side))


def _oracle_one(a):
    import oracle
    oracle.build()
    oracle.persistence(a)
    return a.size


def oracle_sample(name, data, batch_images=1024, side=VOLUME_SAMPLE):
    """A bounded sample of the workload for the CPU oracle: (arrays, units, unit-scale, description)."""
    if name in ("uniform64", "grf1024"):
        return [data], num_cells(data.shape), "the full %s image" % "x".join(map(str, data.shape))
    if name in ("grf256cube_salt", "grf512cube"):
        k = side
        sub = np.ascontiguousarray(data[:k, :k, :k])
        return [sub], num_cells(sub.shape), "a %d^3 corner crop of the %d^3 volume, scaled to cells/s" % (
            k, data.shape[0])
    if name == "batch4096":
        imgs = list(data[:batch_images])
        return imgs, len(imgs), ("the first %d of the 4096 images (forward), per image over the host cores, "
                                 "scaled to images/s" % len(imgs))
    raise ValueError(name)


class OracleRunner:
    """Times the oracle on a sample.  Batches run one image per task on a pool
    of all host cores, started with 'spawn' (no GPU state is inherited)."""

    def __init__(self, name, side=VOLUME_SAMPLE):
        self.name = name
        self.side = side
        self.pool = None
        self.cores = 1
        if WORKLOADS[name]["kind"] == "batch":
            import multiprocessing as mp
            self.cores = os.cpu_count() or 1
            self.pool = mp.get_context("spawn").Pool(self.cores)
            self.pool.map(_oracle_one, [np.zeros((2, 2), np.float32)] * self.cores)  # workers up and built

    def run(self, data):
        import oracle
        oracle.build()
        arrs, units, desc = oracle_sample(self.name, data, side=self.side)
        t0 = time.perf_counter()
        if self.pool is not None:
            self.pool.map(_oracle_one, arrs, chunksize=1)
        else:
            for a in arrs:
                oracle.persistence(a)
        dt = time.perf_counter() - t0
        return units / dt, dt, desc

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()


# ---------------------------------------------------------------------------
# GPU helpers
# ---------------------------------------------------------------------------
def make_step(cr, W, data, dev):
    """(step function, units per step, extra state) for a workload resident on `dev`."""
    import torch
    if W["kind"] == "single":
        img = torch.from_numpy(data).to(dev)

        def step():
            return cr.cr_persistence(img, maxdim=W["maxdim"])
        return step, num_cells(data.shape), {"img": img}
    shapes = [tuple(a.shape) for a in data]
    offs = [0]
    for a in data:
        offs.append(offs[-1] + a.size)
    flat = torch.from_numpy(np.concatenate([a.reshape(-1) for a in data])).to(dev)

    def step():
        bp = cr.cr_persistence_batched(flat, maxdim=1, shapes=shapes, offsets=offs)
        p = bp.pairs
        sel = (p.dim == 1) & torch.isfinite(p.death)
        life = torch.where(sel, p.death - p.birth, torch.zeros_like(p.birth))
        return cr.cr_backward_batched(flat, shapes, offs, bp, -2 * life, 2 * life)
    return step, len(data), {"flat": flat, "shapes": shapes, "offs": offs}


def time_calls(fn, n, stream, flush, dev):
    """Milliseconds of each of n calls, CUDA events on `stream`, L2 flushed before each."""
    import torch
    out = []
    for _ in range(n):
        flush.fill_(1)
        torch.cuda.synchronize(dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        out.append(a.elapsed_time(b))
    return out


def plain_path(cr, data, dev, stream, sub=512):
    """The plain per-image path on the same GPU: a loop of cr_persistence +
    cr_backward over the first `sub` images of a batch, same loss."""
    import torch
    imgs_dev = [torch.from_numpy(a).to(dev) for a in data[:sub]]

    def run():
        for im in imgs_dev:
            p = cr.cr_persistence(im, maxdim=1)
            sel = (p.dim == 1) & torch.isfinite(p.death)
            life = torch.where(sel, p.death - p.birth, torch.zeros_like(p.birth))
            cr.cr_backward(im, p, -2 * life, 2 * life)

    run()
    torch.cuda.synchronize(dev)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    run()
    b.record(stream)
    b.synchronize()
    pms = a.elapsed_time(b)
    return {"images_per_s": sub / (pms / 1e3), "sample": "first %d images, same loss, one stream" % sub}


def measure_extra(cr, name, dev, stream, flush, steps=10, warmup=3, tune=True):
    """One of the other configurations, device-resident, L2 flushed between steps; its launch knobs tuned
    for it first, as the headline's are (outside the timed region)."""
    W = WORKLOADS[name]
    data = make_input(name)
    step, units, st = make_step(cr, W, data, dev)
    tuned = None
    if tune:
        from paper_2005_12692_gb300 import autotune as at
        try:
            tuned = at.autotune(step, tune_candidates(W, data), warmup=2, repeats=3).best
        except cr.CRError:  # keep the default launch shapes
            at.apply(at.DEFAULTS)
    for _ in range(warmup):
        step()
    ms = time_calls(step, steps, stream, flush, dev)
    m = statistics.mean(ms)
    unit = "images/s" if W["kind"] == "batch" else "cells/s"
    out = {"value": units / (m / 1e3), "unit": unit, "ms_per_step": m, "steps": steps, "warmup": warmup,
           "config": workload_config(name, W, data, 1), "tuning": tuned}
    if W["kind"] == "batch":
        pl = plain_path(cr, data, dev, stream)
        out["plain_path"] = pl
        out["batched_over_plain"] = out["value"] / pl["images_per_s"]
    del st
    return out


# ---------------------------------------------------------------------------
# main
# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default per workload: enough for a timed region of ~0.1 s or more)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end loop (profiling runs)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other configurations and side measurements (profiling runs)")
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
    unit = metric.split()[0]

    if args.impl == "reference":
        if rank != 0:
            return 0
        data = make_input(args.workload, args.size)
        runner = OracleRunner(args.workload, side=volume_sample_side(args.warmup + args.steps))
        vals = []
        try:
            for i in range(args.warmup + args.steps):
                v, dt, desc = runner.run(data)
                if i >= args.warmup:
                    vals.append((v, dt))
        finally:
            runner.close()
        value = statistics.mean(v for v, _ in vals)
        line = {"metric": metric, "value": value, "unit": unit, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * statistics.mean(dt for _, dt in vals),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "impl": "reference",
                "config": workload_config(args.workload, W, data, 1, args.size),
                "cpu_baseline": {"value": value, "unit": unit, "cores": runner.cores, "kind": "oracle",
                                 "sample": desc},
                "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
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
    volume = W["kind"] == "single" and len(data.shape) == 3 and min(data.shape) > 1
    rkey = "batch" if W["kind"] == "batch" else ("single3" if volume else "single2")

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    step, units, state = make_step(cr, W, data, dev)

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

    # -------- timed region (device-resident input) --------
    # events bracket the HBM-class and latency-class kernels (a few per step),
    # for the roofline of each; the step time is the events around the step
    L.cr_profile_reset()
    L.cr_profile_select(stage_mask(cr, HBM_STAGES + LATENCY_STAGES))
    L.cr_profile_enable(1)
    launches0 = int(L.cr_launch_count())
    step_ms = []
    barrier()
    t_region0 = time.time()
    last = None
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize(dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        last = step()
        b.record(stream)
        b.synchronize()
        step_ms.append(a.elapsed_time(b))
    launches = int(L.cr_launch_count()) - launches0
    L.cr_profile_enable(0)
    L.cr_profile_select(0xFFFFFFFF)
    timed_stages = read_profile(cr)
    # the backward of the configuration (sum over H1 and H2 of lifetime^2),
    # timed in the same clock window, on the pairs of the last timed step
    backward = None
    if W.get("backward") and W["kind"] == "single":
        img = state["img"]
        sel = (last.dim >= 1) & torch.isfinite(last.death)
        life = torch.where(sel, last.death - last.birth, torch.zeros_like(last.birth))
        gb, gd = -2 * life, 2 * life
        cr.cr_backward(img, last, gb, gd)
        bms = time_calls(lambda: cr.cr_backward(img, last, gb, gd), max(3, args.steps), stream, flush, dev)
        bm = statistics.mean(bms)
        backward = {"ms_per_call": bm, "calls": len(bms), "pairs": last.n,
                    "loss": "sum over H1 and H2 of (death - birth)^2",
                    "fwd_plus_bwd_cells_per_s": units / ((statistics.mean(step_ms) + bm) / 1e3)}
    barrier()
    t_region1 = time.time()
    clk = clocks.stop((t_region0, t_region1))
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    ms_per_step = total_ms / args.steps
    value = job_value(units, world, ms_per_step)

    # -------- rooflines: HBM-class kernels against the measured copy bandwidth --------
    peaks = load_peaks()
    hbm = {}
    for k in HBM_STAGES:
        s = timed_stages.get(k)
        if s and s["launches"] and s["ms"] > 0 and s["bytes"] > 0:
            hbm[k] = roofline_entry(k, s, peaks, args.workload if args.size is None else None)
    rk = ROOFLINE_KERNEL[rkey]
    roof = hbm.get(rk)
    latency = {}
    for k in LATENCY_STAGES:
        s = timed_stages.get(k)
        if s and s["launches"]:
            latency[k] = {"ms_per_launch": s["ms"] / s["launches"], "share_of_step": s["ms"] / sum(step_ms)}
    if "h1_reduce" in latency:
        import ctypes
        st = (ctypes.c_int64 * 26)()
        L.cr_h1_last_stats(st, 26)
        maxit = int(st[8])
        latency["h1_reduce"].update({
            "residual_columns": int(st[0]), "critical_path_iterations": maxit,
            "ns_per_critical_iteration": latency["h1_reduce"]["ms_per_launch"] * 1e6 / maxit if maxit else None,
            "note": "serial chain of the longest column: time = iterations x dependent-load latency"})

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
            del dimg
    else:
        flat, shapes, offs = state["flat"], state["shapes"], state["offs"]
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

    extra = {}
    plain = None
    images = None
    f64 = None
    if not args.no_extra:
        # the plain per-image path beside the batched one
        if W["kind"] == "batch":
            plain = plain_path(cr, data, dev, stream)
            plain["batched_over_plain"] = value / plain["images_per_s"]

        # the localised-feature images (Sec. 4) from one call's pairs, timed alone
        if W["kind"] == "single":
            pr = step()
            shp = tuple(data.shape)
            nd = len(shp)
            vox = int(np.prod(shp))
            lo, hi = float(data.min()), float(data.max())
            nbh = 8 if vox <= (1 << 24) else 2  # histogram channels: 2 x 2 bins per dimension for volumes
            for _ in range(2):
                cr.lifetime_image(shp, pr)
                cr.persistent_histogram_image(shp, pr, nbh, (lo, hi), nbh, hi - lo)
            reps = 10
            res = {}
            for nm, fn, nbytes in (
                    ("lifetime_image", lambda: cr.lifetime_image(shp, pr), 4.0 * nd * vox + 32.0 * pr.n),
                    ("histogram_image_%dx%d" % (nbh, nbh),
                     lambda: cr.persistent_histogram_image(shp, pr, nbh, (lo, hi), nbh, hi - lo),
                     4.0 * nd * nbh * nbh * vox + 32.0 * pr.n)):
                torch.cuda.synchronize(dev)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for _ in range(reps):
                    fn()
                b.record(stream)
                b.synchronize()
                ms = a.elapsed_time(b) / reps
                res[nm] = {"ms": ms, "algorithmic_bytes": nbytes, "gbs": nbytes / (ms / 1e3) / 1e9}
            images = {"pairs": pr.n, **res,
                      "note": "output zero-fill + one scatter per pair; inputs in HBM; not part of the timed step"}
            del pr
            torch.cuda.empty_cache()

        # the float64 input path on the same field (Sec. 3's precision), timed alone
        if W["kind"] == "single":
            try:
                img64 = torch.from_numpy(data.astype(np.float64)).to(dev)
                reps = max(3, min(args.steps, 20)) if len(data.shape) < 3 else 2
                for _ in range(2):
                    cr.cr_persistence_f64(img64, maxdim=W["maxdim"])
                f64_ms = time_calls(lambda: cr.cr_persistence_f64(img64, maxdim=W["maxdim"]), reps, stream,
                                    flush, dev)
                ms64 = statistics.mean(f64_ms)
                f64 = {"value": units / (ms64 / 1e3), "unit": unit, "ms_per_call": ms64, "calls": reps,
                       "note": "cr_persistence_f64 on the same field cast to float64, device-resident, L2 flushed"}
                del img64
                torch.cuda.empty_cache()
            except Exception as e:  # reported, never fatal to the headline numbers
                f64 = {"error": str(e)[:200]}

        # the other configurations, after the headline's measurements
        if args.workload == DEFAULT_WORKLOAD and args.size is None and world == 1:
            del state
            for name in EXTRA_WORKLOADS:
                try:
                    extra[name] = measure_extra(cr, name, dev, stream, flush,
                                                steps=min(WORKLOADS[name]["steps"], 20),
                                                tune=args.autotune == "on")
                except Exception as e:  # reported, never fatal to the headline numbers
                    extra[name] = {"error": str(e)[:200]}
                torch.cuda.empty_cache()

    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": args.gpus * 0 + world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(args.workload, W, data, world, args.size),
            "clocks": clk, "gpu_launches": launches,
            "e2e": {"value": e2e_value, "unit": unit, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "roofline": roof,
            "roofline_hbm_kernels": hbm,
            "latency_kernels": latency,
            "backward": backward,
            "tuning": tuning,
            "plain_path": plain,
            "configs": extra or None,
            "localised_images": images,
            "f64_path": f64,
            "stages": {k: {"ms_per_step": v["ms"] / prof_steps, "launches_per_step": v["launches"] / prof_steps}
                       for k, v in stages.items()},
            "stages_note": "separate profiled pass of %d steps (events around every stage)" % prof_steps}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        runner = OracleRunner(args.workload)
        try:
            v, dt, desc = runner.run(data)
        finally:
            runner.close()
        line["cpu_baseline"] = {"value": v, "unit": unit, "cores": runner.cores, "kind": "oracle",
                                "sample": desc, "seconds": dt}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
