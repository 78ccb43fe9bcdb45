"""Autotuner for the library's launch knobs (include/cr.h, cr_tune_set).

The knobs set launch shapes only: how many blocks the cooperative union-find
grids use, when its rounds stop compacting their edge list, how many warps per
SM run the 3D reduction, and the block size of the persistent launch that
takes the images of a 2D batch from a queue (or the grid-wide kernels
instead).  Results never depend on them (the parity tests run
under every candidate value), so the tuner may pick any candidate by time
alone.

``autotune(run, candidates)`` does coordinate descent: knob by knob, each
candidate value is timed (median of ``repeats`` calls after ``warmup``) with
the other knobs at their best so far, and the fastest value is kept.  It leaves
the best values set in the library and returns them with the timing table.
``save``/``load`` keep choices in a JSON file, keyed by device and workload.
"""
from __future__ import annotations

import json
import os
import statistics
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence, Tuple

from . import (CR_TUNE_BATCH_THREADS, CR_TUNE_RED_BUDGET, CR_TUNE_RED_WARPS, CR_TUNE_UF_COMPACT, CR_TUNE_UF_ITEMS,
               cr_tune_get, cr_tune_set)

KNOBS: Dict[str, int] = {
    "uf_items": CR_TUNE_UF_ITEMS,
    "red_warps": CR_TUNE_RED_WARPS,
    "uf_compact": CR_TUNE_UF_COMPACT,
    "batch_threads": CR_TUNE_BATCH_THREADS,
    "red_budget": CR_TUNE_RED_BUDGET,
}

DEFAULTS: Dict[str, int] = {"uf_items": 8, "red_warps": 16, "uf_compact": 1, "batch_threads": 2, "red_budget": 1024}


def current() -> Dict[str, int]:
    """The library's present knob values."""
    return {name: cr_tune_get(k) for name, k in KNOBS.items()}


def apply(values: Dict[str, int]) -> None:
    """Set knobs by name (unknown names raise KeyError)."""
    for name, v in values.items():
        cr_tune_set(KNOBS[name], int(v))


def cuda_timer(run: Callable[[], object]) -> float:
    """Milliseconds of one call of ``run``, by CUDA events on the current stream."""
    import torch
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record()
    run()
    e.record()
    e.synchronize()
    return float(s.elapsed_time(e))


@dataclass
class TuneResult:
    best: Dict[str, int]
    table: List[Tuple[str, int, float]] = field(default_factory=list)  # (knob, value, median ms)

    def as_dict(self) -> dict:
        return {"best": dict(self.best),
                "table": [{"knob": k, "value": v, "ms": round(ms, 4)} for k, v, ms in self.table]}


def autotune(run: Callable[[], object], candidates: Dict[str, Sequence[int]], warmup: int = 2,
             repeats: int = 5, timer: Optional[Callable[[Callable[[], object]], float]] = None) -> TuneResult:
    """Pick, knob by knob, the candidate value with the smallest median time of ``run``."""
    timer = timer or cuda_timer
    if warmup < 0 or repeats < 1:
        raise ValueError("warmup >= 0 and repeats >= 1 are required")
    best = current()
    table: List[Tuple[str, int, float]] = []
    for name, values in candidates.items():
        if name not in KNOBS:
            raise KeyError("unknown knob %r" % name)
        vals = list(dict.fromkeys(int(v) for v in values))
        if not vals:
            continue
        scores = []
        for v in vals:
            apply({**best, name: v})
            for _ in range(warmup):
                run()
            ms = statistics.median(timer(run) for _ in range(repeats))
            table.append((name, v, ms))
            scores.append((ms, vals.index(v), v))
        best[name] = min(scores)[2]  # ties: the earlier candidate
    apply(best)
    return TuneResult(best=best, table=table)


def save(path: str, key: str, values: Dict[str, int]) -> None:
    """Record ``values`` under ``key`` in the JSON file at ``path`` (other keys are kept)."""
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    data[key] = {k: int(v) for k, v in values.items()}
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def load(path: str, key: str) -> Optional[Dict[str, int]]:
    """The values recorded under ``key``, or None."""
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f).get(key)
