"""Autotuner of the walk's schedule parameters.

The walk of the filter stage has parameters that change its speed but never
its output: the walk mode (two launches with fixed hit ranges, one
persistent launch fed by a device work counter, or the speculative window
walk), the lane cap (bases a lane scores on one side before it hands the
diagonal to a warp), the hits per chunk of the persistent walk and the chunk
order (the diagonal-bin schedule), and the lanes per hit of the speculative
walk (32 / spec_window: one warp, a group or one lane per hit). `tune` times every
candidate of a search space on the caller's own workload with CUDA events,
checks that every candidate returns the same HSP list, byte for byte, and
keeps the fastest. Results are cached in a JSON file keyed by the GPU, the
library build and a signature of the workload, so a workload of the same
shape is tuned once.

The caller supplies `run(params) -> (hsp bytes, stats)`, which runs the
library once with those parameters on the stream `stream`; this module only
times and compares.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os
import time

from . import sfe

# name -> candidate values; entries that make no sense together are skipped
DEFAULT_SPACE = {
    "walk_mode": [sfe.WALK_TWO_LAUNCHES, sfe.WALK_PERSISTENT, sfe.WALK_SPECULATIVE],
    "lane_cap": [64, 128, 256],
    "walk_chunk": [32, 128],
    "walk_schedule": [sfe.SCHED_NATURAL, sfe.SCHED_LARGEST_FIRST],
    # lanes per hit of the speculative walk: 32 / spec_window
    "spec_window": [4, 1, 32],
}


def cache_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "sfe_autotune.json")


def _library_id() -> str:
    h = hashlib.sha256()
    with open(sfe.LIB_PATH, "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def candidates(space: dict) -> list[dict]:
    keys = list(space)
    out = []
    def first(c, k):  # the parameter takes only the space's first value
        return k not in c or c[k] == space[k][0]

    for vals in itertools.product(*(space[k] for k in keys)):
        c = dict(zip(keys, vals))
        mode = c.get("walk_mode", sfe.WALK_TWO_LAUNCHES)
        if mode != sfe.WALK_PERSISTENT:
            # chunk sizes and their order belong to the persistent walk only
            if c.get("walk_schedule", sfe.SCHED_NATURAL) != sfe.SCHED_NATURAL:
                continue
            if not first(c, "walk_chunk"):
                continue
            c.pop("walk_chunk", None)
        if mode == sfe.WALK_SPECULATIVE:
            # lanes per hit come from the window; no lane tier, no hand-off
            if not first(c, "lane_cap"):
                continue
            c.pop("lane_cap", None)
        elif not first(c, "spec_window"):
            continue
        else:
            c.pop("spec_window", None)
        out.append(c)
    return out


def tune(run, signature: str, space: dict | None = None, reps: int = 3, stream=None,
         cache: str | None = None, force: bool = False) -> tuple[dict, list]:
    """Best parameters (a dict of sfe_params fields) for the workload `run`
    executes, and the timing table [(params, median ms)]. `signature` names the
    workload's shape (sizes, pair lengths, seed pattern)."""
    import torch
    space = space or DEFAULT_SPACE
    dev = torch.cuda.current_device()
    key = "|".join([torch.cuda.get_device_name(dev), _library_id(), signature,
                    json.dumps(space, sort_keys=True)])
    cache = cache or cache_path()
    db = {}
    if os.path.exists(cache):
        try:
            with open(cache) as f:
                db = json.load(f)
        except (OSError, ValueError):
            db = {}
    if not force and key in db:
        e = db[key]
        return e["best"], [(t["params"], t["ms"]) for t in e["table"]]
    stream = stream or torch.cuda.current_stream()
    ref = None
    table = []
    for c in candidates(space):
        ms = []
        for r in range(reps + 1):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out, _ = run(c)
            e1.record(stream)
            torch.cuda.synchronize()
            if ref is None:
                ref = out
            elif out != ref:
                raise RuntimeError(f"autotune: parameters {c} changed the HSP list")
            if r > 0:  # the first run of a candidate warms it up
                ms.append(e0.elapsed_time(e1))
        ms.sort()
        table.append((c, ms[len(ms) // 2]))
    best = min(table, key=lambda t: t[1])[0]
    db[key] = {"best": best, "table": [{"params": p, "ms": m} for p, m in table],
               "when": time.strftime("%Y-%m-%d %H:%M:%S")}
    os.makedirs(os.path.dirname(cache), exist_ok=True)
    tmp = cache + ".tmp"
    with open(tmp, "w") as f:
        json.dump(db, f, indent=1, sort_keys=True)
    os.replace(tmp, cache)
    return best, table


def batch_signature(toff, qoff, params) -> str:
    """Shape of a batch: its pair lengths and the seed, hashed."""
    import numpy as np
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(toff, dtype=np.int64).tobytes())
    h.update(np.ascontiguousarray(qoff, dtype=np.int64).tobytes())
    h.update(bytes(params.seed_pattern or b""))
    h.update(str((params.transition, params.strands, params.xdrop)).encode())
    return f"batch:{len(toff) - 1}:{h.hexdigest()[:16]}"
