#!/usr/bin/env python
"""Throughput of the filter stage (spaced-seed hits -> per-diagonal skip ->
ungapped X-drop -> sorted HSPs) on one or more GB300s.

One step = one whole pass of the stage over the 10 Mb x 10 Mb plain workload
(41% GC, 5% repeats, 2000 planted blocks, both strands, 12of19 seed with one
transition, HOXD70, X = 910, threshold 3000): pack, index build, hit count and
write, diagonal grouping, lane and warp walks, HSP sort. Inputs (ASCII bytes)
are resident in HBM when the timed region starts; each step is timed with CUDA
events on the library's stream, with a 256 MiB write between steps to flush L2.

Prints one JSON line (rank 0). `value` is GCUPS of the plain path (the
library's defaults): the oracle-defined cells (seed span plus bases scored on
both sides of every extended hit) per second. `learned_binned` times the same
steps with the persistent walk taking its chunks of hits in the order of the
work predictor (trained first, on the extension log of a plain run of the
same generator at another seed) and checks that its HSP list is byte-identical
to the plain path's. `--impl reference` times the CPU oracle instead on a
bounded sample of the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("ungapped X-drop GCUPS (oracle-defined cells/s), HSPs/s and hits/s; "
          "learned-binned vs plain, bit-exact")
WORKLOAD = "plain_pair_10mb"
OPS_PER_CELL = 4  # score lookup, add, running max, X-drop compare
L2_FLUSH_BYTES = 256 << 20


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sfe", choices=["sfe", "reference"])
    ap.add_argument("--seed", type=int, default=None,
                    help="generator seed (default 2; 5 for large_pair_100mb)")
    ap.add_argument("--scale", type=float, default=1.0, help="workload scale (1.0 = 10 Mb)")
    ap.add_argument("--lane-cap", type=int, default=0)
    ap.add_argument("--tile-hits", type=int, default=0)
    ap.add_argument("--walk-mode", type=int, default=None,
                    help="0: two launches, 1: persistent (default: the library's)")
    ap.add_argument("--walk-chunk", type=int, default=0)
    ap.add_argument("--no-cell-planes", action="store_true",
                    help="lane windows read the 2-bit words (an ablation)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target CPU time of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-binned arm (predictor training and its timed steps)")
    ap.add_argument("--train-seed", type=int, default=100,
                    help="generator seed of the predictor's training pair")
    ap.add_argument("--log-every", type=int, default=20,
                    help="extension log sampling of the training run (1 in N)")
    ap.add_argument("--learned-chunk", type=int, default=64)
    ap.add_argument("--workload", default="plain_pair_10mb",
                    choices=["plain_pair_10mb", "batch_pairs", "large_pair_100mb"],
                    help="batch_pairs: 4096 uneven pairs, eager and as a replayed CUDA graph "
                         "(a separate line, not the headline)")
    ap.add_argument("--pairs", type=int, default=4096)
    ap.add_argument("--no-tune", action="store_true", help="batch: skip the autotuner")
    ap.add_argument("--no-sublines", action="store_true",
                    help="skip the batch and 100 Mb sub-measurements of the default run")
    ap.add_argument("--sub-steps", type=int, default=3)
    ap.add_argument("--sub-warmup", type=int, default=3)
    a = ap.parse_args()
    if a.seed is None:
        a.seed = 5 if a.workload == "large_pair_100mb" else 2
    if a.workload == "large_pair_100mb":  # a separate line: no oracle sample, no predictor
        a.no_learned = a.no_cpu_baseline = True
    if a.scale != 1.0:
        a.no_sublines = True
    return a


# --------------------------------------------------------------- helpers

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def reduce_over_ranks(dist, device, ms: float, counts: list) -> tuple[float, list]:
    """Replicas: the job takes as long as its slowest rank (max of the timed
    milliseconds) and does the work of all ranks (sum of the counts)."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(x) for x in counts], dtype=torch.float64, device=device)
    dist.all_reduce(c)
    return float(t.item()), [float(x) for x in c.tolist()]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}


def alu_peak_tops(sm_count: int, sm_mhz: float) -> float:
    """Issue-limited int32 peak: every SM issues one warp instruction per clock on each
    of its 4 sub-partitions, 32 lanes each (128 lane-ops per SM per clock)."""
    return sm_count * 128 * sm_mhz * 1e6 / 1e12


def kernel_traffic(kernel: str) -> float | None:
    """DRAM bytes per launch from the committed ncu summary of `kernel`, if the kernel's
    source has not changed since (the summary records the source hash)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_plain_pair_10mb.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"source_sha256:\s*([0-9a-f]{64})", txt)
    t = re.search(r"dram_bytes_per_launch_full:\s*([0-9.eE+]+)", txt)
    src = os.path.join(ROOT, "paper_2606_06811_gb300", "csrc", "xdrop.cu")
    if not (m and t and os.path.exists(src)):
        return None
    if hashlib.sha256(open(src, "rb").read()).hexdigest() != m.group(1):
        return None
    return float(t.group(1))


def radix_passes(nbits: int) -> int:
    """Passes of the library's LSD radix sort over an nbits-wide key: as few as
    9-bit digits allow, or 10-bit ones where that saves a pass."""
    if nbits <= 0:
        return 0
    return min((nbits + 8) // 9, (nbits + 9) // 10)


def stage_rooflines(st: dict, stage_ms: dict, tlen: int, qlen: int, weight: int, strands: int,
                    hbm_gbs: float) -> dict:
    """Achieved HBM bandwidth of the memory-bound stages from their algorithmic
    bytes per step (the minimum each stage must move; re-reads are not counted):
      index: per target position, the 8-byte key written, 16 B per radix pass
        (read + write), 12 B of CSR work (key read, position written), and
        8 B per merged probe-set entry (1 + weight per position: position read,
        entry written); plus six 4-byte sweeps of the 4^weight-entry tables;
      count: per query position and strand, the 4-byte table word read, the
        count written and its 8-byte scan written;
      write: per hit, the 4-byte merged-list entry read and the 8-byte hit written;
      sort: per hit, 16 B per radix pass over the bits_for(tlen + qlen)-bit
        diagonal word (each 8-byte key read and written once)."""
    npos = max(0, tlen - (19 - 1))
    nq = max(0, qlen - (19 - 1)) * strands
    dbits = max(1, (tlen + qlen).bit_length())
    hits = st["hits"]
    algo = {
        "index": npos * (8 + 16 * radix_passes(2 * weight) + 12 + 8 * (1 + weight))
        + 6 * 4 * (4 ** weight),
        "count": nq * 16,
        "write": hits * 12,
        "sort": hits * 16 * radix_passes(dbits),
    }
    out = {}
    for k, b in algo.items():
        ms = stage_ms.get(k, 0.0)
        if ms <= 0:
            continue
        gbs = b / (ms / 1e3) / 1e9
        out[k] = {"bound": "hbm", "algorithmic_bytes": int(b), "ms": round(ms, 4),
                  "achieved": round(gbs, 1), "peak": hbm_gbs, "unit": "GB/s",
                  "frac": round(gbs / hbm_gbs, 4)}
    return out


# ------------------------------------------------------------ workloads

def make_workload(seed: int, scale: float, name: str = WORKLOAD):
    import synth
    pair = getattr(synth, name)(seed, scale=scale)
    return pair, np.frombuffer(synth.decode(pair.T), np.uint8), np.frombuffer(
        synth.decode(pair.Q), np.uint8)


def oracle_sample(pair, seconds: float):
    """Time the CPU oracle, as it stands, on the full target against a query prefix
    sized so the run takes about `seconds`. Returns (cells, hsps, hits, secs, qlen)."""
    import oracle
    qlen = min(pair.qlen, 20_000)
    while True:
        t0 = time.perf_counter()
        r = oracle.run(pair.T, pair.Q[:qlen])
        dt = time.perf_counter() - t0
        if dt >= 0.6 * seconds or qlen >= pair.qlen:
            return r.cells, int(r.hsps.size), r.hits, dt, qlen
        grow = max(2.0, 0.9 * seconds / max(dt, 1e-3))
        qlen = int(min(pair.qlen, qlen * grow))


def oracle_sample_cores(pair, qlen: int, reps: int = 1):
    """The oracle's multi-threaded form on every host core, on the same sample
    (full target x query prefix of qlen). Returns (cells, hsps, hits, secs, cores)."""
    import oracle
    cores = oracle.host_cores()
    secs, r = 0.0, None
    for _ in range(reps):
        t0 = time.perf_counter()
        r = oracle.run_par(pair.T, pair.Q[:qlen], threads=cores)
        secs += time.perf_counter() - t0
    return r.cells * reps, int(r.hsps.size) * reps, r.hits * reps, secs, cores


def cpu_baseline_line(pair, seconds: float) -> dict:
    """The oracle on the machine's host cores: one thread, and every core, on the
    same query prefix of the same pair."""
    c1, h1, ht1, dt1, qlen = oracle_sample(pair, seconds)
    reps = 3
    cn, hn, htn, dtn, cores = oracle_sample_cores(pair, qlen, reps)
    sample = (f"full {pair.tlen:,} bp target x {qlen:,} bp query prefix, both strands")
    return {"value": cn / dtn / 1e9, "unit": "GCUPS", "cores": cores, "kind": "oracle",
            "sample": f"{sample}; multi-threaded form on {cores} cores, {reps} runs, "
                      f"{dtn:.1f} s",
            "single_core": {"value": c1 / dt1 / 1e9, "unit": "GCUPS", "cores": 1,
                            "sample": f"{sample}; serial form, {dt1:.1f} s"},
            "hsps_per_s": hn / dtn, "hits_per_s": htn / dtn}


# ------------------------------------------------------------------ arms

def run_reference(a, rank, world):
    if rank != 0:
        return 0
    import oracle
    pair, _, _ = make_workload(a.seed, a.scale)
    cores = oracle.host_cores()
    # each step times the oracle's multi-threaded form on every host core over
    # the full target and a query prefix, sized so the whole run (warm-up and
    # timed steps) takes about 10 x --cpu-seconds (150 s by default)
    a_total = 10.0 * a.cpu_seconds
    per = max(1.0, a_total / max(1, a.steps + a.warmup))
    qlen = min(pair.qlen, 200_000)
    while True:
        t0 = time.perf_counter()
        oracle.run_par(pair.T, pair.Q[:qlen], threads=cores)
        dt = time.perf_counter() - t0
        if dt >= 0.6 * per or qlen >= pair.qlen:
            break
        qlen = int(min(pair.qlen, qlen * max(1.5, 0.9 * per / max(dt, 1e-3))))
    cells = hsps = hits = 0
    secs = 0.0
    for i in range(a.warmup + a.steps):
        t0 = time.perf_counter()
        r = oracle.run_par(pair.T, pair.Q[:qlen], threads=cores)
        dt = time.perf_counter() - t0
        if i >= a.warmup:
            cells += r.cells
            hsps += int(r.hsps.size)
            hits += r.hits
            secs += dt
    gcups = cells / secs / 1e9
    sample = (f"full {pair.tlen:,} bp target x {qlen:,} bp query prefix of {WORKLOAD}, "
              f"both strands, per step; the oracle's multi-threaded form on {cores} cores")
    line = {
        "impl": "reference", "metric": METRIC, "value": gcups, "unit": "GCUPS",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": secs / a.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "tlen": pair.tlen, "qlen_sample": qlen,
                   "seed_pattern": "1110100110010101111", "transition": 1, "strands": 2,
                   "xdrop": 910, "hsp_thresh": 3000},
        "hsps_per_s": hsps / secs, "hits_per_s": hits / secs,
        "cpu_baseline": {"value": gcups, "unit": "GCUPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": gcups, "unit": "GCUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def train_predictor(a, pkg, ctx, dev):
    """Train the work predictor on a plain run of the same generator at another
    seed; returns (predictor, info)."""
    import torch
    from paper_2606_06811_gb300 import predictor
    t0 = time.perf_counter()
    tr = make_workload(a.train_seed, a.scale)[0]
    recs, _ = predictor.collect(ctx, tr.T, tr.Q, a.log_every, cap=1 << 24,
                                params=pkg.default_params(input_codes=1))
    data = predictor.training_data(ctx, [(tr.T, tr.Q, recs)])
    t1 = time.perf_counter()
    pred = predictor.train(ctx, data, epochs=2, batch=8192, lr=2e-3, seed=3)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    info = {"train_workload": f"{WORKLOAD} seed {a.train_seed}", "samples": int(data.n),
            "log_every": a.log_every, "epochs": 2, "batch": 8192, "lr": 2e-3,
            "train_loss": [round(x, 5) for x in pred.history],
            "collect_s": round(t1 - t0, 3), "train_s": round(t2 - t1, 3)}
    data.close()
    return pred, info


def predictor_r2(a, pkg, ctx, pred, pair) -> dict:
    """Accuracy of the FP16 predictor on the benchmark pair's own extensions."""
    import torch
    from paper_2606_06811_gb300 import predictor
    recs, _ = predictor.collect(ctx, pair.T, pair.Q, a.log_every, cap=1 << 24,
                                params=pkg.default_params(input_codes=1))
    data = predictor.training_data(ctx, [(pair.T, pair.Q, recs)])
    out = torch.zeros(data.n, dtype=torch.float32, device=recs.device)
    ctx.mlp_predict(data, pred.model, out)
    y = torch.log1p((recs[:, 4] + recs[:, 5]).double())
    mse = float(((out.double() - y) ** 2).mean())
    var = float(y.var(unbiased=False))
    data.close()
    return {"eval_samples": int(y.numel()), "mse": round(mse, 5), "target_var": round(var, 5),
            "r2": round(1 - mse / var, 4)}


def run_sfe(a, rank, world, local):
    import torch
    import paper_2606_06811_gb300 as pkg
    from paper_2606_06811_gb300 import build as cuda_build

    cuda_build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    pair, Ta, Qa = make_workload(a.seed, a.scale, a.workload)
    T = torch.from_numpy(Ta.copy()).to(dev)
    Q = torch.from_numpy(Qa.copy()).to(dev)
    stream = torch.cuda.Stream(device=dev)
    ctx = pkg.Context(local, stream=stream)
    walk = {} if a.walk_mode is None else {"walk_mode": a.walk_mode}
    if a.walk_chunk:
        walk["walk_chunk"] = a.walk_chunk
    base_flags = pkg.TIME_STAGES | (pkg.NO_CELL_PLANES if a.no_cell_planes else 0)
    params = pkg.default_params(flags=base_flags, lane_cap=a.lane_cap,
                                tile_hits=a.tile_hits, **walk)
    cap = 1 << 22
    out = torch.zeros((cap, 5), dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count

    def step(prm=params):
        with torch.cuda.stream(stream):
            flush.fill_(1)  # evicts L2 between steps, outside the events
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hs, st = ctx.run(T, Q, prm, out=out)
        e1.record(stream)
        return e0, e1, st, int(hs.shape[0])

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    recs = [step() for _ in range(a.steps)]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall = time.perf_counter() - w0
    clk = clocks.stop()

    step_ms = [e0.elapsed_time(e1) for e0, e1, _, _ in recs]
    total_ms = float(sum(step_ms))
    stats = [st for _, _, st, _ in recs]
    cells = sum(s["cells"] for s in stats)
    hsps = sum(n for *_, n in recs)
    hits = sum(s["hits"] for s in stats)
    launches = sum(s["launches"] for s in stats)
    stage_ms = {k: sum(s["stage_ms"][k] for s in stats) / a.steps for k in pkg.STAGES}
    stage_launch = {k: sum(s["stage_launches"][k] for s in stats) / a.steps for k in pkg.STAGES}

    if dist:
        total_ms, (cells, hsps, hits) = reduce_over_ranks(dist, dev, total_ms,
                                                          [cells, hsps, hits])

    secs = total_ms / 1e3
    gcups = cells / secs / 1e9
    s0 = stats[0]

    # dominant kernel: the lane walk (skip + X-drop), integer-ALU bound
    peaks = measured_peaks()
    lane_ms = stage_ms["walk_lanes"] / max(1.0, stage_launch["walk_lanes"])
    # the persistent walk scores the warp tier's cells in the same launch (its
    # follow-up warp launch only walks entries left by consumers that gave up)
    persistent = a.walk_mode in (None, 1)
    lane_cells = (s0["cells"] - (0 if persistent else s0["warp_cells"])) / \
        max(1.0, stage_launch["walk_lanes"])
    achieved = lane_cells * OPS_PER_CELL / (lane_ms / 1e3) / 1e12
    peak = alu_peak_tops(sm_count, peaks["sm_max_mhz"])
    roofline = {"kernel": "walk_lanes_kernel", "bound": "alu", "achieved": achieved,
                "peak": peak, "unit": "Tops/s (int32)", "frac": achieved / peak,
                "traffic": kernel_traffic("walk_lanes"),
                "peak_source": (f"{sm_count} SMs x 128 int32 lanes/clk x "
                                f"{peaks['sm_max_mhz']:.0f} MHz (issue limit)"),
                "ops_per_cell": OPS_PER_CELL,
                "ms_per_launch": lane_ms, "launches_per_step": stage_launch["walk_lanes"]}
    dom = max(stage_ms, key=stage_ms.get)
    stages_hbm = stage_rooflines(s0, stage_ms, pair.tlen, pair.qlen, 12, 2, peaks["hbm_gbs"])

    line = {
        "metric": METRIC, "value": gcups, "unit": "GCUPS", "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": total_ms / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": a.workload, "seed": a.seed, "tlen": pair.tlen, "qlen": pair.qlen,
                   "seed_pattern": "1110100110010101111", "transition": 1, "strands": 2,
                   "scores": "HOXD70", "xdrop": 910, "hsp_thresh": 3000,
                   "lane_cap": a.lane_cap or "default", "walk": walk or "default",
                   "cell_planes": not a.no_cell_planes,
                   "parallelism": f"replicas{world}",
                   "l2": "256 MiB write between steps, outside the per-step events",
                   "input": "ASCII bytes resident in HBM"},
        "hsps_per_s": hsps / secs, "hits_per_s": hits / secs,
        "per_step": {"cells": s0["cells"], "hits": s0["hits"], "extended": s0["extended"],
                     "hsps": recs[0][3], "warp_tasks": s0["warp_tasks"],
                     "warp_cells": s0["warp_cells"], "tiles": s0["tiles"],
                     "shadow_cells": s0["shadow_cells"],
                     "shadow_fraction": s0["shadow_cells"] / max(1, s0["cells"])},
        "stage_ms": {k: round(v, 4) for k, v in stage_ms.items()},
        "dominant_stage": dom,
        "roofline": roofline,
        "stage_roofline": stages_hbm,
        "gpu_launches": int(launches),
        "clocks": clk,
        "wall_s": wall,
    }

    if not a.no_learned:
        # learned-binned arm: persistent walk, chunks ordered by predicted work
        plain_out = out[: recs[0][3]].clone()
        pred, info = train_predictor(a, pkg, ctx, dev)
        lp = pkg.default_params(flags=base_flags, lane_cap=a.lane_cap,
                                tile_hits=a.tile_hits, walk_mode=pkg.WALK_PERSISTENT,
                                walk_schedule=pkg.SCHED_PREDICTED, walk_chunk=a.learned_chunk,
                                model=pred.model.data_ptr())
        for _ in range(a.warmup):
            step(lp)
        torch.cuda.synchronize()
        lrecs = [step(lp) for _ in range(a.steps)]
        torch.cuda.synchronize()
        l_ms = [e0.elapsed_time(e1) for e0, e1, _, _ in lrecs]
        lst = [st for _, _, st, _ in lrecs]
        l_cells = sum(x["cells"] for x in lst)
        same = (lrecs[-1][3] == plain_out.shape[0] and
                torch.equal(out[: lrecs[-1][3]], plain_out))
        line["learned_binned"] = {
            "value": l_cells / (sum(l_ms) / 1e3) / 1e9, "unit": "GCUPS",
            "ms_per_step": sum(l_ms) / a.steps,
            "bit_exact_vs_plain": bool(same),
            "hsps_per_s": sum(n for *_, n in lrecs) / (sum(l_ms) / 1e3),
            "walk": f"persistent, chunks of {a.learned_chunk} hits ordered by predicted work",
            "stage_ms": {k: round(sum(x["stage_ms"][k] for x in lst) / a.steps, 4)
                         for k in pkg.STAGES},
            "predictor": dict(info, **predictor_r2(a, pkg, ctx, pred, pair)),
        }

    if not a.no_e2e:
        Th = torch.from_numpy(Ta.copy()).pin_memory()
        Qh = torch.from_numpy(Qa.copy()).pin_memory()
        hout = np.zeros(cap, dtype=pkg.HSP_DTYPE)
        pe = pkg.default_params(lane_cap=a.lane_cap, tile_hits=a.tile_hits, **walk)
        ctx.run(Th, Qh, pe, out=hout)  # warm the host path
        ts = []
        e_cells = 0
        nh = 0
        for _ in range(a.steps):
            t0 = time.perf_counter()
            hs, st = ctx.run(Th, Qh, pe, out=hout)  # H2D inside, HSPs read back to host
            ts.append(time.perf_counter() - t0)
            e_cells += st["cells"]
            nh = int(hs.shape[0])
        line["e2e"] = {"value": e_cells / sum(ts) / 1e9, "unit": "GCUPS",
                       "h2d_bytes_per_step": int(Ta.size + Qa.size),
                       "d2h_bytes_per_step": int(nh * 20 + 8 * 24),
                       "path": "sfe_run with pinned host buffers (host wall clock)"}

    if a.workload == WORKLOAD and not a.no_sublines:
        torch.cuda.synchronize()
        line["seeds"] = run_seed_sweep(a, ctx, T, Q, pair, out, step)
        line["speculative_window"] = run_spec_study(a, ctx, T, Q, pair)
        hs_plain, _ = ctx.run(T, Q, pkg.default_params(), out=out)
        line["gapped"] = run_gapped_study(a, ctx, T, Q, pair, hs_plain.clone())
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_line(pair, a.cpu_seconds)
    ctx.close()
    if a.workload == WORKLOAD and not a.no_sublines:
        # the other configurations, each in its own sub-object (fewer steps)
        del out, flush
        torch.cuda.empty_cache()
        sub = argparse.Namespace(**vars(a))
        sub.steps, sub.warmup = a.sub_steps, max(3, a.sub_warmup)
        line["batch_pairs"] = run_batch_bench(sub, rank, world, local, emit=False)
        torch.cuda.empty_cache()
        line["ydrop_filter"] = run_ydrop_filter_study(sub, local)
        torch.cuda.empty_cache()
        sub.seed = 5
        line["large_pair_100mb"] = run_large(sub, local)
        torch.cuda.empty_cache()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_batch_bench(a, rank, world, local, emit: bool = True):
    """The batch of uneven pairs: autotuned walk parameters, then eager calls
    (sfe_run_batch) and replays of the captured graph (sfe_batch_plan_run)."""
    import torch
    import synth
    from synth.workloads import concat_batch
    import paper_2606_06811_gb300 as pkg
    from paper_2606_06811_gb300 import autotune
    from paper_2606_06811_gb300 import build as cuda_build

    cuda_build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t0 = time.perf_counter()
    pairs = synth.batch_pairs(seed=3, n_pairs=a.pairs)
    Tc, toff, Qc, qoff = concat_batch(pairs)
    gen_s = time.perf_counter() - t0
    T = torch.from_numpy(np.frombuffer(synth.decode(Tc), np.uint8).copy()).to(dev)
    Q = torch.from_numpy(np.frombuffer(synth.decode(Qc), np.uint8).copy()).to(dev)
    stream = torch.cuda.Stream(device=dev)
    ctx = pkg.Context(local, stream=stream)
    cap = 1 << 22
    out = torch.zeros((cap, 6), dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    base = pkg.default_params()
    tuned, table = {}, []
    if not a.no_tune:
        def trial(c):
            h, st = ctx.run_batch(T, toff, Q, qoff, pkg.default_params(**c), out=out)
            return h.cpu().numpy().tobytes(), st
        with torch.cuda.stream(stream):
            tuned, table = autotune.tune(trial, autotune.batch_signature(toff, qoff, base),
                                         stream=stream)
    params = pkg.default_params(**tuned)

    def timed(fn):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h, st = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), st, h

    eager = lambda: ctx.run_batch(T, toff, Q, qoff, params, out=out)  # noqa: E731
    plan = ctx.batch_plan(toff, qoff, params)
    pout = torch.zeros_like(out)
    replay = lambda: plan.run(T, Q, out=pout)  # noqa: E731
    for _ in range(a.warmup):
        timed(eager)
        timed(replay)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    res = {"eager": [], "graph": []}
    last = {}
    for _ in range(a.steps):
        for name, fn in (("eager", eager), ("graph", replay)):
            ms, st, h = timed(fn)
            res[name].append((ms, st))
            last[name] = h
    clk = clocks.stop()
    same = bool(torch.equal(last["eager"], last["graph"]))
    st_t = ctx.run_batch(T, toff, Q, qoff, pkg.default_params(flags=pkg.TIME_STAGES, **tuned),
                         out=out)[1]

    def summary(rows):
        ms = sum(r[0] for r in rows)
        cells = sum(r[1]["cells"] for r in rows)
        return {"value": cells / (ms / 1e3) / 1e9, "unit": "GCUPS",
                "ms_per_step": ms / len(rows),
                "hsps_per_s": rows[0][1]["hsps"] * len(rows) / (ms / 1e3),
                "launches_per_step": rows[0][1]["launches"]}

    g = summary(res["graph"])
    s0 = res["graph"][0][1]
    line = {
        "metric": METRIC, "value": g["value"], "unit": "GCUPS", "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": g["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": "batch_pairs", "pairs": a.pairs, "seed": 3,
                   "tbases": int(toff[-1]), "qbases": int(qoff[-1]),
                   "path": "sfe_batch_plan_run (captured CUDA graph)", "walk": tuned or "defaults",
                   "l2": "256 MiB write between steps, outside the per-step events"},
        "per_step": {"cells": s0["cells"], "hits": s0["hits"], "extended": s0["extended"],
                     "hsps": s0["hsps"]},
        "eager": summary(res["eager"]),
        "graph_equals_eager": same,
        "stage_ms_eager": {k: round(v, 4) for k, v in st_t["stage_ms"].items()},
        "autotune": [{"params": p, "ms": round(m, 3)} for p, m in table],
        "gpu_launches": int(sum(r[1]["launches"] for r in res["graph"])),
        "clocks": clk, "generate_s": round(gen_s, 2),
    }
    plan.close()
    ctx.close()
    if not emit:
        return line
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


P22 = "1110111000011101011011"  # this build's 14-of-22 mask (Section 7 names the weight)
SEED_SWEEP = [("1110100110010101111", 1), ("1110100110010101111", 2), (P22, 1), (P22, 2),
              (P22, 4)]


def block_recovery(pair, H) -> dict:
    """Planted homologous blocks found by an HSP: on the block's strand, overlapping
    its target range, on a diagonal within 50 + 3% of its length of the block's
    (indels drift the diagonal). Returns the fraction of blocks with such an HSP
    and the fraction of the blocks' target bases such HSPs cover."""
    if not pair.blocks or H.shape[0] == 0:
        return {"blocks": len(pair.blocks), "blocks_found": 0.0, "block_bases_covered": 0.0}
    s, t0, q0, ln = (H[:, k].astype(np.int64) for k in range(4))
    found, covered, total = 0, 0, 0
    maxlen = int(ln.max())
    for b in pair.blocks:
        strand = 1 if b.rc else 0
        qb = (pair.qlen - b.qstart - b.qlen) if b.rc else b.qstart
        d0, tol = b.tstart - qb, 50 + 0.03 * b.tlen
        lo = np.searchsorted(s * (1 << 40) + t0, strand * (1 << 40) + b.tstart - maxlen)
        hi = np.searchsorted(s * (1 << 40) + t0, strand * (1 << 40) + b.tstart + b.tlen)
        sel = np.arange(lo, hi)
        sel = sel[(t0[sel] + ln[sel] > b.tstart) & (np.abs(t0[sel] - q0[sel] - d0) <= tol)]
        total += b.tlen
        if sel.size == 0:
            continue
        found += 1
        a = np.maximum(t0[sel], b.tstart)
        e = np.minimum(t0[sel] + ln[sel], b.tstart + b.tlen)
        order = np.argsort(a)
        a, e = a[order], e[order]
        run_end, cov = -1, 0
        for x, y in zip(a.tolist(), e.tolist()):
            if y <= run_end:
                continue
            cov += y - max(x, run_end)
            run_end = y
        covered += cov
    return {"blocks": len(pair.blocks), "blocks_found": found / len(pair.blocks),
            "block_bases_covered": covered / max(1, total)}


def run_seed_sweep(a, ctx, T, Q, pair, out, step_fn) -> list:
    """Section 7: heavier seeds and a larger step against 12of19 with step 1, on
    the same pair: hits, cells, HSPs, time per step and planted-block recovery."""
    import paper_2606_06811_gb300 as pkg
    rows = []
    for pattern, step in SEED_SWEEP:
        prm = pkg.default_params(flags=pkg.TIME_STAGES, seed_pattern=pattern, step=step)
        for _ in range(a.sub_warmup):
            step_fn(prm)
        recs = [step_fn(prm) for _ in range(a.sub_steps)]
        ms = sum(e0.elapsed_time(e1) for e0, e1, _, _ in recs) / len(recs)
        st, n = recs[-1][2], recs[-1][3]
        H = out[:n].cpu().numpy()
        rows.append({"seed": pattern, "weight": pattern.count("1"), "span": len(pattern),
                     "step": step, "ms_per_step": round(ms, 3),
                     "gcups": st["cells"] / (ms / 1e3) / 1e9, "hits": st["hits"],
                     "extended": st["extended"], "cells": st["cells"], "hsps": n,
                     "stage_ms": {k: round(v, 3) for k, v in st["stage_ms"].items()},
                     **block_recovery(pair, H)})
    base = rows[0]
    for r in rows:
        r["speedup_vs_12of19_step1"] = round(base["ms_per_step"] / r["ms_per_step"], 3)
        r["block_bases_vs_12of19_step1"] = round(
            r["block_bases_covered"] / max(1e-12, base["block_bases_covered"]), 4)
    return rows


SPEC_WINDOWS = [1, 2, 4, 8, 16, 32]
GAPPED_BATCHES = [64, 1024, 16384, 0]


def gapped_recovery(pair, A) -> dict:
    """Planted blocks covered by gapped alignments (boxes): on the block's
    strand, overlapping its target range, with the box's start or end diagonal
    within 50 + 3% of the block's length of the block's diagonal."""
    total, covered, found = 0, 0, 0
    for b in pair.blocks:
        strand = 1 if b.rc else 0
        qb = (pair.qlen - b.qstart - b.qlen) if b.rc else b.qstart
        d0, tol = b.tstart - qb, 50 + 0.03 * b.tlen
        m = ((A["strand"] == strand) & (A["tstart"] < b.tstart + b.tlen) & (A["tend"] > b.tstart) &
             ((np.abs(A["tstart"] - A["qstart"] - d0) <= tol) |
              (np.abs(A["tend"] - A["qend"] - d0) <= tol)))
        total += b.tlen
        if not m.any():
            continue
        found += 1
        iv = sorted(zip(np.maximum(A["tstart"][m], b.tstart).tolist(),
                        np.minimum(A["tend"][m], b.tstart + b.tlen).tolist()))
        end, cov = -1, 0
        for x, y in iv:
            if y > end:
                cov += y - max(x, end)
                end = y
        covered += cov
    return {"blocks_found": found / max(1, len(pair.blocks)),
            "block_bases_covered": covered / max(1, total)}


def run_gapped_study(a, ctx, T, Q, pair, hsps) -> dict:
    """The gapped Y-drop stage after the filter (Algorithm 1 / 3) on the pair's
    HSPs: time, shadow work and planted-block recovery against the batch size."""
    import paper_2606_06811_gb300 as pkg
    rows = []
    for K in GAPPED_BATCHES:
        prm = pkg.ydrop_params(batch=K)
        for _ in range(1):
            A, st = ctx.gapped_extend(T, Q, hsps, prm)
        A, st = ctx.gapped_extend(T, Q, hsps, prm)
        work = st["cells"] + st["shadow_cells"]
        rows.append({"batch": K if K else "all", "device_ms": round(st["device_ms"], 3),
                     "total_ms": round(st["total_ms"], 3), "batches": st["batches"],
                     "extended": st["extended"], "skipped": st["skipped"],
                     "shadow": st["shadow"], "shadow_fraction": st["shadow_cells"] / max(1, work),
                     "cells": st["cells"], "committed": st["committed"],
                     "gcups_device": work / max(1e-9, st["device_ms"] / 1e3) / 1e9,
                     **gapped_recovery(pair, A)})
    return {"anchors": int(hsps.shape[0]), "gap_open": 400, "gap_extend": 30, "ydrop": 9400,
            "gapped_thresh": 3000, "band": 256, "rows": rows,
            "ungapped_hsps": block_recovery(pair, hsps.cpu().numpy())}


def run_ydrop_filter_study(a, local) -> dict:
    """Y-drop as the filter (Darwin-WGA's idea, the paper's closing section): the
    seed hits of a 1 Mb pair of the 10 Mb generator extended directly by the 2-D
    Y-drop (Y = X = 910, threshold 3000) against the X-drop filter followed by the
    gapped stage (Y = 9400), both through the same kernels."""
    import torch
    import paper_2606_06811_gb300 as pkg
    dev = torch.device("cuda", local)
    pair, Ta, Qa = make_workload(2, 0.1)
    T = torch.from_numpy(Ta.copy()).to(dev)
    Q = torch.from_numpy(Qa.copy()).to(dev)
    res = {"workload": "plain_pair_10mb at scale 0.1", "tlen": pair.tlen, "qlen": pair.qlen}
    with pkg.Context(local) as ctx:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ctx.run(T, Q, pkg.default_params())
        torch.cuda.synchronize()
        e0.record()
        hs, st = ctx.run(T, Q, pkg.default_params())
        e1.record()
        torch.cuda.synchronize()
        filt_ms = e0.elapsed_time(e1)
        H = torch.from_numpy(np.ascontiguousarray(hs).view(np.int32).reshape(-1, 5).copy()).to(dev)
        A, gst = ctx.gapped_extend(T, Q, H, pkg.ydrop_params())
        res["xdrop_then_gapped"] = {"filter_ms": round(filt_ms, 3), "hsps": int(H.shape[0]),
                                    "gapped_device_ms": round(gst["device_ms"], 3),
                                    "gapped_total_ms": round(gst["total_ms"], 3),
                                    "alignments": gst["committed"], **gapped_recovery(pair, A)}
        ix = ctx.index_build(T, pkg.default_params())
        try:
            cap = 1 << 24
            while True:
                buf = torch.zeros((cap, 3), dtype=torch.int32, device=dev)
                try:
                    _, n = ctx.seed_hits(ix, Q, out=buf)
                    break
                except pkg.SfeError:
                    cap *= 2
        finally:
            ix.close()
        anc = torch.zeros((n, 5), dtype=torch.int32, device=dev)
        anc[:, :3] = buf[:n]
        anc[:, 3] = 19
        prm = pkg.ydrop_params(ydrop=910)
        ctx.gapped_extend(T, Q, anc, prm)
        A2, yst = ctx.gapped_extend(T, Q, anc, prm)
        res["ydrop_as_filter"] = {"anchors": int(n), "ydrop": 910,
                                  "device_ms": round(yst["device_ms"], 3),
                                  "total_ms": round(yst["total_ms"], 3),
                                  "extended": yst["extended"], "skipped": yst["skipped"],
                                  "shadow": yst["shadow"], "cells": yst["cells"],
                                  "alignments": yst["committed"], **gapped_recovery(pair, A2)}
    return res


def block_diagonal_hits(hits, pair):
    """The hits (device int32 tensor (n, 3): strand, tpos, qpos) that lie on a
    planted block's diagonal band (the block's diagonal on its strand within
    50 + 3% of its length, as in block_recovery)."""
    import torch
    out = []
    for strand in (0, 1):
        iv = []
        for b in pair.blocks:
            if int(b.rc) != strand:
                continue
            qb = (pair.qlen - b.qstart - b.qlen) if b.rc else b.qstart
            d0, tol = b.tstart - qb, int(50 + 0.03 * b.tlen)
            iv.append((d0 - tol, d0 + tol))
        if not iv:
            continue
        iv.sort()
        merged = [list(iv[0])]
        for lo, hi in iv[1:]:
            if lo <= merged[-1][1]:
                merged[-1][1] = max(merged[-1][1], hi)
            else:
                merged.append([lo, hi])
        dev = hits.device
        lo = torch.tensor([m[0] for m in merged], dtype=torch.int64, device=dev)
        hi = torch.tensor([m[1] for m in merged], dtype=torch.int64, device=dev)
        h = hits[hits[:, 0] == strand]
        d = h[:, 1].long() - h[:, 2].long()
        k = torch.searchsorted(lo, d, right=True) - 1
        ok = (k >= 0) & (d <= hi[k.clamp(min=0)])
        out.append(h[ok])
    return torch.cat(out).contiguous() if out else hits[:0]


def run_spec_study(a, ctx, T, Q, pair) -> dict:
    """Algorithm 3's speculative window on the per-diagonal skip: walk time and
    shadow fraction (speculative work on hits a commit then covered, over the
    useful cells) against the window, on the whole pair and on the hits of the
    planted blocks' diagonals alone; the default lane walk for reference."""
    import torch
    import paper_2606_06811_gb300 as pkg
    res = {"windows": SPEC_WINDOWS, "whole_pair": [], "block_diagonals": []}

    def timed(fn, reps):
        for _ in range(a.sub_warmup):
            fn()
        rows = [fn() for _ in range(reps)]
        return rows[-1][1], sum(r[0] for r in rows) / reps

    for k in SPEC_WINDOWS:
        prm = pkg.default_params(flags=pkg.TIME_STAGES, walk_mode=pkg.WALK_SPECULATIVE,
                                 spec_window=k)

        def one():
            hs, st = ctx.run(T, Q, prm, cap=1 << 22)
            return st["stage_ms"]["walk_warps"], st
        st, ms = timed(one, a.sub_steps)
        res["whole_pair"].append({"window": k, "walk_ms": round(ms, 3), "cells": st["cells"],
                                  "shadow_cells": st["shadow_cells"],
                                  "shadow_fraction": st["shadow_cells"] / max(1, st["cells"])})
    ix = ctx.index_build(T, pkg.default_params())
    try:
        cap = 1 << 28
        while True:  # device buffer for every hit of both strands
            buf = torch.zeros((cap, 3), dtype=torch.int32, device=T.device)
            try:
                _, n = ctx.seed_hits(ix, Q, out=buf)
                break
            except pkg.SfeError:
                del buf
                cap *= 2
        sub = block_diagonal_hits(buf[:n], pair)
        del buf
        res["block_diagonal_hits"] = int(sub.shape[0])
        for k in [0] + SPEC_WINDOWS:
            walk = (pkg.default_params(flags=pkg.TIME_STAGES) if k == 0 else
                    pkg.default_params(flags=pkg.TIME_STAGES, walk_mode=pkg.WALK_SPECULATIVE,
                                       spec_window=k))
            ctx.set_walk(walk)

            def one():
                hs, st = ctx.ungapped_xdrop(ix, Q, sub, oracle_scores(), 910, 3000)
                return st["stage_ms"]["walk_lanes"] + st["stage_ms"]["walk_warps"], st
            st, ms = timed(one, a.sub_steps)
            row = {"window": k if k else "lane walk (default)", "walk_ms": round(ms, 3),
                   "cells": st["cells"], "shadow_cells": st["shadow_cells"],
                   "shadow_fraction": st["shadow_cells"] / max(1, st["cells"])}
            res["block_diagonals"].append(row)
        ctx.set_walk(None)
    finally:
        ix.close()
    return res


def oracle_scores():
    """HOXD70 as the library's default parameters hold it (4 x 4, target-major)."""
    import paper_2606_06811_gb300 as pkg
    return np.array(list(pkg.default_params().scores), dtype=np.int32).reshape(4, 4)


def run_large(a, local) -> dict:
    """The 100 Mb x 100 Mb pair (query-tiled, skip state carried across
    tiles): the plain path and the learned-binned persistent path, GCUPS of
    each and whether their HSP lists are byte-identical."""
    import torch
    import paper_2606_06811_gb300 as pkg
    dev = torch.device("cuda", local)
    t0 = time.perf_counter()
    pair, Ta, Qa = make_workload(a.seed, 1.0, "large_pair_100mb")
    gen_s = time.perf_counter() - t0
    T = torch.from_numpy(Ta.copy()).to(dev)
    Q = torch.from_numpy(Qa.copy()).to(dev)
    del Ta, Qa
    stream = torch.cuda.Stream(device=dev)
    ctx = pkg.Context(local, stream=stream)
    cap = 1 << 23
    out = torch.zeros((cap, 5), dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    def step(prm):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hs, st = ctx.run(T, Q, prm, out=out)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), st, int(hs.shape[0])

    def arm(prm):
        for _ in range(a.warmup):
            step(prm)
        rows = [step(prm) for _ in range(a.steps)]
        ms = sum(r[0] for r in rows)
        st = rows[0][1]
        return {"value": sum(r[1]["cells"] for r in rows) / (ms / 1e3) / 1e9, "unit": "GCUPS",
                "ms_per_step": ms / len(rows), "hsps_per_s": rows[0][2] * len(rows) / (ms / 1e3),
                "per_step": {"cells": st["cells"], "hits": st["hits"], "hsps": rows[0][2],
                             "tiles": st["tiles"], "warp_tasks": st["warp_tasks"]},
                "stage_ms": {k: round(v, 2) for k, v in st["stage_ms"].items()}}

    clocks = ClockSampler(local)
    clocks.start()
    plain = arm(pkg.default_params(flags=pkg.TIME_STAGES))
    plain_out = out[: plain["per_step"]["hsps"]].clone()
    res = {"workload": "large_pair_100mb", "seed": a.seed, "tlen": pair.tlen, "qlen": pair.qlen,
           "steps": a.steps, "warmup": a.warmup, "generate_s": round(gen_s, 1),
           "plain": plain}
    if not a.no_learned:
        from paper_2606_06811_gb300 import predictor
        t1 = time.perf_counter()
        tr = make_workload(a.train_seed, 0.2, "large_pair_100mb")[0]
        recs, _ = predictor.collect(ctx, tr.T, tr.Q, a.log_every, cap=1 << 25,
                                    params=pkg.default_params(input_codes=1))
        data = predictor.training_data(ctx, [(tr.T, tr.Q, recs)])
        pred = predictor.train(ctx, data, epochs=2, batch=8192, lr=2e-3, seed=3)
        data.close()
        train_s = time.perf_counter() - t1
        lp = pkg.default_params(flags=pkg.TIME_STAGES, walk_mode=pkg.WALK_PERSISTENT,
                                walk_schedule=pkg.SCHED_PREDICTED, walk_chunk=256,
                                model=pred.model.data_ptr())
        learned = arm(lp)
        n = learned["per_step"]["hsps"]
        learned["bit_exact_vs_plain"] = bool(n == plain_out.shape[0] and
                                             torch.equal(out[:n], plain_out))
        learned["walk"] = "persistent, chunks of 256 hits ordered by predicted work"
        learned["predictor"] = {"train_workload": f"large_pair_100mb seed {a.train_seed} "
                                                  f"at scale 0.2", "train_s": round(train_s, 1)}
        res["learned_binned"] = learned
    res["clocks"] = clocks.stop()
    ctx.close()
    return res


def main():
    a = args_parse()
    rank, world, local = dist_env()
    if a.impl == "reference":
        return run_reference(a, rank, world)
    if a.workload == "batch_pairs":
        return run_batch_bench(a, rank, world, local)
    return run_sfe(a, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
