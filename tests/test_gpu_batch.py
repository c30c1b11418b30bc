"""Batch of uneven pairs (sfe_run_batch) against the oracle run pair by pair.

Bit-exact per pair: the batch HSP list, split by pair, equals the oracle's
list for that pair; hits, extended hits and cells add up to the oracle's.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from synth.workloads import concat_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_06811_gb300 as P
    return P


def oracle_batch(pairs, **kw):
    rows, hits, ext, cells = [], 0, 0, 0
    for i, p in enumerate(pairs):
        r = oracle.run(p.T, p.Q, **kw)
        h = r.hsps.view(np.int32).reshape(-1, 5)
        rows.append(np.concatenate([np.full((h.shape[0], 1), i, np.int32), h], 1))
        hits, ext, cells = hits + r.hits, ext + r.extended, cells + r.cells
    H = np.concatenate(rows) if rows else np.zeros((0, 6), np.int32)
    return H, hits, ext, cells


def gpu_batch(P, pairs, **kw):
    T, toff, Q, qoff = concat_batch(pairs)
    with P.Context(0) as ctx:
        h, st = ctx.run_batch(T, toff, Q, qoff, P.default_params(input_codes=1, **kw))
    return np.ascontiguousarray(h).view(np.int32).reshape(-1, 6), st


def check(P, pairs, **kw):
    names = {"hsp_thresh": "thresh", "seed_pattern": "pattern"}
    okw = {names.get(k, k): v for k, v in kw.items()
           if k not in ("lane_cap", "lanes_per_sm", "tile_hits", "walk_mode", "walk_chunk",
                        "walk_schedule", "spec_window")}
    H, hits, ext, cells = oracle_batch(pairs, **okw)
    G, st = gpu_batch(P, pairs, **kw)
    assert G.shape == H.shape and np.array_equal(G, H)
    assert (st["hits"], st["extended"], st["cells"]) == (hits, ext, cells)
    return G


def test_batch_uneven_pairs(pkg):
    pairs = synth.batch_pairs(seed=3, n_pairs=96, len_lo=1000, len_hi=40_000)
    G = check(pkg, pairs)
    assert len(np.unique(G[:, 0])) > 10


def test_batch_with_degenerate_pairs(pkg):
    st = synth.Stream(8, "deg")
    pairs = []
    for i, (n, m) in enumerate([(0, 50), (18, 18), (19, 19), (5000, 10), (3000, 3000), (1, 1),
                                (700, 900)]):
        T = synth.iid_bases(st.child("T", i), n, 0.5)
        Q = T[:m].copy() if n >= m else synth.iid_bases(st.child("Q", i), m, 0.5)
        pairs.append(synth.Pair(T, Q))
    check(pkg, pairs, hsp_thresh=0)


def test_batch_single_strand_and_lane_cap(pkg):
    pairs = synth.batch_pairs(seed=4, n_pairs=40, len_lo=2000, len_hi=30_000)
    check(pkg, pairs, strands=2, lane_cap=16)
    check(pkg, pairs, strands=1)


@pytest.mark.parametrize("mode,sched,chunk", [(0, 0, 0), (1, 1, 16), (1, 0, 3), (1, 3, 8)])
def test_batch_walk_modes(pkg, mode, sched, chunk):
    pairs = synth.batch_pairs(seed=6, n_pairs=64, len_lo=1000, len_hi=30_000)
    check(pkg, pairs, walk_mode=mode, walk_schedule=sched, walk_chunk=chunk, lane_cap=32)


@pytest.mark.parametrize("window", [1, 4, 32])
def test_batch_speculative_window(pkg, window):
    """The speculative window walk (32 / window lanes per hit) over a batch:
    every pair's HSPs as the oracle's, chunks that split pairs included."""
    pairs = synth.batch_pairs(seed=8, n_pairs=48, len_lo=1000, len_hi=20_000)
    check(pkg, pairs, walk_mode=pkg.WALK_SPECULATIVE, spec_window=window, walk_chunk=5)


def _variant(pairs):
    """Pairs of the same lengths with other content: reverse-complemented
    targets and reversed queries."""
    out = []
    for p in pairs:
        T = (3 - p.T[::-1]).astype(np.uint8)
        Q = np.ascontiguousarray(p.Q[::-1]).astype(np.uint8)
        out.append(synth.Pair(T, Q, [], p.name + "'", p.gc))
    return out


@pytest.mark.parametrize("kw", [{}, {"walk_mode": 1, "walk_chunk": 8},
                                {"walk_mode": 1, "walk_schedule": 3, "walk_chunk": 16}],
                         ids=["two-launch", "persistent", "persistent-random"])
def test_batch_plan_replays_a_captured_graph(pkg, kw):
    pairs = synth.batch_pairs(seed=12, n_pairs=48, len_lo=1000, len_hi=30_000)
    T, toff, Q, qoff = concat_batch(pairs)
    H, hits, ext, cells = oracle_batch(pairs)
    with pkg.Context(0) as ctx:
        # a hit capacity far too small: the first run grows the plan and captures again
        plan = ctx.batch_plan(toff, qoff, pkg.default_params(input_codes=1, **kw), hit_cap=1000)
        for _ in range(2):
            h, st = plan.run(T, Q)
            G = np.ascontiguousarray(h).view(np.int32).reshape(-1, 6)
            assert np.array_equal(G, H)
            assert (st["hits"], st["extended"], st["cells"]) == (hits, ext, cells)
            assert st["launches"] > 10
        # new sequences of the same lengths, through the same graph
        other = _variant(pairs)
        T2, toff2, Q2, qoff2 = concat_batch(other)
        assert np.array_equal(toff2, toff) and np.array_equal(qoff2, qoff)
        H2, hits2, _, cells2 = oracle_batch(other)
        h, st = plan.run(T2, Q2)
        G2 = np.ascontiguousarray(h).view(np.int32).reshape(-1, 6)
        assert np.array_equal(G2, H2)
        assert (st["hits"], st["cells"]) == (hits2, cells2)
        plan.close()


def test_batch_plan_rejects_stage_timing_and_bad_offsets(pkg):
    with pkg.Context(0) as ctx:
        with pytest.raises(pkg.SfeError):
            ctx.batch_plan([0, 100], [0, 100], pkg.default_params(flags=pkg.TIME_STAGES))
        with pytest.raises(pkg.SfeError):
            ctx.batch_plan([0, 100, 50], [0, 10, 20], pkg.default_params())


def test_autotuner_keeps_the_output_and_caches_its_choice(pkg, tmp_path):
    import torch
    from paper_2606_06811_gb300 import autotune
    pairs = synth.batch_pairs(seed=13, n_pairs=32, len_lo=1000, len_hi=20_000)
    T, toff, Q, qoff = concat_batch(pairs)
    H, *_ = oracle_batch(pairs)
    space = {"walk_mode": [0, 1], "lane_cap": [32, 256], "walk_chunk": [8, 64],
             "walk_schedule": [0, 1]}
    cache = str(tmp_path / "tune.json")
    with pkg.Context(0) as ctx:
        def run(c):
            h, st = ctx.run_batch(T, toff, Q, qoff, pkg.default_params(input_codes=1, **c))
            return np.ascontiguousarray(h).tobytes(), st
        sig = autotune.batch_signature(toff, qoff, pkg.default_params())
        best, table = autotune.tune(run, sig, space=space, reps=1, cache=cache)
        assert len(table) == len(autotune.candidates(space)) == 2 + 8
        assert best in [c for c, _ in table]
        G = np.ascontiguousarray(run(best)[0])
        assert np.array_equal(np.frombuffer(G, np.int32).reshape(-1, 6), H)

        def never(c):
            raise AssertionError("a cached workload is not timed again")
        best2, _ = autotune.tune(never, sig, space=space, reps=1, cache=cache)
        assert best2 == best
    torch.cuda.synchronize()


@pytest.mark.parametrize("pattern,step", [("1110111000011101011011", 1),
                                          ("1110111000011101011011", 3),
                                          ("1110100110010101111", 2)])
def test_batch_heavier_seed_and_step(pkg, pattern, step):
    pairs = synth.batch_pairs(seed=6, n_pairs=48, len_lo=2000, len_hi=30_000)
    G = check(pkg, pairs, seed_pattern=pattern, step=step)
    assert G.shape[0] > 0
