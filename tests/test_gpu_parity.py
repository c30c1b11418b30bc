"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bit-exact: the sorted HSP lists (strand, tpos, qpos, len, int32 score) and the
work counters (hits, extended hits, cells) must be identical.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from tests import bruteforce as bf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_06811_gb300 as P
    return P


@pytest.fixture(scope="module")
def ctx(pkg):
    c = pkg.Context(0)
    yield c
    c.close()


def as_i32(h) -> np.ndarray:
    return np.ascontiguousarray(h).view(np.int32).reshape(-1, 5)


def assert_same(got, st, ref):
    a, b = as_i32(got), as_i32(ref.hsps)
    assert a.shape == b.shape, (a.shape, b.shape)
    if a.size:
        bad = np.flatnonzero((a != b).any(1))
        assert bad.size == 0, f"first mismatch at {bad[0]}: gpu {a[bad[0]]} oracle {b[bad[0]]}"
    assert (st["hits"], st["extended"], st["cells"]) == (ref.hits, ref.extended, ref.cells), \
        (st, ref.stats)


def run_both(pkg, ctx, T, Q, **kw):
    okw = {k: v for k, v in kw.items() if k in ("pattern", "transition", "strands", "scores",
                                                 "X", "thresh", "flags", "step")}
    ref = oracle.run(T, Q, **okw)
    pmap = {"pattern": "seed_pattern", "X": "xdrop", "thresh": "hsp_thresh"}
    pkw = {pmap.get(k, k): v for k, v in kw.items()}
    pkw.setdefault("input_codes", 1)
    got, st = ctx.run(T, Q, pkg.default_params(**pkw))
    return got, st, ref


def test_tiny_pair_full(pkg, ctx):
    p = synth.tiny_pair(1)
    got, st, ref = run_both(pkg, ctx, p.T, p.Q)
    assert_same(got, st, ref)
    assert len(got) >= 50


@pytest.mark.parametrize("lane_cap", [1, 16, 40, 1 << 30])
def test_lane_cap_does_not_change_output(pkg, ctx, lane_cap):
    p = synth.tiny_pair(2, length=60_000, n_blocks=15)
    got, st, ref = run_both(pkg, ctx, p.T, p.Q, lane_cap=lane_cap)
    assert_same(got, st, ref)
    # shadow work: what lanes scored on the extensions they handed to warps,
    # at most the seed span plus both sides up to the cap and one window more
    if lane_cap < (1 << 30):
        assert st["warp_tasks"] > 0 and st["shadow_cells"] > 0
        assert st["shadow_cells"] <= st["warp_tasks"] * (19 + 2 * (lane_cap + 16))
    else:
        assert st["shadow_cells"] == 0


@pytest.mark.parametrize("tile_hits", [1, 777, 5000])
def test_query_tiles_carry_the_skip_state(pkg, ctx, tile_hits):
    p = synth.tiny_pair(3, length=50_000, n_blocks=12)
    got, st, ref = run_both(pkg, ctx, p.T, p.Q, tile_hits=tile_hits)
    assert_same(got, st, ref)
    assert st["tiles"] > 1


def _pair(seed, n, m, gc=0.5, blocks=4):
    st = synth.Stream(seed, "gpu")
    T = synth.iid_bases(st.child("T"), n, gc)
    Q = synth.iid_bases(st.child("Q"), m, gc)
    if blocks and n > 2000 and m > 2000:
        synth.plant_blocks(st.child("b"), T, Q, blocks, 300, 1500, 0.80, 0.97, 0.5, 0.01, gc)
    return T, Q


def _asym(seed):
    st = synth.Stream(seed, "scores")
    M = st.integers(-60, 40, 16).reshape(4, 4).astype(np.int32)
    M[np.arange(4), np.arange(4)] = st.integers(50, 120, 4)
    return M


@pytest.mark.parametrize("case", [
    dict(), dict(transition=False), dict(pattern="1101011"), dict(pattern="11011", transition=False),
    dict(pattern="111010010100110111"), dict(X=0), dict(X=50), dict(X=5000),
    dict(thresh=0), dict(thresh=-100000), dict(flags=1, thresh=1000), dict(strands=1),
    dict(strands=2), dict(scores="asym", X=300, thresh=500),
    # the packed window's limits: X just below and at 2^23, scores near 2^19
    dict(X=(1 << 23) - 1), dict(X=1 << 23), dict(scores="x4096", X=910 * 4096, thresh=3000 * 4096),
    dict(scores="x4096", X=1 << 23, thresh=3000 * 4096),
], ids=lambda c: ",".join(f"{k}={v}" for k, v in c.items()) or "default")
def test_parameters(pkg, ctx, case):
    case = dict(case)
    if case.get("scores") == "asym":
        case["scores"] = _asym(5)
    elif case.get("scores") == "x4096":
        case["scores"] = oracle.HOXD70.astype(np.int64) * 4096
    T, Q = _pair(11, 9_001, 7_333)
    got, st, ref = run_both(pkg, ctx, T, Q, **case)
    assert_same(got, st, ref)


@pytest.mark.parametrize("n,m", [(0, 100), (100, 0), (0, 0), (18, 18), (19, 19), (19, 40),
                                 (33, 17), (1, 1000), (4097, 65), (16, 16), (31, 47)])
def test_ragged_and_degenerate_lengths(pkg, ctx, n, m):
    T, Q = _pair(n * 7 + m, n, m, blocks=0)
    got, st, ref = run_both(pkg, ctx, T, Q, thresh=-100000)
    assert_same(got, st, ref)


def test_identical_sequences_long_extensions(pkg, ctx):
    st = synth.Stream(31, "ident")
    T = synth.iid_bases(st, 20_000, 0.5)
    got, stt, ref = run_both(pkg, ctx, T, T.copy())
    assert_same(got, stt, ref)
    assert stt["warp_tasks"] > 0


def test_poly_a_hit_explosion(pkg, ctx):
    T = np.zeros(3000, np.uint8)
    Q = np.zeros(2500, np.uint8)
    Q[1000] = 2
    got, st, ref = run_both(pkg, ctx, T, Q, thresh=0)
    assert_same(got, st, ref)


def test_period19_repeats(pkg, ctx):
    st = synth.Stream(5, "p19")
    unit = synth.iid_bases(st, 19, 0.5)
    T = np.tile(unit, 300)
    Q = np.tile(unit, 200)[7:]
    got, stt, ref = run_both(pkg, ctx, T, Q, thresh=0)
    assert_same(got, stt, ref)


def test_plain_generator_scaled(pkg, ctx):
    p = synth.plain_pair_10mb(2, scale=0.02)  # 200 kb with repeats and rc blocks
    got, st, ref = run_both(pkg, ctx, p.T, p.Q)
    assert_same(got, st, ref)


def test_ascii_input_and_host_device_buffers(pkg, ctx):
    import torch
    p = synth.tiny_pair(4, length=40_000, n_blocks=10)
    Ta = np.frombuffer(synth.decode(p.T), np.uint8).copy()
    Qa = np.frombuffer(synth.decode(p.Q), np.uint8).copy()
    Qa[::7] += 32  # lower case is accepted
    ref = oracle.run(p.T, p.Q)
    params = pkg.default_params()
    for T, Q in ((Ta, Qa), (torch.from_numpy(Ta).cuda(), torch.from_numpy(Qa).cuda())):
        got, st = ctx.run(T, Q, params)
        assert_same(got, st, ref)
    # device output buffer
    out = torch.zeros((4096, 5), dtype=torch.int32, device="cuda")
    o, st = ctx.run(torch.from_numpy(Ta).cuda(), torch.from_numpy(Qa).cuda(), params, out=out)
    assert np.array_equal(o.cpu().numpy(), as_i32(ref.hsps))


def test_bad_symbol_is_rejected(pkg, ctx):
    T = np.frombuffer(b"ACGTNACGT" * 10, np.uint8).copy()
    with pytest.raises(pkg.SfeError) as e:
        ctx.run(T, T, pkg.default_params())
    assert e.value.code == -1


def test_small_hsp_capacity_reports_needed_count(pkg, ctx):
    p = synth.tiny_pair(1)
    ref = oracle.run(p.T, p.Q)
    got, st = ctx.run(p.T, p.Q, pkg.default_params(input_codes=1), cap=3)  # retries on overflow
    assert np.array_equal(as_i32(got), as_i32(ref.hsps))


def test_seed_hits_api(pkg, ctx):
    T, Q = _pair(21, 12_000, 9_000)
    ix = ctx.index_build(T, pkg.default_params(input_codes=1))
    hits = ctx.seed_hits(ix, Q, strands=3)
    for s, Qs in ((0, Q), (1, bf.revcomp(Q))):
        t, q = oracle.seed_hits(T, Qs)
        h = hits[hits["strand"] == s]
        assert np.array_equal(h["tpos"], t) and np.array_equal(h["qpos"], q)
    ix.close()


def test_ungapped_xdrop_api_on_shuffled_oracle_hits(pkg, ctx):
    T, Q = _pair(22, 15_000, 11_000)
    ix = ctx.index_build(T, pkg.default_params(input_codes=1))
    recs = []
    for s, Qs in ((0, Q), (1, bf.revcomp(Q))):
        t, q = oracle.seed_hits(T, Qs)
        recs.append(np.stack([np.full(t.size, s), t, q], 1))
    H = np.concatenate(recs).astype(np.int32)
    H = H[synth.Stream(3, "perm").integers(0, 1 << 30, H.shape[0]).argsort(kind="stable")]
    got, st = ctx.ungapped_xdrop(ix, Q, np.ascontiguousarray(H), oracle.HOXD70, 910, 3000)
    ref = oracle.run(T, Q)
    assert_same(got, st, ref)
    ix.close()


@pytest.mark.parametrize("mode,chunk,sched,cap", [
    (0, 0, 0, 96), (1, 1, 0, 16), (1, 7, 1, 16), (1, 32, 1, 96), (1, 500, 0, 16),
    (1, 32, 0, 1 << 30), (1, 64, 1, 1), (1, 16, 3, 16), (0, 0, 0, 0),
])
def test_walk_modes_chunks_and_schedules(pkg, ctx, mode, chunk, sched, cap):
    """Persistent or two-launch walks, any chunk size and chunk order: same output."""
    p = synth.tiny_pair(2, length=60_000, n_blocks=15)
    got, st, ref = run_both(pkg, ctx, p.T, p.Q, walk_mode=mode, walk_chunk=chunk,
                            walk_schedule=sched, lane_cap=cap)
    assert_same(got, st, ref)


@pytest.mark.parametrize("n,m", [(19, 19), (20, 27), (33, 41), (9_001, 7_333), (60_007, 40_003)])
@pytest.mark.parametrize("windows", ["planes", "two_bit"])
def test_window_sources_agree(pkg, ctx, n, m, windows):
    """The lane windows of one pair's walk come from the 4-bit cell planes
    (the default where they fit) or from the 2-bit words; each gives the
    oracle's output, on lengths with ragged ends of the planes' 8-base words
    and of the 2-bit words' 16-base words, with hits next to both ends."""
    T, Q = _pair(40 + n % 7, n, m, blocks=6)
    ref = oracle.run(T, Q)
    flags = {"planes": 0, "two_bit": pkg.NO_CELL_PLANES}[windows]
    for cap in (16, 0):
        got, st = ctx.run(T, Q, pkg.default_params(input_codes=1, flags=flags, lane_cap=cap))
        assert_same(got, st, ref)
    # the same with the skip advanced only by passing HSPs
    ref = oracle.run(T, Q, flags=1)
    got, st = ctx.run(T, Q, pkg.default_params(input_codes=1, flags=flags | 1))
    assert_same(got, st, ref)


@pytest.mark.parametrize("chunk", [1, 2, 7, 64])
def test_persistent_walk_chunk_starts_and_skips(pkg, ctx, chunk):
    """Persistent walk with tiny chunks (a chunk boundary at almost every hit,
    diagonals that start before their chunk) and on nearly identical
    sequences (long runs of skipped hits)."""
    st = synth.Stream(33, "ident3")
    T = synth.iid_bases(st, 20_000, 0.5)
    Q = T.copy()
    Q[5000:5400] = synth.iid_bases(st.child("q"), 400, 0.5)
    got, stt, ref = run_both(pkg, ctx, T, Q, walk_mode=pkg.WALK_PERSISTENT, walk_chunk=chunk,
                             lane_cap=64)
    assert_same(got, stt, ref)
    p = synth.tiny_pair(3, length=50_000, n_blocks=12)
    got, stt, ref = run_both(pkg, ctx, p.T, p.Q, walk_mode=pkg.WALK_PERSISTENT, walk_chunk=chunk)
    assert_same(got, stt, ref)


def test_persistent_walk_on_identical_sequences(pkg, ctx):
    st = synth.Stream(32, "ident2")
    T = synth.iid_bases(st, 30_000, 0.5)
    got, stt, ref = run_both(pkg, ctx, T, T.copy(), walk_mode=pkg.WALK_PERSISTENT, walk_chunk=8,
                             walk_schedule=1, lane_cap=16)
    assert_same(got, stt, ref)
    assert stt["warp_tasks"] > 0


# ------------------------------------------------------------------ heavier seeds and step
P22 = "1110111000011101011011"  # the 14-of-22 mask (Section 7 names the weight, not the mask)


@pytest.mark.parametrize("pattern,step,transition", [
    (P22, 1, True), (P22, 2, True), (P22, 5, False), (oracle.DEFAULT_PATTERN, 3, True),
    (oracle.DEFAULT_PATTERN, 2, False), ("1101011", 4, True),
])
def test_heavier_seed_and_step(pkg, ctx, pattern, step, transition):
    """Section 7's heavier seed and the index stride (only target positions
    divisible by the step are seeds), against the oracle, on the plain
    generator at 200 kb and on ragged lengths."""
    p = synth.plain_pair_10mb(9, scale=0.02 if pattern.count("1") > 8 else 0.003)
    got, st, ref = run_both(pkg, ctx, p.T, p.Q, pattern=pattern, step=step, transition=transition)
    assert_same(got, st, ref)
    T, Q = _pair(71, 4099, 3001, blocks=4)
    got, st, ref = run_both(pkg, ctx, T, Q, pattern=pattern, step=step, transition=transition,
                            lane_cap=16)
    assert_same(got, st, ref)


def test_seed_hits_api_with_step(pkg, ctx):
    p = synth.tiny_pair(6, length=80_000, n_blocks=12)
    ix = ctx.index_build(p.T, pkg.default_params(input_codes=1, seed_pattern=P22, step=3))
    try:
        h = ctx.seed_hits(ix, p.Q)
    finally:
        ix.close()
    for s, Qs in ((0, p.Q), (1, oracle.revcomp(p.Q))):
        t, q = oracle.seed_hits(p.T, Qs, P22, True, 3)
        mine = h[h["strand"] == s]
        assert np.array_equal(mine["tpos"], t) and np.array_equal(mine["qpos"], q)


@pytest.mark.parametrize("pattern,step", [(oracle.DEFAULT_PATTERN, 1), (oracle.DEFAULT_PATTERN, 3),
                                          (P22, 1), (P22, 2), ("1101011", 1)])
@pytest.mark.parametrize("dense", [False, True])
def test_sparse_and_dense_index_agree(pkg, ctx, pattern, step, dense):
    """The position table over the keys' top bits (the default where the
    target fills few of the 4^weight keys) and the dense table over every key
    (forced by a test hook) give the oracle's hits and HSPs, through sfe_run
    and through sfe_index_build + sfe_seed_hits."""
    hooks = pkg.sfe.TEST_DENSE_INDEX if dense else 0
    # a weight-5 seed hits about every 4^5 / 13 positions per diagonal: a smaller pair
    p = synth.tiny_pair(12, length=120_000 if pattern.count("1") > 8 else 15_000, n_blocks=15)
    got, st, ref = run_both(pkg, ctx, p.T, p.Q, pattern=pattern, step=step, test_hooks=hooks)
    assert_same(got, st, ref)
    ix = ctx.index_build(p.T, pkg.default_params(input_codes=1, seed_pattern=pattern, step=step,
                                                 test_hooks=hooks))
    try:
        h = ctx.seed_hits(ix, p.Q)
    finally:
        ix.close()
    for s, Qs in ((0, p.Q), (1, oracle.revcomp(p.Q))):
        t, q = oracle.seed_hits(p.T, Qs, pattern, True, step)
        mine = h[h["strand"] == s]
        assert np.array_equal(mine["tpos"], t) and np.array_equal(mine["qpos"], q)


# ------------------------------------------------------------------ speculative window
@pytest.mark.parametrize("window", [1, 2, 4, 8, 16, 32])
def test_speculative_window_keeps_the_output(pkg, ctx, window):
    """Algorithm 3's speculative batch on the per-diagonal skip: any window of
    hits extended at once and committed in t order gives the serial output;
    window 1 does no shadow work, larger windows do on dense diagonals."""
    kw = dict(walk_mode=pkg.WALK_SPECULATIVE, spec_window=window)
    p = synth.tiny_pair(2, length=60_000, n_blocks=15)
    got, st, ref = run_both(pkg, ctx, p.T, p.Q, **kw)
    assert_same(got, st, ref)
    st_ = synth.Stream(34, "spec")
    T = synth.iid_bases(st_, 20_000, 0.5)
    got, st, ref = run_both(pkg, ctx, T, T.copy(), **kw)  # one long, dense diagonal per strand
    assert_same(got, st, ref)
    assert (st["shadow_cells"] == 0) if window == 1 else (st["shadow_cells"] > 0)
    T, Q = _pair(72, 9001, 7333, blocks=6)
    got, st, ref = run_both(pkg, ctx, T, Q, thresh=1000, flags=1, **kw)  # skip-passing-only
    assert_same(got, st, ref)
    got, st, ref = run_both(pkg, ctx, T, Q, tile_hits=500, walk_chunk=3, **kw)  # E across tiles
    assert_same(got, st, ref)


def test_speculative_window_through_the_hit_list_call(pkg, ctx):
    p = synth.tiny_pair(7, length=50_000, n_blocks=12)
    ref = oracle.run(p.T, p.Q)
    ix = ctx.index_build(p.T, pkg.default_params(input_codes=1))
    try:
        hits = ctx.seed_hits(ix, p.Q)
        ctx.set_walk(pkg.default_params(walk_mode=pkg.WALK_SPECULATIVE, spec_window=4))
        got, st = ctx.ungapped_xdrop(ix, p.Q, hits, oracle.HOXD70, 910, 3000)
        ctx.set_walk(None)
    finally:
        ix.close()
    assert_same(got, st, ref)


def test_a_pair_longer_than_31_bit_diagonals_is_rejected(pkg, ctx):
    """A target and a query whose lengths add to 2^31 or more would need a
    32-bit diagonal index: the call refuses them before touching the data."""
    import ctypes as C
    lib = pkg.sfe.lib()
    n = C.c_int64(0)
    prm = pkg.default_params()
    tlen, qlen = (1 << 31) - 2048, 4096
    code = lib.sfe_run(ctx.h, None, tlen, None, qlen, C.byref(prm), None, 0, C.byref(n), None)
    assert code == -1 and b"2^31" in lib.sfe_last_error()


def test_speculative_window_rejects_bad_windows(pkg, ctx):
    p = synth.tiny_pair(2, length=5_000, n_blocks=2)
    for bad in (3, 64, -1):
        with pytest.raises(pkg.SfeError):
            ctx.run(p.T, p.Q, pkg.default_params(input_codes=1, walk_mode=pkg.WALK_SPECULATIVE,
                                                 spec_window=bad))
