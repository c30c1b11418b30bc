"""The seeded input generators against what they state: the published
SplitMix64 outputs, counter-based streams, base composition, substitution
identity and Ts:Tv, indel balance, planted blocks copied where recorded and
repeat coverage. Statistical checks use bounds of five standard deviations
(or looser, stated) derived from the generator's stated parameters."""
from __future__ import annotations

import math

import numpy as np

import synth
from synth import genome, rng


def test_splitmix64_published_outputs():
    # the first outputs of SplitMix64 whose state starts at 0 (Steele, Lea and
    # Flood 2014; the sequence used to seed the xoshiro generators)
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    assert [int(x) for x in rng.splitmix64(0, 0, 4)] == want
    # output i depends only on (key, i)
    assert [int(x) for x in rng.splitmix64(0, 2, 2)] == want[2:]


def test_streams_are_counter_based_and_named():
    a = rng.Stream(7, "x", 3)
    b = rng.Stream(7, "x", 3)
    whole = a.u64(10)
    parts = np.concatenate([b.u64(3), b.u64(7)])
    assert np.array_equal(whole, parts)
    assert np.array_equal(rng.Stream(7, "x").child(3).u64(5), rng.Stream(7, "x", 3).u64(5))
    assert not np.array_equal(rng.Stream(7, "x").u64(5), rng.Stream(7, "y").u64(5))
    assert not np.array_equal(rng.Stream(7, "x").u64(5), rng.Stream(8, "x").u64(5))


def test_uniform_integers_and_log_uniform():
    st = rng.Stream(1, "u")
    n = 200_000
    u = st.uniform(n)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / n)
    k = st.integers(-3, 4, n)
    assert k.min() == -3 and k.max() == 3
    counts = np.bincount(k + 3, minlength=7)
    p = 1 / 7
    assert np.all(np.abs(counts / n - p) < 5 * math.sqrt(p * (1 - p) / n))
    lu = st.log_uniform_int(10, 10_000, n)
    assert lu.min() >= 10 and lu.max() <= 10_000
    # log-uniform: half the mass below the geometric mean of the range
    below = np.mean(lu < math.sqrt(10 * 10_001))
    assert abs(below - 0.5) < 0.01


def test_iid_bases_composition():
    n, gc = 400_000, 0.41
    x = genome.iid_bases(rng.Stream(2, "b"), n, gc)
    frac = np.bincount(x, minlength=4) / n
    want = np.array([(1 - gc) / 2, gc / 2, gc / 2, (1 - gc) / 2])
    sd = np.sqrt(want * (1 - want) / n)
    assert np.all(np.abs(frac - want) < 5 * sd), (frac, want)


def test_mutate_identity_and_ts_tv():
    n, identity = 300_000, 0.8
    st = rng.Stream(3, "m")
    src = genome.iid_bases(st.child("s"), n, 0.5)
    out = genome.mutate(st.child("m"), src, identity)
    assert out.size == n  # no indels asked for
    x = src ^ out
    sub = x != 0
    p = 1 - identity
    assert abs(sub.mean() - p) < 5 * math.sqrt(p * (1 - p) / n)
    k = int(sub.sum())
    ts = np.mean(x[sub] == 2)
    assert abs(ts - 2 / 3) < 5 * math.sqrt(2 / 9 / k)  # Ts:Tv 2:1
    tv1 = np.sum(x[sub] == 1) / max(1, np.sum(x[sub] != 2))
    assert abs(tv1 - 0.5) < 5 * math.sqrt(0.25 / (k / 3))  # both transversion kinds


def test_mutate_indels_are_balanced():
    n, rate = 200_000, 0.01
    st = rng.Stream(4, "i")
    src = genome.iid_bases(st.child("s"), n, 0.5)
    out = genome.mutate(st.child("m"), src, 1.0, indel_rate=rate, indel_max=5)
    # insertions and deletions have equal odds and the same length law, so the
    # length change has mean 0; its sd is sqrt(events * E[len^2]) with
    # E[len^2] < 25
    sd = math.sqrt(n * rate * 25)
    assert out.size != n and abs(out.size - n) < 5 * sd


def test_planted_blocks_are_copies_where_recorded():
    st = rng.Stream(5, "p")
    T = genome.iid_bases(st.child("T"), 100_000, 0.5)
    for rc_prob in (0.0, 1.0):
        Q = genome.iid_bases(st.child("Q", rc_prob), 80_000, 0.5)
        blocks = genome.plant_blocks(st.child("b", rc_prob), T, Q, 12, 500, 3000, 1.0, 1.0,
                                     rc_prob, 0.0, 0.5)
        assert len(blocks) == 12
        for b in blocks:
            assert b.rc == (rc_prob == 1.0) and b.tlen == b.qlen and 500 <= b.tlen <= 3000
            src = T[b.tstart:b.tstart + b.tlen]
            got = Q[b.qstart:b.qstart + b.qlen]
            assert np.array_equal(got, genome.revcomp_codes(src) if b.rc else src)
    # at identity 0.75..0.85 without indels each block keeps its stated identity
    Q = genome.iid_bases(st.child("Q2"), 80_000, 0.5)
    blocks = genome.plant_blocks(st.child("b2"), T, Q, 10, 2000, 3000, 0.75, 0.85, 0.0, 0.0, 0.5)
    for b in blocks:
        same = np.mean(T[b.tstart:b.tstart + b.tlen] == Q[b.qstart:b.qstart + b.qlen])
        sd = math.sqrt(b.identity * (1 - b.identity) / b.tlen)
        assert abs(same - b.identity) < 5 * sd


def test_repeats_cover_the_stated_fraction():
    n, gc, frac = 300_000, 0.41, 0.05
    st = rng.Stream(6, "r")
    s = genome.iid_bases(st.child("s"), n, gc)
    before = s.copy()
    genome.plant_repeats(st.child("rep"), [s], frac, 20, 300, 300, 0.10, 0.10, gc)
    # copies of at least frac * n bases (at most one copy more) land at uniform
    # positions: expected coverage 1 - exp(-written / n); an overwritten base
    # differs from the old one with probability 1 - sum(p_b^2) for two
    # independent bases at this GC
    p_diff = 1 - (2 * ((1 - gc) / 2) ** 2 + 2 * (gc / 2) ** 2)
    lo = p_diff * (1 - math.exp(-frac))
    hi = p_diff * (1 - math.exp(-(frac + 300 / n)))
    changed = np.mean(before != s)
    assert 0.8 * lo < changed < 1.2 * hi, (changed, lo, hi)


def test_plain_workload_recipe_at_small_scale():
    a = synth.plain_pair_10mb(2, scale=0.01)
    b = synth.plain_pair_10mb(2, scale=0.01)
    assert np.array_equal(a.T, b.T) and np.array_equal(a.Q, b.Q)  # reproducible
    assert a.tlen == 100_000 and a.gc == 0.41
    gc = np.mean((a.T == 1) | (a.T == 2))
    assert abs(gc - 0.41) < 0.01
    assert len(a.blocks) == 20
    for blk in a.blocks:
        assert 1000 <= blk.tlen <= 20_000 and 0.70 <= blk.identity <= 0.90
        assert 0 <= blk.qstart and blk.qstart + blk.qlen <= a.qlen


def test_batch_workload_recipe():
    from synth.workloads import concat_batch
    pairs = synth.batch_pairs(3, n_pairs=200)
    assert len(pairs) == 200
    tl = np.array([p.tlen for p in pairs])
    assert tl.min() >= 1000 and tl.max() <= 256_000
    # log-uniform lengths: about half below the geometric mean of the range
    assert abs(np.mean(tl < math.sqrt(1000 * 256_001)) - 0.5) < 5 * math.sqrt(0.25 / 200)
    assert all(0.35 <= p.gc <= 0.60 and len(p.blocks) <= 20 for p in pairs)
    T, toff, Q, qoff = concat_batch(pairs[:5])
    assert toff[-1] == T.size == sum(p.tlen for p in pairs[:5])
    assert np.array_equal(T[toff[2]:toff[3]], pairs[2].T)
    assert np.array_equal(Q[qoff[4]:qoff[5]], pairs[4].Q)


def test_large_workload_recipe_at_small_scale():
    p = synth.large_pair_100mb(5, scale=0.001)
    assert p.tlen == p.qlen == 100_000 and len(p.blocks) == 20
    assert abs(np.mean((p.T == 1) | (p.T == 2)) - 0.41) < 0.015
    for blk in p.blocks:
        assert 1000 <= blk.tlen <= 50_000 and 0.65 <= blk.identity <= 0.90
