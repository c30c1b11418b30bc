"""Pins of the CPU oracle against things other than itself.

* hand-derived worked cases (tests/golden/hand_cases.json);
* brute force: every window of every diagonal for the hit set, whole prefix-sum
  arrays for each X-drop extension, and a literal query-order loop with a
  per-diagonal masking state for the skip (Algorithm 1's shape);
* symmetries: minus strand == plus strand of the reverse complement computed
  independently; swapping T and Q with the transposed score matrix transposes
  every HSP;
* invariants: every HSP score is the sum of its substitution scores;
* workload properties: planted homologous segments are recovered, i.i.d.
  background gives no HSP above the threshold, hit counts match the closed
  form for uniform i.i.d. sequences.
"""
from __future__ import annotations

import json
import os

import numpy as np
import pytest

import oracle
import synth
from tests import bruteforce as bf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")
P19 = oracle.DEFAULT_PATTERN


def _hand_cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


def check_hand_case(c) -> bool:
    r = oracle.run(synth.encode_ascii(c["T"]), synth.encode_ascii(c["Q"]), c["pattern"],
                   bool(c["transition"]), c["strands"], c["scores"], c["X"], c["thresh"],
                   c.get("flags", 0))
    got = [list(map(int, x)) for x in r.hsps.tolist()]
    return (got == c["hsps"] and r.hits == c["hits"] and r.extended == c["extended"]
            and r.cells == c["cells"])


@pytest.mark.parametrize("case", _hand_cases(), ids=lambda c: c["name"])
def test_hand_case(case):
    assert check_hand_case(case)


def _rand_pair(seed, n, m, gc=0.5, homology=True):
    st = synth.Stream(seed, "pin")
    T = synth.iid_bases(st.child("T"), n, gc)
    Q = synth.iid_bases(st.child("Q"), m, gc)
    if homology and n > 400 and m > 400:
        synth.plant_blocks(st.child("b"), T, Q, 3, 150, 400, 0.85, 0.97, 0.5, 0.01, gc)
    return T, Q


def _rand_asym_scores(seed):
    st = synth.Stream(seed, "scores")
    M = st.integers(-60, 40, 16).reshape(4, 4).astype(np.int32)
    M[np.arange(4), np.arange(4)] = st.integers(50, 120, 4)
    return M


def check_hits_bruteforce(seed=11, n=2500, m=1800, pattern=P19, transition=True, gc=0.5, step=1):
    T, Q = _rand_pair(seed, n, m, gc)
    for Qs in (Q, bf.revcomp(Q)):
        t1, q1 = oracle.seed_hits(T, Qs, pattern, transition, step)
        t2, q2 = bf.hits_by_diagonal(T, Qs, pattern, transition, step)
        if not (np.array_equal(t1, t2) and np.array_equal(q1, q2)):
            return False
    return True


@pytest.mark.parametrize("pattern,transition,gc", [
    (P19, True, 0.5), (P19, False, 0.5), (P19, True, 0.3), ("1101011", True, 0.5),
    ("11011", False, 0.6),
])
def test_hits_match_bruteforce(pattern, transition, gc):
    assert check_hits_bruteforce(7, 2000, 1500, pattern, transition, gc)


def _adversarial_pair(kind):
    st = synth.Stream(5, kind)
    if kind == "polyA":
        T = np.zeros(300, np.uint8)
        Q = np.zeros(250, np.uint8)
        Q[100] = 2  # one transition
    elif kind == "period19":
        unit = synth.iid_bases(st, 19, 0.5)
        T = np.tile(unit, 20)
        Q = np.tile(unit, 13)[5:]
    elif kind == "identical":
        T = synth.iid_bases(st, 600, 0.5)
        Q = T.copy()
    elif kind == "short":
        T = synth.iid_bases(st, 18, 0.5)
        Q = synth.iid_bases(st.child("q"), 40, 0.5)
    else:
        T = np.zeros(0, np.uint8)
        Q = synth.iid_bases(st, 40, 0.5)
    return T, Q


def check_hits_adversarial(kind):
    """The oracle's hits on a degenerate pair equal the brute force's (identical
    sequences and repeats put hits on the first and last positions)."""
    T, Q = _adversarial_pair(kind)
    for Qs in (Q, bf.revcomp(Q)):
        t1, q1 = oracle.seed_hits(T, Qs)
        t2, q2 = bf.hits_by_diagonal(T, Qs, P19, True)
        if not (np.array_equal(t1, t2) and np.array_equal(q1, q2)):
            return False
    return True


@pytest.mark.parametrize("kind", ["polyA", "period19", "identical", "short", "empty"])
def test_hits_adversarial(kind):
    assert check_hits_adversarial(kind)


def check_xdrop_exhaustive(seed=3, scores=None, X=910, nhits=300):
    T, Q = _rand_pair(seed, 3000, 2600)
    M = oracle.HOXD70 if scores is None else scores
    t, q = bf.hits_by_diagonal(T, Q, P19, True)
    if t.size == 0:
        return False
    st = synth.Stream(seed, "pick")
    pick = st.integers(0, t.size, min(nhits, t.size))
    for i in pick:
        a = oracle.xdrop(T, Q, int(t[i]), int(q[i]), 19, M, X)
        b = bf.extend(T, Q, int(t[i]), int(q[i]), 19, M, X)
        for k in ("tpos", "qpos", "len", "score", "end", "cells"):
            if a[k] != b[k]:
                return False
    return True


@pytest.mark.parametrize("X", [0, 50, 910, 5000])
def test_xdrop_matches_exhaustive_hoxd70(X):
    assert check_xdrop_exhaustive(3, None, X)


@pytest.mark.parametrize("seed", [1, 2])
def test_xdrop_matches_exhaustive_asymmetric(seed):
    assert check_xdrop_exhaustive(seed, _rand_asym_scores(seed), 300)


def check_serial_loop(seed=4, n=2200, m=2000, flags=0, scores=None, X=910, thresh=1500,
                      pattern=P19, transition=True, step=1):
    T, Q = _rand_pair(seed, n, m)
    M = oracle.HOXD70 if scores is None else scores
    r = oracle.run(T, Q, pattern, transition, 3, M, X, thresh, flags, step=step)
    ref, st = bf.serial_query_order(T, Q, pattern, transition, 3, M, X, thresh,
                                    bool(flags & oracle.SKIP_PASSING_ONLY), step)
    got = [tuple(map(int, x)) for x in r.hsps.tolist()]
    return (got == ref and r.hits == st["hits"] and r.extended == st["extended"]
            and r.cells == st["cells"])


@pytest.mark.parametrize("flags", [0, oracle.SKIP_PASSING_ONLY])
def test_skip_matches_serial_query_order(flags):
    assert check_serial_loop(4, flags=flags)


def test_skip_matches_serial_query_order_asymmetric():
    assert check_serial_loop(9, scores=_rand_asym_scores(9), X=200, thresh=400)


def check_strand_symmetry(seed=6):
    T, Q = _rand_pair(seed, 3000, 2500)
    minus = oracle.run(T, Q, strands=2, thresh=500)
    plus_rc = oracle.run(T, bf.revcomp(Q), strands=1, thresh=500)
    a = minus.hsps.copy()
    b = plus_rc.hsps.copy()
    b["strand"] = 1
    return np.array_equal(a, b) and minus.cells == plus_rc.cells and a.size > 0


def test_strand_symmetry():
    assert check_strand_symmetry()


def check_swap_symmetry(seed=8, scores=None):
    T, Q = _rand_pair(seed, 2600, 2100)
    M = oracle.HOXD70 if scores is None else np.asarray(scores)
    fwd = oracle.run(T, Q, strands=1, scores=M, thresh=300)
    rev = oracle.run(Q, T, strands=1, scores=np.ascontiguousarray(M.T), thresh=300)
    a = sorted((int(h["tpos"]), int(h["qpos"]), int(h["len"]), int(h["score"]))
               for h in fwd.hsps)
    b = sorted((int(h["qpos"]), int(h["tpos"]), int(h["len"]), int(h["score"]))
               for h in rev.hsps)
    return a == b and fwd.cells == rev.cells and len(a) > 0


@pytest.mark.parametrize("asym", [False, True])
def test_swap_symmetry(asym):
    assert check_swap_symmetry(8, _rand_asym_scores(8) if asym else None)


def test_hsp_score_is_sum_of_substitution_scores():
    p = synth.tiny_pair(1)
    r = oracle.run(p.T, p.Q)
    assert r.hsps.size > 0
    Qm = bf.revcomp(p.Q)
    M = oracle.HOXD70.astype(np.int64)
    for h in r.hsps:
        Qs = p.Q if h["strand"] == 0 else Qm
        t0, q0, L = int(h["tpos"]), int(h["qpos"]), int(h["len"])
        assert int(M[p.T[t0:t0 + L], Qs[q0:q0 + L]].sum()) == int(h["score"])
        assert L >= 19
        assert abs(int(h["score"])) < 2 ** 31


def test_run_diagonal_agrees_with_run():
    T, Q = _rand_pair(12, 2500, 2500)
    full = oracle.run(T, Q, strands=1, thresh=0, keep_log=True)
    diags = np.unique(full.ext["t"] - full.ext["q"])
    st = synth.Stream(1, "diag")
    for d in diags[st.integers(0, diags.size, 25)]:
        one = oracle.run_diagonal(T, Q, 0, int(d), thresh=0)
        mine = full.hsps[full.hsps["tpos"] - full.hsps["qpos"] == d]
        assert np.array_equal(one.hsps, mine)


def test_tiny_pair_planted_recovery():
    """Each of the 50 planted 85%-identity segments yields an HSP >= 3000 on its diagonal."""
    p = synth.tiny_pair(1)
    r = oracle.run(p.T, p.Q)
    h = r.hsps[r.hsps["strand"] == 0]
    found = 0
    for b in p.blocks:
        d = b.tstart - b.qstart
        m = ((h["tpos"] >= b.tstart - 50) & (h["tpos"] < b.tstart + b.tlen) &
             (np.abs(h["tpos"] - h["qpos"] - d) <= 30))
        found += bool(m.any())
    assert found >= 48, found


def test_iid_background_has_no_hsps():
    st = synth.Stream(21, "bg")
    T = synth.iid_bases(st.child("T"), 200_000, 0.5)
    Q = synth.iid_bases(st.child("Q"), 200_000, 0.5)
    r = oracle.run(T, Q)
    assert r.hsps.size == 0
    assert r.extended > 0.95 * r.hits  # isolated random hits are almost never skipped


def test_iid_hit_count_matches_closed_form():
    """Uniform i.i.d.: P(hit) = 4^-12 (exact) + 12 * 4^-11 * 4^-1... = 13 * 4^-12 per window pair."""
    st = synth.Stream(22, "count")
    n = m = 150_000
    T = synth.iid_bases(st.child("T"), n, 0.5)
    Q = synth.iid_bases(st.child("Q"), m, 0.5)
    t, q = oracle.seed_hits(T, Q)
    expect = (n - 18) * (m - 18) * 13 * 4.0 ** -12
    # windows overlap along a diagonal, so the spread is a few times Poisson
    assert abs(t.size - expect) < 8 * np.sqrt(expect), (t.size, expect)


def test_hoxd70_published_symmetries():
    M = oracle.HOXD70
    comp = [3, 2, 1, 0]
    assert np.array_equal(M, M.T)
    for a in range(4):
        for b in range(4):
            assert M[a, b] == M[comp[a], comp[b]]
    # the four transitions score alike and every transversion scores below them
    assert {M[0, 2], M[2, 0], M[1, 3], M[3, 1]} == {-31}
    assert oracle.XDROP == 10 * M[0, 0]


@pytest.mark.parametrize("qtile,threads", [(0, 1), (0, 4), (1, 2), (97, 3), (1000, 8), (4096, 5)])
def test_parallel_form_equals_serial(qtile, threads):
    """or_run_par (query tiles with the skip state carried, blocks of diagonals
    walked on several threads) gives the serial oracle's HSPs and counters."""
    T, Q = _rand_pair(21, 6000, 5000)
    ref = oracle.run(T, Q, thresh=800)
    got = oracle.run_par(T, Q, thresh=800, qtile=qtile, threads=threads)
    assert np.array_equal(got.hsps, ref.hsps) and ref.hsps.size > 0
    assert (got.hits, got.extended, got.cells) == (ref.hits, ref.extended, ref.cells)


@pytest.mark.parametrize("n,m", [(0, 0), (0, 50), (50, 0), (18, 18), (19, 19), (19, 40),
                                 (40, 19), (33, 4097)])
def test_parallel_form_ragged_and_empty(n, m):
    T, Q = _rand_pair(22, n, m, homology=False)
    ref = oracle.run(T, Q, thresh=0)
    for qtile, threads in ((0, 3), (7, 2)):
        got = oracle.run_par(T, Q, thresh=0, qtile=qtile, threads=threads)
        assert np.array_equal(got.hsps, ref.hsps)
        assert (got.hits, got.extended, got.cells) == (ref.hits, ref.extended, ref.cells)


def test_parallel_form_dense_diagonals_across_tiles():
    """Identical sequences and a period-19 repeat: long diagonals full of
    skipped hits, cut by query tiles of 13 positions."""
    for kind in ("polyA", "period19", "identical"):
        T, Q = _adversarial_pair(kind)
        ref = oracle.run(T, Q, thresh=0)
        got = oracle.run_par(T, Q, thresh=0, qtile=13, threads=4)
        assert np.array_equal(got.hsps, ref.hsps)
        assert (got.hits, got.extended, got.cells) == (ref.hits, ref.extended, ref.cells)


# ------------------------------------------------------------------ heavier seeds and step
# Section 7 raises the seed weight (14 of 22) and the spacing between indexed
# target positions (the step). The oracle's reading: with step s only target
# positions t with t % s == 0 are in the position table.

P22 = "1110111000011101011011"  # the 14-of-22 mask of this build (weight 14, span 22)


def test_heavier_mask_shape():
    assert len(P22) == 22 and P22.count("1") == 14 and P22[0] == P22[-1] == "1"


@pytest.mark.parametrize("pattern,transition,step", [
    (P19, True, 2), (P19, True, 3), (P19, False, 5), (P22, True, 1), (P22, True, 4),
    ("1101011", True, 7),
])
def test_hits_with_step_match_bruteforce(pattern, transition, step):
    assert check_hits_bruteforce(13, 2500, 2200, pattern, transition, 0.5, step)


@pytest.mark.parametrize("pattern,step", [(P19, 3), (P22, 1), (P22, 2)])
def test_skip_with_step_matches_serial_query_order(pattern, step):
    assert check_serial_loop(14, 2600, 2400, thresh=1200, pattern=pattern, step=step)


def test_step_one_is_the_default_and_steps_only_thin_the_hits():
    T, Q = _rand_pair(15, 4000, 3500)
    base = oracle.run(T, Q, thresh=800)
    assert np.array_equal(oracle.run(T, Q, thresh=800, step=1).hsps, base.hsps)
    t1, q1 = oracle.seed_hits(T, Q)
    for s in (2, 3, 8):
        t, q = oracle.seed_hits(T, Q, step=s)
        keep = t1 % s == 0
        assert np.array_equal(t, t1[keep]) and np.array_equal(q, q1[keep])


@pytest.mark.parametrize("step", [2, 5])
def test_parallel_form_with_step(step):
    T, Q = _rand_pair(16, 5000, 4500)
    ref = oracle.run(T, Q, P22, thresh=600, step=step)
    got = oracle.run_par(T, Q, P22, thresh=600, step=step, qtile=333, threads=3)
    assert np.array_equal(got.hsps, ref.hsps)
    assert (got.hits, got.extended, got.cells) == (ref.hits, ref.extended, ref.cells)


def test_run_diagonal_with_step_agrees_with_run():
    """The one-diagonal walk with a step: its HSPs equal the whole run's on that
    diagonal, and its hit count equals the brute force's hits there."""
    T, Q = _rand_pair(17, 2500, 2500)
    full = oracle.run(T, Q, strands=1, thresh=0, keep_log=True, step=3)
    bt, bq = bf.hits_by_diagonal(T, Q, P19, True, 3)
    diags = np.unique(full.ext["t"] - full.ext["q"])
    st = synth.Stream(2, "diag")
    for d in diags[st.integers(0, diags.size, 20)]:
        one = oracle.run_diagonal(T, Q, 0, int(d), thresh=0, step=3)
        mine = full.hsps[full.hsps["tpos"] - full.hsps["qpos"] == d]
        assert np.array_equal(one.hsps, mine)
        assert one.hits == int(np.count_nonzero(bt - bq == d))
