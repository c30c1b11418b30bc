"""Pins of the oracle's gapped (Y-drop) stage (Algorithm 1 and Algorithm 3).

* brute force: with Y and the band too large to prune anything, a half
  extension's best and its first best cell equal those of the whole
  affine-gap DP matrix computed row by row (tests/bruteforce.py);
* reduction to the filter: when a gap can never stay live (gap open > Y), the
  Y-drop half is the ungapped X-drop side with X = Y (the pinned or_xdrop);
* a worked case: two matching segments split by a 2-base insertion align as
  one alignment whose score is both segments minus open + 2 x extend;
* symmetry: swapping T and Q with the transposed matrix keeps the best score;
* Algorithm 3 with any batch size commits exactly Algorithm 1's alignments
  (the paper's claim for its speculative batches), and its skipped plus
  shadow anchors are Algorithm 1's skipped anchors;
* workload fact: planted segments with 1% indels, split into several HSPs by
  the filter, come out as one gapped alignment each.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from tests import bruteforce as bf


def _seq(st, n, gc=0.5):
    return synth.iid_bases(st, n, gc)


def _mutate(st, src, identity):
    return synth.mutate(st, src, identity, indel_rate=0.0, gc=0.5)


def check_half_bruteforce(seed=1, reps=30) -> bool:
    st = synth.Stream(seed, "ybf")
    for r in range(reps):
        n, m = st.child("n", r).integers(1, 28, 2)
        T = _seq(st.child("T", r), int(n))
        Q = _mutate(st.child("Q", r), T[: int(m)] if m <= n else np.concatenate(
            [T, _seq(st.child("x", r), int(m - n))]), 0.7)
        M = oracle.HOXD70 if r % 2 == 0 else _asym(st.child("M", r))
        go, ge = (400, 30) if r % 3 else (60, 15)
        for direction in (+1, -1):
            if direction > 0:
                h = oracle.ydrop_half(T, 0, Q, 0, +1, M, go, ge, Y=1 << 28, band=1024)
                H = bf.gotoh_half_full(T, Q, M, go, ge)
            else:
                h = oracle.ydrop_half(T, T.size, Q, Q.size, -1, M, go, ge, Y=1 << 28, band=1024)
                H = bf.gotoh_half_full(T[::-1], Q[::-1], M, go, ge)
            best, i, j = bf.first_max_by_antidiagonal(H)
            if (h["best"], h["bi"], h["bj"]) != (best, i, j):
                return False
    return True


def _asym(st):
    M = st.integers(-80, 30, 16).reshape(4, 4).astype(np.int32)
    M[np.arange(4), np.arange(4)] = st.integers(60, 110, 4)
    return M


# Small cases where the best score is reached by two cells of one
# anti-diagonal (found by a search over random sequences with the brute
# force): the half must report the one with the lower i.
TIE_CASES = [([2, 0, 2, 1], [2, 1, 2], 0, 5), ([2, 1], [3, 1, 2], 0, 10),
             ([2, 1, 3, 3], [1, 2, 0], 10, 0), ([1, 2, 3, 3, 3, 2], [2, 1, 0, 1, 1], 10, 0)]


def check_ties() -> bool:
    for T, Q, go, ge in TIE_CASES:
        T, Q = np.array(T, np.uint8), np.array(Q, np.uint8)
        h = oracle.ydrop_half(T, 0, Q, 0, +1, oracle.HOXD70, go, ge, Y=1 << 28, band=64)
        best, i, j = bf.first_max_by_antidiagonal(bf.gotoh_half_full(T, Q, oracle.HOXD70, go, ge))
        if (h["best"], h["bi"], h["bj"]) != (best, i, j):
            return False
    return True


def test_half_matches_the_whole_dp_when_nothing_is_pruned():
    assert check_half_bruteforce(1, 40)


def test_ties_on_one_anti_diagonal_take_the_lower_i():
    assert check_ties()


def check_gap_free_is_xdrop(seed=2, reps=40) -> bool:
    st = synth.Stream(seed, "yx")
    T = _seq(st.child("T"), 3000)
    Q = T.copy()
    Q[::7] = _seq(st.child("m"), Q[::7].size)  # about 1/7 substitutions, no indels
    for r in range(reps):
        t = int(st.child("t", r).integers(40, 2900, 1)[0])
        Y = int(st.child("Y", r).integers(100, 3000, 1)[0])
        x = oracle.xdrop(T, Q, t, t, span=0, X=Y)
        f = oracle.ydrop_half(T, t, Q, t, +1, gap_open=Y + 1, gap_extend=1, Y=Y)
        b = oracle.ydrop_half(T, t, Q, t, -1, gap_open=Y + 1, gap_extend=1, Y=Y)
        if (f["bi"], f["bj"], b["bi"], b["bj"]) != (x["rext"], x["rext"], x["lext"], x["lext"]):
            return False
        if f["best"] + b["best"] != x["score"]:
            return False
    return True


def test_gap_free_half_is_the_xdrop_side():
    assert check_gap_free_is_xdrop()


def check_insertion_case() -> bool:
    st = synth.Stream(3, "yins")
    A, B = _seq(st.child("A"), 80), _seq(st.child("B"), 80)
    T = np.concatenate([A, B])
    Q = np.concatenate([A, np.array([2, 2], np.uint8), B])
    M = oracle.HOXD70.astype(np.int64)
    full = int(M[A, A].sum() + M[B, B].sum() - (400 + 2 * 30))
    h = oracle.ydrop_half(T, 0, Q, 0, +1)
    return h["best"] == full and (h["bi"], h["bj"]) == (160, 162)


def test_insertion_is_bridged():
    assert check_insertion_case()


def check_swap(seed=4) -> bool:
    st = synth.Stream(seed, "yswap")
    T = _seq(st.child("T"), 400)
    Q = synth.mutate(st.child("Q"), T, 0.8, indel_rate=0.02, gc=0.5)
    M = _asym(st.child("M"))
    a = oracle.ydrop_half(T, 0, Q, 0, +1, M, 300, 20, Y=2000)
    b = oracle.ydrop_half(Q, 0, T, 0, +1, M.T.copy(), 300, 20, Y=2000)
    return a["best"] == b["best"] and a["best"] > 0


def test_swapping_target_and_query_keeps_the_score():
    assert check_swap()


def _pair_with_hsps(seed, n=60_000, blocks=12):
    p = synth.tiny_pair(seed, length=n, n_blocks=blocks)
    r = oracle.run(p.T, p.Q)
    return p, r.hsps


def check_batches_equal_serial(seed=5, batches=(1, 2, 7, 1000)) -> bool:
    p, H = _pair_with_hsps(seed)
    ref = oracle.gapped(p.T, p.Q, H)
    if ref.aligns.size == 0:
        return False
    for K in batches:
        g = oracle.gapped(p.T, p.Q, H, batch=K)
        if not np.array_equal(g.aligns, ref.aligns):
            return False
        s, r = g.stats, ref.stats
        if s["skipped"] + s["shadow"] != r["skipped"] or s["extended"] != r["extended"]:
            return False
        if s["cells"] != r["cells"] or (K == 1 and s["shadow"] != 0):
            return False
    return True


def test_speculative_batches_commit_the_serial_alignments():
    assert check_batches_equal_serial()


def check_planted_segments_one_alignment_each(seed=6) -> bool:
    """Blocks of 1.5-3 kb at 85-95% identity with 1% indels: the filter splits
    them into several HSPs, the gapped stage aligns each in one piece."""
    st = synth.Stream(seed, "yplant")
    T = _seq(st.child("T"), 80_000)
    Q = _seq(st.child("Q"), 80_000)
    blocks = synth.plant_blocks(st.child("b"), T, Q, 8, 1500, 3000, 0.85, 0.95, 0.0, 0.01, 0.5)
    H = oracle.run(T, Q).hsps
    g = oracle.gapped(T, Q, H)
    ok = 0
    for b in blocks:
        on = g.aligns[(g.aligns["strand"] == 0) & (g.aligns["tstart"] < b.tstart + b.tlen) &
                      (g.aligns["tend"] > b.tstart)]
        if on.size == 1 and (on["tend"] - on["tstart"])[0] >= 0.9 * b.tlen:
            ok += 1
        hs = H[(H["strand"] == 0) & (H["tpos"] < b.tstart + b.tlen) &
               (H["tpos"] + H["len"] > b.tstart)]
    return ok >= len(blocks) - 1 and H.size > g.aligns.size


def test_planted_segments_align_in_one_piece():
    assert check_planted_segments_one_alignment_each()


def check_band_and_pruning_setwise(seed=7, reps=30) -> bool:
    """Pruned and banded halves (finite Y, small bands) against the set-based
    restatement, cells included."""
    st = synth.Stream(seed, "yset")
    for r in range(reps):
        n = int(st.child("n", r).integers(5, 70, 1)[0])
        T = _seq(st.child("T", r), n)
        Q = synth.mutate(st.child("Q", r), T, 0.75, indel_rate=0.05, gc=0.5)
        Y = int(st.child("Y", r).integers(50, 1500, 1)[0])
        band = int([1, 2, 3, 5, 8, 64][r % 6])
        go, ge = [(400, 30), (40, 10), (120, 5)][r % 3]
        h = oracle.ydrop_half(T, 0, Q, 0, +1, oracle.HOXD70, go, ge, Y, band)
        ref = bf.ydrop_half_sets(T, Q, oracle.HOXD70, go, ge, Y, band)
        if (h["best"], h["bi"], h["bj"], h["cells"]) != ref:
            return False
    return True


def test_pruning_and_band_match_the_set_restatement():
    assert check_band_and_pruning_setwise()


def stage_restated(T, Q, H, thresh=oracle.GAPPED_THRESH):
    """Algorithm 1's loop written out in Python around the (separately pinned)
    half extension: HSPs by decreasing score (then strand, tpos, qpos, len),
    anchor at the HSP's midpoint, skipped when inside the box of an alignment
    committed on its strand, committed when the two halves reach thresh.
    Returns (committed boxes sorted, anchors extended, their DP cells)."""
    Qm = bf.revcomp(Q)
    order = sorted(range(H.size), key=lambda k: (-int(H["score"][k]), int(H["strand"][k]),
                                                  int(H["tpos"][k]), int(H["qpos"][k]),
                                                  int(H["len"][k])))
    boxes, extended, cells = [], 0, 0
    for k in order:
        s, tp, qp, ln = (int(H[f][k]) for f in ("strand", "tpos", "qpos", "len"))
        ta, qa = tp + ln // 2, qp + ln // 2
        if any(b[0] == s and b[1] <= ta < b[2] and b[3] <= qa < b[4] for b in boxes):
            continue
        Qs = Q if s == 0 else Qm
        f = oracle.ydrop_half(T, ta, Qs, qa, +1)
        r = oracle.ydrop_half(T, ta, Qs, qa, -1)
        extended += 1
        cells += f["cells"] + r["cells"]
        score = f["best"] + r["best"]
        if score >= thresh:
            boxes.append((s, ta - r["bi"], ta + f["bi"], qa - r["bj"], qa + f["bj"], score))
    return sorted(boxes, key=lambda b: (b[0], b[1], b[3], b[2], b[4], b[5])), extended, cells


def _with_boundary_anchors(p, H):
    """H plus two low-scoring one-base records whose midpoints sit exactly on
    the end of the first committed box and one base inside it."""
    g = oracle.gapped(p.T, p.Q, H)
    b = g.aligns[0]
    qa = (int(b["qstart"]) + int(b["qend"])) // 2
    extra = np.zeros(2, dtype=oracle.HSP_DTYPE)
    for r, t in enumerate((int(b["tend"]), int(b["tend"]) - 1)):
        extra[r] = (int(b["strand"]), t, qa, 1, -1000 - r)
    return np.concatenate([H, extra])


def check_stage_restated(seed=8, thresh=oracle.GAPPED_THRESH) -> bool:
    p, H = _pair_with_hsps(seed, 50_000, 10)
    H = _with_boundary_anchors(p, H)
    g = oracle.gapped(p.T, p.Q, H, thresh=thresh)
    got = [tuple(int(x) for x in (a["strand"], a["tstart"], a["tend"], a["qstart"], a["qend"],
                                  a["score"])) for a in g.aligns]
    ref, extended, cells = stage_restated(p.T, p.Q, H, thresh)
    return (got == ref and len(ref) > 0 and g.stats["extended"] == extended and
            g.stats["cells"] == cells and g.stats["skipped"] > 0)


@pytest.mark.parametrize("thresh", [oracle.GAPPED_THRESH, 6000])
def test_stage_matches_algorithm_1_written_out(thresh):
    assert check_stage_restated(8, thresh)
