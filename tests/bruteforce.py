"""Independent brute-force restatements used to pin the oracle.

These are written in a different shape from the oracle (numpy over whole
diagonals and whole prefix-sum arrays instead of an index and serial loops),
so that a mistake in one is not repeated in the other.
"""
from __future__ import annotations

import numpy as np


def care_offsets(pattern: str) -> list[int]:
    return [i for i, c in enumerate(pattern) if c == "1"]


def revcomp(x: np.ndarray) -> np.ndarray:
    # complement by table lookup rather than by xor
    comp = np.array([3, 2, 1, 0], dtype=np.uint8)
    return comp[np.asarray(x, dtype=np.uint8)][::-1].copy()


def hits_by_diagonal(T, Qs, pattern: str, transition: bool, step: int = 1):
    """Every (t, q) hit by testing every window of every diagonal. O(|T||Q|).
    With a step, only windows that start at a target position divisible by it."""
    T = np.asarray(T, dtype=np.int16)
    Qs = np.asarray(Qs, dtype=np.int16)
    span = len(pattern)
    care = care_offsets(pattern)
    ts, qs = [], []
    for d in range(-(len(Qs) - span), len(T) - span + 1):
        t0 = max(0, d)
        q0 = t0 - d
        n = min(len(T) - t0, len(Qs) - q0)
        nwin = n - span + 1
        if nwin <= 0:
            continue
        a = T[t0:t0 + n]
        b = Qs[q0:q0 + n]
        same = a == b
        # transition partner: A<->G and C<->T, written as an explicit pair set
        trans = ((a == 0) & (b == 2)) | ((a == 2) & (b == 0)) | ((a == 1) & (b == 3)) | \
                ((a == 3) & (b == 1))
        mism = np.zeros(nwin, dtype=np.int32)
        ntr = np.zeros(nwin, dtype=np.int32)
        for c in care:
            mism += ~same[c:c + nwin]
            ntr += trans[c:c + nwin]
        ok = mism == 0
        if transition:
            ok |= (mism == 1) & (ntr == 1)
        idx = np.flatnonzero(ok)
        if idx.size:
            ts.append(t0 + idx)
            qs.append(q0 + idx)
    if not ts:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    t = np.concatenate(ts).astype(np.int64)
    q = np.concatenate(qs).astype(np.int64)
    keep = t % step == 0
    t, q = t[keep], q[keep]
    order = np.lexsort((t, t - q))
    return t[order], q[order]


def _side(s: np.ndarray, X: int):
    """(best length, bases scored, best) of one extension from its score sequence.

    Exhaustive over prefix sums: the running maximum includes the empty
    extension (0); the scan ends at the first index where max - sum > X (that
    base is scored) or at the end of the data; the best length is the first
    index attaining the final maximum.
    """
    if s.size == 0:
        return 0, 0, 0
    P = np.cumsum(s.astype(np.int64))
    B = np.maximum.accumulate(np.maximum(P, 0))
    over = np.flatnonzero(B - P > X)
    K = int(over[0]) if over.size else s.size - 1
    best = int(B[K])
    if best <= 0:
        return 0, K + 1, 0
    first = int(np.flatnonzero(P[:K + 1] == best)[0])
    return first + 1, K + 1, best


def extend(T, Qs, t: int, q: int, span: int, M, X: int) -> dict:
    T = np.asarray(T, dtype=np.int64)
    Qs = np.asarray(Qs, dtype=np.int64)
    M = np.asarray(M, dtype=np.int64).reshape(4, 4)
    seed = int(M[T[t:t + span], Qs[q:q + span]].sum())
    nr = min(len(T) - t - span, len(Qs) - q - span)
    right = M[T[t + span:t + span + nr], Qs[q + span:q + span + nr]]
    nl = min(t, q)
    left = M[T[t - nl:t][::-1], Qs[q - nl:q][::-1]] if nl > 0 else np.zeros(0, np.int64)
    rl, rs, rb = _side(right, X)
    ll, ls, lb = _side(left, X)
    return {"tpos": t - ll, "qpos": q - ll, "len": span + ll + rl, "score": seed + rb + lb,
            "end": t + span + rl, "cells": span + rs + ls}


def serial_query_order(T, Q, pattern, transition, strands, M, X, thresh, skip_passing_only=False,
                       step=1):
    """Algorithm 1's shape: one pass over the hits in query order, with a masking
    state kept per (strand, diagonal). Hits from `hits_by_diagonal`, extensions
    from `extend` above."""
    span = len(pattern)
    out = []
    st = {"hits": 0, "extended": 0, "cells": 0}
    for s in (0, 1):
        if not strands & (1 << s):
            continue
        Qs = Q if s == 0 else revcomp(Q)
        t, q = hits_by_diagonal(T, Qs, pattern, transition, step)
        order = np.lexsort((t, q))
        E = {}
        for i in order:
            ti, qi = int(t[i]), int(q[i])
            st["hits"] += 1
            d = ti - qi
            if ti < E.get(d, -(1 << 62)):
                continue
            e = extend(T, Qs, ti, qi, span, M, X)
            st["extended"] += 1
            st["cells"] += e["cells"]
            if e["score"] >= thresh or not skip_passing_only:
                E[d] = e["end"]
            if e["score"] >= thresh:
                out.append((s, e["tpos"], e["qpos"], e["len"], e["score"]))
    out.sort()
    return out, st


def gotoh_half_full(Tseg, Qseg, M, gap_open, gap_extend):
    """Affine-gap DP of one extension half over whole segments, no pruning:
    Tseg / Qseg already oriented (step k consumes Tseg[k-1]). Row by row,
    H[0][0] = 0, a gap of L bases costs open + L * extend. Returns the H matrix."""
    n, m = len(Tseg), len(Qseg)
    NEG = -(1 << 40)
    H = np.full((n + 1, m + 1), NEG, dtype=np.int64)
    E = np.full((n + 1, m + 1), NEG, dtype=np.int64)
    F = np.full((n + 1, m + 1), NEG, dtype=np.int64)
    H[0, 0] = 0
    M = np.asarray(M, dtype=np.int64).reshape(4, 4)
    for i in range(n + 1):
        for j in range(m + 1):
            if i == 0 and j == 0:
                continue
            e = max(E[i, j - 1] - gap_extend, H[i, j - 1] - gap_open - gap_extend) if j else NEG
            f = max(F[i - 1, j] - gap_extend, H[i - 1, j] - gap_open - gap_extend) if i else NEG
            dg = H[i - 1, j - 1] + M[Tseg[i - 1], Qseg[j - 1]] if i and j else NEG
            E[i, j], F[i, j] = e, f
            H[i, j] = max(dg, e, f)
    return H


def first_max_by_antidiagonal(H):
    """Maximum of H and its first cell in the order (i + j, then i)."""
    best = int(H.max())
    cells = [(i + j, i, j) for i, j in zip(*np.nonzero(H == best))]
    d, i, j = min(cells)
    return best, int(i), int(j)


def ydrop_half_sets(Tseg, Qseg, M, gap_open, gap_extend, Y, band):
    """The Y-drop half written with Python sets and dicts: live cells of the last
    two anti-diagonals; the candidates of anti-diagonal d are every i from the
    lowest to the highest cell next to a live cell of d - 1 or one diagonal
    step from a live cell of d - 2 (inside the matrix), the `band` of lowest i
    kept; stop after two anti-diagonals without a live cell. Returns
    (best, i, j, cells) with the first best cell by (anti-diagonal, i)."""
    n, m = len(Tseg), len(Qseg)
    M = np.asarray(M, dtype=np.int64).reshape(4, 4)
    prev2, prev1 = {}, {(0, 0): (0, None, None)}  # cell -> (H, E, F) of live cells
    best, bi, bj, cells = 0, 0, 0, 0
    d = 0
    while prev1 or prev2:
        d += 1
        cand = {i for (i, j) in prev1} | {i + 1 for (i, j) in prev1} | \
            {i + 1 for (i, j) in prev2}
        cand = [i for i in range(min(cand), max(cand) + 1) if 0 <= i <= n and 0 <= d - i <= m]
        cand = cand[:band]
        cur, dbest, dcell = {}, None, None
        for i in cand:
            j = d - i
            cells += 1
            opts = []
            if (i - 1, j - 1) in prev2 and i >= 1 and j >= 1:
                opts.append(prev2[(i - 1, j - 1)][0] + M[Tseg[i - 1], Qseg[j - 1]])
            e = f = None
            if (i, j - 1) in prev1:
                h1, e1, _ = prev1[(i, j - 1)]
                e = h1 - gap_open - gap_extend if e1 is None else max(
                    e1 - gap_extend, h1 - gap_open - gap_extend)
                opts.append(e)
            if (i - 1, j) in prev1:
                h1, _, f1 = prev1[(i - 1, j)]
                f = h1 - gap_open - gap_extend if f1 is None else max(
                    f1 - gap_extend, h1 - gap_open - gap_extend)
                opts.append(f)
            if not opts:
                continue
            h = max(opts)
            if h < best - Y:
                continue
            cur[(i, j)] = (h, e, f)
            if dbest is None or h > dbest:
                dbest, dcell = h, (i, j)
        if dbest is not None and dbest > best:
            best, (bi, bj) = dbest, dcell
        prev2, prev1 = prev1, cur
        if not prev1 and not prev2:
            break
    return best, bi, bj, cells
