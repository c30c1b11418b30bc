"""Parity at full workload sizes, in the launch configuration the benchmark uses.

The oracle cannot run a whole 10 Mb x 10 Mb pair in test time, but it can
walk single diagonals exactly (hits found by testing every position of the
diagonal), so sampled diagonals are compared HSP by HSP, and properties that
hold at any size are checked on every HSP.
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


def run_gpu(P, pair, **kw):
    import torch
    dev = torch.device("cuda", 0)
    T = torch.from_numpy(np.frombuffer(synth.decode(pair.T), np.uint8).copy()).to(dev)
    Q = torch.from_numpy(np.frombuffer(synth.decode(pair.Q), np.uint8).copy()).to(dev)
    with P.Context(0) as ctx:
        hsps, st = ctx.run(T, Q, P.default_params(**kw), cap=1 << 22)
    return np.ascontiguousarray(hsps).view(np.int32).reshape(-1, 5), st


def check_scores(pair, H):
    """Every HSP score is the sum of its substitution scores; spans in bounds."""
    M = oracle.HOXD70.astype(np.int64)
    Qm = bf.revcomp(pair.Q)
    assert (H[:, 3] >= 19).all()
    for s, Qs in ((0, pair.Q), (1, Qm)):
        h = H[H[:, 0] == s]
        if h.size == 0:
            continue
        t0, q0, L = h[:, 1].astype(np.int64), h[:, 2].astype(np.int64), h[:, 3].astype(np.int64)
        assert (t0 >= 0).all() and (q0 >= 0).all()
        assert (t0 + L <= pair.tlen).all() and (q0 + L <= pair.qlen).all()
        starts = np.concatenate([[0], np.cumsum(L)[:-1]])
        off = np.arange(int(L.sum())) - np.repeat(starts, L)
        tt = np.repeat(t0, L) + off
        qq = np.repeat(q0, L) + off
        cell = M[pair.T[tt], Qs[qq]]
        sums = np.add.reduceat(cell, starts)
        assert np.array_equal(sums, h[:, 4].astype(np.int64))


def check_diagonals(pair, H, picks):
    Qm = bf.revcomp(pair.Q)
    for s, d in picks:
        Qs = pair.Q if s == 0 else Qm
        ref = oracle.run_diagonal(pair.T, Qs, s, d)
        mine = H[(H[:, 0] == s) & (H[:, 1] - H[:, 2] == d)]
        assert np.array_equal(mine, ref.hsps.view(np.int32).reshape(-1, 5)), (s, d)


def pick_diagonals(pair, H, n_hsp, n_rand, seed):
    st = synth.Stream(seed, "diag")
    picks = []
    if H.shape[0]:
        for i in st.integers(0, H.shape[0], n_hsp):
            picks.append((int(H[i, 0]), int(H[i, 1] - H[i, 2])))
    lo, hi = -(pair.qlen - 19), pair.tlen - 19
    for i, d in enumerate(st.integers(lo, hi + 1, n_rand)):
        picks.append((i % 2, int(d)))
    # the blocks' own diagonals (dense in hits, many skips)
    for b in pair.blocks[:4]:
        if not b.rc:
            picks.append((0, b.tstart - b.qstart))
    return picks


def test_plain_pair_10mb_full_size(pkg):
    pair = synth.plain_pair_10mb(2)  # the benchmark's workload and seed
    H, st = run_gpu(pkg, pair)
    assert st["hits"] > 1e8 and H.shape[0] > 1e5
    check_scores(pair, H)
    check_diagonals(pair, H, pick_diagonals(pair, H, 8, 6, 1))


def test_large_pair_100mb_full_size_tiled(pkg):
    pair = synth.large_pair_100mb(5)
    H, st = run_gpu(pkg, pair)
    assert st["tiles"] > 10  # the query is tiled, with the skip state carried across tiles
    assert H.shape[0] > 1e6
    sub = H[synth.Stream(9, "sub").integers(0, H.shape[0], 200_000)]
    check_scores(pair, sub)
    check_diagonals(pair, H, pick_diagonals(pair, H, 5, 3, 2))
