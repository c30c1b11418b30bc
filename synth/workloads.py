"""The five synthetic workloads of the hot path, by what they are.

* tiny_pair: 200 kb x 200 kb, uniform ACGT, 50 planted homologous segments of
  300-2000 bp at 85% identity (Ts:Tv 2:1, 1% short indels).
* plain_pair_10mb: 10 Mb x 10 Mb at 41% GC, 5% repeats from 20 consensuses of
  300 bp at 10% divergence, 2000 planted blocks of 1-20 kb (log-uniform) at
  70-90% identity, half reverse-complemented.
* batch_pairs: 4096 uneven pairs, lengths log-uniform 1-256 kb, GC uniform
  35-60%, 0-20 planted blocks each at 70-90% identity.
* large_pair_100mb: 100 Mb x 100 Mb at 41% GC, 8% repeats from 50 consensuses
  of 300-6000 bp at 5-20% divergence, 20000 planted blocks of 1-50 kb at
  65-90% identity, half inverted (reverse-complemented), all moved to random
  query positions (translocations).

Every function takes a `scale` in (0, 1] that shrinks sequence lengths and
block/repeat counts proportionally, for tests.
"""
from __future__ import annotations

import numpy as np

from .genome import Pair, iid_bases, plant_blocks, plant_repeats
from .rng import Stream

INDEL_RATE = 0.01


def tiny_pair(seed: int = 1, scale: float = 1.0, length: int = 200_000,
              n_blocks: int = 50) -> Pair:
    st = Stream(seed, "tiny_pair")
    n = max(1, int(length * scale))
    T = iid_bases(st.child("T"), n, 0.5)
    Q = iid_bases(st.child("Q"), n, 0.5)
    nb = max(0, int(round(n_blocks * scale)))
    blocks = plant_blocks(st.child("blocks"), T, Q, nb, 300, 2000, 0.85, 0.85, 0.0,
                          INDEL_RATE, 0.5)
    return Pair(T, Q, blocks, f"tiny_pair(seed={seed},n={n})", 0.5)


def plain_pair_10mb(seed: int = 2, scale: float = 1.0) -> Pair:
    st = Stream(seed, "plain_pair_10mb")
    n = max(1000, int(10_000_000 * scale))
    gc = 0.41
    T = iid_bases(st.child("T"), n, gc)
    Q = iid_bases(st.child("Q"), n, gc)
    plant_repeats(st.child("rep"), [T, Q], 0.05, 20, 300, 300, 0.10, 0.10, gc)
    nb = max(1, int(round(2000 * scale)))
    blocks = plant_blocks(st.child("blocks"), T, Q, nb, 1000, 20000, 0.70, 0.90, 0.5,
                          INDEL_RATE, gc)
    return Pair(T, Q, blocks, f"plain_pair_10mb(seed={seed},n={n})", gc)


def batch_pairs(seed: int = 3, n_pairs: int = 4096, len_lo: int = 1000,
                len_hi: int = 256_000) -> list[Pair]:
    st = Stream(seed, "batch_pairs")
    tl = st.child("tlen").log_uniform_int(len_lo, len_hi, n_pairs)
    ql = st.child("qlen").log_uniform_int(len_lo, len_hi, n_pairs)
    gcs = 0.35 + 0.25 * st.child("gc").uniform(n_pairs)
    nbs = st.child("nblocks").integers(0, 21, n_pairs)
    out = []
    for i in range(n_pairs):
        pst = st.child("pair", i)
        gc = float(gcs[i])
        T = iid_bases(pst.child("T"), int(tl[i]), gc)
        Q = iid_bases(pst.child("Q"), int(ql[i]), gc)
        hi = int(min(20000, tl[i], ql[i]))
        blocks = plant_blocks(pst.child("blocks"), T, Q, int(nbs[i]), min(300, hi), hi,
                              0.70, 0.90, 0.5, INDEL_RATE, gc)
        out.append(Pair(T, Q, blocks, f"batch_pairs[{i}]", gc))
    return out


def large_pair_100mb(seed: int = 5, scale: float = 1.0) -> Pair:
    st = Stream(seed, "large_pair_100mb")
    n = max(1000, int(100_000_000 * scale))
    gc = 0.41
    T = iid_bases(st.child("T"), n, gc)
    Q = iid_bases(st.child("Q"), n, gc)
    plant_repeats(st.child("rep"), [T, Q], 0.08, 50, 300, 6000, 0.05, 0.20, gc)
    nb = max(1, int(round(20000 * scale)))
    blocks = plant_blocks(st.child("blocks"), T, Q, nb, 1000, 50000, 0.65, 0.90, 0.5,
                          INDEL_RATE, gc)
    return Pair(T, Q, blocks, f"large_pair_100mb(seed={seed},n={n})", gc)


WORKLOADS = {
    "tiny_pair": tiny_pair,
    "plain_pair_10mb": plain_pair_10mb,
    "batch_pairs": batch_pairs,
    "large_pair_100mb": large_pair_100mb,
}


def concat_batch(pairs: list[Pair]):
    """Concatenate a batch into flat code arrays plus int64 offsets (n+1 each)."""
    toff = np.zeros(len(pairs) + 1, dtype=np.int64)
    qoff = np.zeros(len(pairs) + 1, dtype=np.int64)
    toff[1:] = np.cumsum([p.tlen for p in pairs])
    qoff[1:] = np.cumsum([p.qlen for p in pairs])
    T = np.concatenate([p.T for p in pairs]) if pairs else np.zeros(0, np.uint8)
    Q = np.concatenate([p.Q for p in pairs]) if pairs else np.zeros(0, np.uint8)
    return T, toff, Q, qoff
