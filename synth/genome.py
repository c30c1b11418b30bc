"""Building blocks of the synthetic genome pairs.

Codes: A=0, C=1, G=2, T=3 (one uint8 per base). The complement of x is x^3 and
the transition partner of x (A<->G, C<->T) is x^2. These are input-construction
helpers only.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .rng import Stream

BASES = np.frombuffer(b"ACGT", dtype=np.uint8)
_ASCII_TO_CODE = np.full(256, 255, dtype=np.uint8)
for _i, _c in enumerate(b"ACGT"):
    _ASCII_TO_CODE[_c] = _i
    _ASCII_TO_CODE[_c + 32] = _i


def decode(codes: np.ndarray) -> bytes:
    """2-bit codes (one per byte) -> ASCII 'ACGT' bytes."""
    return BASES[np.asarray(codes, dtype=np.uint8)].tobytes()


def encode_ascii(s) -> np.ndarray:
    """ASCII ACGTacgt -> codes; raises on any other symbol."""
    a = np.frombuffer(s.encode() if isinstance(s, str) else bytes(s), dtype=np.uint8)
    c = _ASCII_TO_CODE[a]
    if c.size and c.max() == 255:
        raise ValueError("sequence holds a symbol outside ACGTacgt")
    return c


def iid_bases(st: Stream, n: int, gc: float) -> np.ndarray:
    """n i.i.d. bases with P(C)=P(G)=gc/2 and P(A)=P(T)=(1-gc)/2."""
    pa = (1.0 - gc) / 2.0
    cum = np.array([pa, pa + gc / 2.0, pa + gc], dtype=np.float64)
    return np.searchsorted(cum, st.uniform(n), side="right").astype(np.uint8)


def revcomp_codes(x: np.ndarray) -> np.ndarray:
    return (x[::-1] ^ 3).astype(np.uint8)


def mutate(st: Stream, seq: np.ndarray, identity: float, ts_frac: float = 2.0 / 3.0,
           indel_rate: float = 0.0, indel_max: int = 5, gc: float = 0.5) -> np.ndarray:
    """Copy `seq` with substitutions at rate 1-identity and optional short indels.

    A substituted base becomes its transition partner with probability ts_frac
    (2/3 gives Ts:Tv = 2:1), else one of its two transversion partners with
    equal probability. Indel events start at rate `indel_rate` per base, are an
    insertion or a deletion with equal probability, and have a geometric length
    (p = 1/2) truncated to 1..indel_max. Inserted bases are i.i.d. at `gc`.
    """
    seq = np.asarray(seq, dtype=np.uint8)
    n = seq.size
    out = seq.copy()
    if n == 0:
        return out
    sub = st.uniform(n) < (1.0 - identity)
    k = int(sub.sum())
    if k:
        u = st.uniform(k)
        v = st.uniform(k)
        flip = np.where(u < ts_frac, 2, np.where(v < 0.5, 1, 3)).astype(np.uint8)
        out[sub] ^= flip
    if indel_rate <= 0.0:
        return out
    ev = np.flatnonzero(st.uniform(n) < indel_rate)
    if ev.size == 0:
        return out
    # geometric(1/2) truncated to [1, indel_max]
    g = np.floor(-np.log2(1.0 - st.uniform(ev.size))).astype(np.int64) + 1
    lens = np.minimum(g, indel_max)
    is_ins = st.uniform(ev.size) < 0.5
    # deletions: mark [pos, pos+len) clipped to the sequence
    keep = np.ones(n, dtype=bool)
    dpos, dlen = ev[~is_ins], lens[~is_ins]
    if dpos.size:
        starts = np.repeat(dpos, dlen)
        offs = np.arange(int(dlen.sum())) - np.repeat(np.cumsum(dlen) - dlen, dlen)
        idx = starts + offs
        keep[idx[idx < n]] = False
    ipos, ilen = ev[is_ins], lens[is_ins]
    if ipos.size:
        ins_vals = iid_bases(st, int(ilen.sum()), gc)
        where = np.repeat(ipos, ilen)
        out = np.insert(out, where, ins_vals)
        keep = np.insert(keep, where, np.ones(where.size, dtype=bool))
    return out[keep]


def _place_disjoint(st: Stream, lens: np.ndarray, n: int) -> np.ndarray | None:
    """Random non-overlapping start positions for intervals of `lens` in [0, n).

    Returns None when the intervals cannot fit with some slack.
    """
    total = int(lens.sum())
    if total > 0.8 * n:
        return None
    free = n - total
    order = np.argsort(st.uniform(lens.size), kind="stable")
    cuts = np.sort(st.integers(0, free + 1, lens.size))
    starts = np.empty(lens.size, dtype=np.int64)
    acc = 0
    for rank, i in enumerate(order):
        starts[i] = cuts[rank] + acc
        acc += int(lens[i])
    return starts


def plant_repeats(st: Stream, seqs: list[np.ndarray], frac: float, n_cons: int,
                  cons_len_lo: int, cons_len_hi: int, div_lo: float, div_hi: float,
                  gc: float) -> None:
    """Overwrite about `frac` of each sequence with diverged copies of shared consensuses.

    Each copy takes a random consensus, is mutated with substitutions only at a
    divergence uniform in [div_lo, div_hi], is reverse-complemented with
    probability 1/2 and overwrites a uniform random position.
    """
    cl = st.log_uniform_int(cons_len_lo, cons_len_hi, n_cons)
    cons = [iid_bases(st.child("cons", i), int(cl[i]), gc) for i in range(n_cons)]
    for si, s in enumerate(seqs):
        sst = st.child("copies", si)
        target_bases = int(frac * s.size)
        placed = 0
        j = 0
        while placed < target_bases:
            c = int(sst.integers(0, n_cons, 1)[0])
            div = sst.scalar_uniform(div_lo, div_hi)
            cp = mutate(sst.child("m", j), cons[c], 1.0 - div)
            if sst.uniform(1)[0] < 0.5:
                cp = revcomp_codes(cp)
            if cp.size >= s.size:
                break
            p = int(sst.integers(0, s.size - cp.size + 1, 1)[0])
            s[p:p + cp.size] = cp
            placed += cp.size
            j += 1


@dataclass
class Block:
    tstart: int
    tlen: int
    qstart: int
    qlen: int
    identity: float
    rc: bool


def plant_blocks(st: Stream, T: np.ndarray, Q: np.ndarray, n_blocks: int, len_lo: int,
                 len_hi: int, id_lo: float, id_hi: float, rc_prob: float,
                 indel_rate: float, gc: float) -> list[Block]:
    """Copy `n_blocks` homologous blocks from T into Q (Q is modified in place).

    Lengths are log-uniform on [len_lo, len_hi], identity uniform on
    [id_lo, id_hi], Ts:Tv 2:1, short indels at `indel_rate`. A block is
    reverse-complemented with probability rc_prob. Positions are disjoint in
    both sequences when the blocks fit, else independent and uniform (later
    blocks overwrite earlier ones in Q).
    """
    if n_blocks == 0 or T.size < len_lo or Q.size < len_lo:
        return []
    hi = min(len_hi, T.size, Q.size)
    lo = min(len_lo, hi)
    lens = st.log_uniform_int(lo, hi, n_blocks)
    ts = _place_disjoint(st.child("tpos"), lens, T.size)
    if ts is None:
        ts = np.array([int(st.integers(0, T.size - L + 1, 1)[0]) for L in lens])
    ids = id_lo + (id_hi - id_lo) * st.uniform(n_blocks)
    rcs = st.uniform(n_blocks) < rc_prob
    copies = []
    for i in range(n_blocks):
        src = T[ts[i]:ts[i] + lens[i]]
        cp = mutate(st.child("blk", i), src, float(ids[i]), indel_rate=indel_rate, gc=gc)
        if rcs[i]:
            cp = revcomp_codes(cp)
        copies.append(cp[: Q.size])
    qlens = np.array([c.size for c in copies], dtype=np.int64)
    qs = _place_disjoint(st.child("qpos"), qlens, Q.size)
    if qs is None:
        qs = np.array([int(st.integers(0, Q.size - L + 1, 1)[0]) for L in qlens])
    out = []
    for i, cp in enumerate(copies):
        Q[qs[i]:qs[i] + cp.size] = cp
        out.append(Block(int(ts[i]), int(lens[i]), int(qs[i]), int(cp.size), float(ids[i]),
                         bool(rcs[i])))
    return out


@dataclass
class Pair:
    """A synthetic target/query pair with the record of what was planted."""
    T: np.ndarray
    Q: np.ndarray
    blocks: list = field(default_factory=list)
    name: str = ""
    gc: float = 0.5

    @property
    def tlen(self) -> int:
        return int(self.T.size)

    @property
    def qlen(self) -> int:
        return int(self.Q.size)
