"""CPU oracle for the seed-hit + diagonal-skip + ungapped X-drop hot path.

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
CPU-baseline leg (and its `--impl reference` arm) may import this package. It
is the plain serial definition that the CUDA library is checked against bit
for bit; it shares no code with that library and imports nothing from it.

The arithmetic lives in `sfe_oracle.c` (plain C). This module only marshals
numpy arrays through ctypes. Every definition it relies on is stated in the
header comment of `sfe_oracle.c`; the MLP reference for learned binning is in
`mlp.py`.
"""
from __future__ import annotations

import contextlib
import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import build as _build

DEFAULT_PATTERN = "1110100110010101111"  # 12 of 19, Section 7

# HOXD70 (Chiaromonte, Yap and Miller 2002), rows = target base, columns =
# query base, order A C G T; the substitution scores of the paper's LASTZ
# pipeline (Section 2). Recalled from the literature; pinned in the tests by
# its published symmetries, not by a printed copy.
HOXD70 = np.array([
    [91, -114, -31, -123],
    [-114, 100, -125, -31],
    [-31, -125, 100, -114],
    [-123, -31, -114, 91],
], dtype=np.int32)
XDROP = 910       # LASTZ default: 10 x the A:A score
HSP_THRESH = 3000  # LASTZ default ungapped threshold

SKIP_PASSING_ONLY = 1

HSP_DTYPE = np.dtype([("strand", "<i4"), ("tpos", "<i4"), ("qpos", "<i4"), ("len", "<i4"),
                      ("score", "<i4")])
EXT_DTYPE = np.dtype({
    "names": ["strand", "t", "q", "lext", "rext", "lscored", "rscored", "score"],
    "formats": ["<i4"] * 7 + ["<i8"],
    "offsets": [0, 4, 8, 12, 16, 20, 24, 32],
    "itemsize": 40,
})


class _Half(C.Structure):
    _fields_ = [("best", C.c_int64), ("bi", C.c_int32), ("bj", C.c_int32), ("cells", C.c_int64)]


class _GStats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("anchors", "skipped", "extended", "cells", "shadow",
                                          "shadow_cells", "committed", "batches")]


GALIGN_DTYPE = np.dtype([("strand", "<i4"), ("tstart", "<i4"), ("tend", "<i4"),
                         ("qstart", "<i4"), ("qend", "<i4"), ("score", "<i4")])
# LASTZ's default gapped scoring with HOXD70: gap open 400, extend 30 (a gap of
# L bases costs 400 + 30 L), Y = 400 + 300 x 30, gapped threshold 3000.
GAP_OPEN, GAP_EXTEND, YDROP, GAPPED_THRESH, BAND = 400, 30, 9400, 3000, 256


class _Stats(C.Structure):
    _fields_ = [("hits", C.c_int64), ("extended", C.c_int64), ("cells", C.c_int64),
                ("hsps", C.c_int64)]


class _Ext(C.Structure):
    _fields_ = [("strand", C.c_int32), ("t", C.c_int32), ("q", C.c_int32),
                ("lext", C.c_int32), ("rext", C.c_int32), ("lscored", C.c_int32),
                ("rscored", C.c_int32), ("_pad", C.c_int32), ("score", C.c_int64)]


_lib = None


def _bind(path: str):
    L = C.CDLL(path)
    u8p = C.POINTER(C.c_uint8)
    i32p = C.POINTER(C.c_int32)
    i64p = C.POINTER(C.c_int64)
    L.or_encode.argtypes = [u8p, C.c_int64, u8p]
    L.or_encode.restype = C.c_int
    L.or_revcomp.argtypes = [u8p, C.c_int64, u8p]
    L.or_revcomp.restype = None
    L.or_run.argtypes = [u8p, C.c_int64, u8p, C.c_int64, C.c_char_p, C.c_int, C.c_int, C.c_int,
                         i32p, C.c_int32, C.c_int32, C.c_int, C.c_int, C.POINTER(C.c_int)]
    L.or_run.restype = C.c_void_p
    L.or_run_par.argtypes = [u8p, C.c_int64, u8p, C.c_int64, C.c_char_p, C.c_int, C.c_int,
                             C.c_int, i32p, C.c_int32, C.c_int32, C.c_int, C.c_int64, C.c_int,
                             C.POINTER(C.c_int)]
    L.or_run_par.restype = C.c_void_p
    L.or_run_diagonal.argtypes = [u8p, C.c_int64, u8p, C.c_int64, C.c_int, C.c_int64,
                                  C.c_int64, C.c_char_p, C.c_int, C.c_int, i32p, C.c_int32,
                                  C.c_int32, C.c_int, C.c_int, C.POINTER(C.c_int)]
    L.or_run_diagonal.restype = C.c_void_p
    L.or_seed_hits.argtypes = [u8p, C.c_int64, u8p, C.c_int64, C.c_char_p, C.c_int, C.c_int,
                               i64p, i64p, C.c_int64, C.POINTER(C.c_int)]
    L.or_seed_hits.restype = C.c_int64
    L.or_xdrop.argtypes = [u8p, C.c_int64, u8p, C.c_int64, C.c_int64, C.c_int64, C.c_int,
                           i32p, C.c_int32, C.POINTER(_Ext)]
    L.or_xdrop.restype = None
    L.or_ydrop_half.argtypes = [u8p, C.c_int64, C.c_int64, u8p, C.c_int64, C.c_int64, C.c_int,
                                i32p, C.c_int32, C.c_int32, C.c_int32, C.c_int,
                                C.POINTER(_Half)]
    L.or_ydrop_half.restype = None
    L.or_gapped.argtypes = [u8p, C.c_int64, u8p, C.c_int64, C.c_void_p, C.c_int64, i32p,
                            C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int, C.c_int64,
                            C.c_void_p, C.c_int64, C.POINTER(_GStats)]
    L.or_gapped.restype = C.c_int64
    L.or_result_count.argtypes = [C.c_void_p]
    L.or_result_count.restype = C.c_int64
    L.or_result_ext_count.argtypes = [C.c_void_p]
    L.or_result_ext_count.restype = C.c_int64
    L.or_result_stats.argtypes = [C.c_void_p, C.POINTER(_Stats)]
    L.or_result_stats.restype = None
    L.or_result_copy.argtypes = [C.c_void_p, C.c_void_p]
    L.or_result_copy.restype = None
    L.or_result_copy_ext.argtypes = [C.c_void_p, C.c_void_p]
    L.or_result_copy_ext.restype = None
    L.or_result_free.argtypes = [C.c_void_p]
    L.or_result_free.restype = None
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = _bind(_build.build())
    return _lib


# When set, run() computes through the multi-threaded form (or_run_par) with
# these (qtile, threads); the pin battery runs in both forms.
_parallel: tuple | None = None


@contextlib.contextmanager
def use_parallel(qtile: int = 0, threads: int = 0):
    """Route run() through the multi-threaded form of the oracle."""
    global _parallel
    saved = _parallel
    _parallel = (int(qtile), int(threads))
    try:
        yield
    finally:
        _parallel = saved


@contextlib.contextmanager
def use_library(path: str):
    """Temporarily route every oracle call through another build of sfe_oracle.c.

    The mutation tests use this to check that the pins reject oracles with a
    planted mistake.
    """
    global _lib
    saved = lib()
    _lib = _bind(path)
    try:
        yield
    finally:
        _lib = saved


def _u8(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a if a.size else np.zeros(1, np.uint8)[:0]


def _ptr(a, t):
    if a.size == 0:
        a = np.zeros(1, dtype=a.dtype)
        _keep.append(a)
    return a.ctypes.data_as(C.POINTER(t))


_keep: list = []


def _scores(scores) -> np.ndarray:
    m = np.ascontiguousarray(np.asarray(scores, dtype=np.int32).reshape(16))
    return m


def encode(ascii_bytes: bytes) -> np.ndarray:
    a = np.frombuffer(bytes(ascii_bytes), dtype=np.uint8).copy()
    out = np.zeros(max(1, a.size), dtype=np.uint8)
    if lib().or_encode(_ptr(a, C.c_uint8), a.size, _ptr(out, C.c_uint8)) != 0:
        raise ValueError("symbol outside ACGTacgt")
    return out[: a.size]


def revcomp(Q) -> np.ndarray:
    Q = _u8(Q)
    out = np.zeros(max(1, Q.size), dtype=np.uint8)
    lib().or_revcomp(_ptr(Q, C.c_uint8), Q.size, _ptr(out, C.c_uint8))
    return out[: Q.size]


@dataclass
class Result:
    hsps: np.ndarray          # HSP_DTYPE, sorted by (strand, tpos, qpos, len, score)
    hits: int
    extended: int
    cells: int
    ext: np.ndarray | None    # EXT_DTYPE log of every extension (processing order)

    @property
    def stats(self) -> dict:
        return {"hits": self.hits, "extended": self.extended, "cells": self.cells,
                "hsps": int(self.hsps.size)}


def _collect(h, err, keep_log) -> Result:
    if not h:
        raise RuntimeError(f"oracle error {err.value}")
    L = lib()
    try:
        n = L.or_result_count(h)
        out = np.zeros(n, dtype=HSP_DTYPE)
        if n:
            L.or_result_copy(h, out.ctypes.data)
        st = _Stats()
        L.or_result_stats(h, C.byref(st))
        ext = None
        if keep_log:
            m = L.or_result_ext_count(h)
            ext = np.zeros(m, dtype=EXT_DTYPE)
            if m:
                L.or_result_copy_ext(h, ext.ctypes.data)
        return Result(out, st.hits, st.extended, st.cells, ext)
    finally:
        L.or_result_free(h)


def run(T, Q, pattern: str = DEFAULT_PATTERN, transition: bool = True, strands: int = 3,
        scores=HOXD70, X: int = XDROP, thresh: int = HSP_THRESH, flags: int = 0,
        keep_log: bool = False, step: int = 1) -> Result:
    """The filter stage on one pair: hits -> per-diagonal skip -> X-drop -> sorted HSPs.
    step: index stride (only target positions t % step == 0 are seeds)."""
    if _parallel is not None and not keep_log:
        return run_par(T, Q, pattern, transition, strands, scores, X, thresh, flags,
                       qtile=_parallel[0], threads=_parallel[1], step=step)
    T, Q = _u8(T), _u8(Q)
    M = _scores(scores)
    err = C.c_int(0)
    h = lib().or_run(_ptr(T, C.c_uint8), T.size, _ptr(Q, C.c_uint8), Q.size, pattern.encode(),
                     int(step), int(transition), int(strands), _ptr(M, C.c_int32), int(X),
                     int(thresh), int(flags), int(keep_log), C.byref(err))
    return _collect(h, err, keep_log)


def run_par(T, Q, pattern: str = DEFAULT_PATTERN, transition: bool = True, strands: int = 3,
            scores=HOXD70, X: int = XDROP, thresh: int = HSP_THRESH, flags: int = 0,
            qtile: int = 0, threads: int = 0, step: int = 1) -> Result:
    """run() on several threads (or_run_par): query tiles of qtile positions
    (0: one tile), the skip state carried across tiles, blocks of diagonals
    walked in parallel; threads 0 = every core OpenMP offers. Same result as
    run(), without the extension log."""
    T, Q = _u8(T), _u8(Q)
    M = _scores(scores)
    err = C.c_int(0)
    h = lib().or_run_par(_ptr(T, C.c_uint8), T.size, _ptr(Q, C.c_uint8), Q.size,
                         pattern.encode(), int(step), int(transition), int(strands),
                         _ptr(M, C.c_int32),
                         int(X), int(thresh), int(flags), int(qtile), int(threads),
                         C.byref(err))
    return _collect(h, err, False)


def host_cores() -> int:
    """Cores this process may run on (the oracle's default thread count)."""
    import os
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def run_diagonal(T, Qs, strand: int, d: int, E0: int = -(1 << 62), pattern: str = DEFAULT_PATTERN,
                 transition: bool = True, scores=HOXD70, X: int = XDROP,
                 thresh: int = HSP_THRESH, flags: int = 0, keep_log: bool = False,
                 step: int = 1) -> Result:
    """The walk restricted to diagonal d = t - q of Qs (Qs already strand-oriented)."""
    T, Qs = _u8(T), _u8(Qs)
    M = _scores(scores)
    err = C.c_int(0)
    h = lib().or_run_diagonal(_ptr(T, C.c_uint8), T.size, _ptr(Qs, C.c_uint8), Qs.size,
                              int(strand), int(d), int(E0), pattern.encode(), int(step),
                              int(transition),
                              _ptr(M, C.c_int32), int(X), int(thresh), int(flags),
                              int(keep_log), C.byref(err))
    return _collect(h, err, keep_log)


def seed_hits(T, Qs, pattern: str = DEFAULT_PATTERN, transition: bool = True, step: int = 1):
    """All hits (t, q) of T against the strand-oriented Qs, sorted by (t - q, t)."""
    T, Qs = _u8(T), _u8(Qs)
    err = C.c_int(0)
    L = lib()
    empty = np.zeros(1, dtype=np.int64)
    n = L.or_seed_hits(_ptr(T, C.c_uint8), T.size, _ptr(Qs, C.c_uint8), Qs.size,
                       pattern.encode(), int(step), int(transition), _ptr(empty, C.c_int64),
                       _ptr(empty, C.c_int64), 0, C.byref(err))
    if n < 0:
        raise RuntimeError(f"oracle error {err.value}")
    t = np.zeros(max(n, 1), dtype=np.int64)
    q = np.zeros(max(n, 1), dtype=np.int64)
    L.or_seed_hits(_ptr(T, C.c_uint8), T.size, _ptr(Qs, C.c_uint8), Qs.size, pattern.encode(),
                   int(step), int(transition), _ptr(t, C.c_int64), _ptr(q, C.c_int64), n,
                   C.byref(err))
    return t[:n], q[:n]


def xdrop(T, Qs, t: int, q: int, span: int = 19, scores=HOXD70, X: int = XDROP) -> dict:
    """One ungapped X-drop extension of the hit (t, q)."""
    T, Qs = _u8(T), _u8(Qs)
    M = _scores(scores)
    e = _Ext()
    lib().or_xdrop(_ptr(T, C.c_uint8), T.size, _ptr(Qs, C.c_uint8), Qs.size, int(t), int(q),
                   int(span), _ptr(M, C.c_int32), int(X), C.byref(e))
    return {"lext": e.lext, "rext": e.rext, "lscored": e.lscored, "rscored": e.rscored,
            "score": e.score, "tpos": t - e.lext, "qpos": q - e.lext,
            "len": span + e.lext + e.rext, "end": t + span + e.rext,
            "cells": span + e.lscored + e.rscored}


def ydrop_half(T, t0: int, Qs, q0: int, direction: int, scores=HOXD70, gap_open: int = GAP_OPEN,
               gap_extend: int = GAP_EXTEND, Y: int = YDROP, band: int = BAND) -> dict:
    """One half of a gapped Y-drop extension from anchor (t0, q0): forward
    (direction +1) over T[t0:], Qs[q0:], backward (-1) over T[:t0], Qs[:q0] reversed.
    Returns best, (bi, bj) (bases consumed at the best cell) and cells."""
    T, Qs = _u8(T), _u8(Qs)
    M = _scores(scores)
    h = _Half()
    TL = T.size - t0 if direction > 0 else t0
    QL = Qs.size - q0 if direction > 0 else q0
    lib().or_ydrop_half(_ptr(T, C.c_uint8), int(t0), int(TL), _ptr(Qs, C.c_uint8), int(q0),
                        int(QL), int(direction), _ptr(M, C.c_int32), int(gap_open),
                        int(gap_extend), int(Y), int(band), C.byref(h))
    return {"best": h.best, "bi": h.bi, "bj": h.bj, "cells": h.cells}


@dataclass
class Gapped:
    aligns: np.ndarray   # GALIGN_DTYPE, sorted by (strand, tstart, qstart, tend, qend, score)
    stats: dict


def gapped(T, Q, hsps, scores=HOXD70, gap_open: int = GAP_OPEN, gap_extend: int = GAP_EXTEND,
           Y: int = YDROP, thresh: int = GAPPED_THRESH, band: int = BAND,
           batch: int = 0) -> Gapped:
    """The gapped stage over a pair's HSPs (HSP_DTYPE): anchors at the HSPs'
    midpoints in decreasing score, skipped when inside a committed alignment,
    Y-drop extended, committed at >= thresh. batch 0: Algorithm 1 (serial);
    batch K: Algorithm 3 (speculative batches of K, serial commit)."""
    T, Q = _u8(T), _u8(Q)
    H = np.ascontiguousarray(np.asarray(hsps).view(HSP_DTYPE))
    M = _scores(scores)
    st = _GStats()
    L = lib()
    out = np.zeros(max(1, H.size), dtype=GALIGN_DTYPE)
    hp = H.ctypes.data if H.size else None
    n = L.or_gapped(_ptr(T, C.c_uint8), T.size, _ptr(Q, C.c_uint8), Q.size, hp, H.size,
                    _ptr(M, C.c_int32), int(gap_open), int(gap_extend), int(Y), int(thresh),
                    int(band), int(batch), out.ctypes.data, out.size, C.byref(st))
    if n < 0:
        raise RuntimeError("oracle gapped stage failed")
    return Gapped(out[:n].copy(), {k: int(getattr(st, k)) for k, _ in _GStats._fields_})
