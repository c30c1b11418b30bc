"""Two contexts driven from two host threads at once.

A context belongs to one host thread; the library keeps no other mutable
state that calls share (the launch counter is per host thread, SM counts and
function attributes are per device). So two threads, each with its own
context, get the same HSPs and the same per-call statistics (including the
number of kernels a call launched) as one thread alone.
"""
from __future__ import annotations

import threading

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_06811_gb300 as P
    return P


KEYS = ("hits", "extended", "cells", "hsps", "launches", "tiles")


def test_two_threads_two_contexts(pkg):
    pairs = [synth.tiny_pair(seed=s, length=60_000, n_blocks=10) for s in (31, 32)]
    params = pkg.default_params(input_codes=1)
    alone = []
    with pkg.Context(0) as ctx:
        for p in pairs:
            h, st = ctx.run(p.T, p.Q, params)
            alone.append((h.copy(), {k: st[k] for k in KEYS}))
    for p, (h, _) in zip(pairs, alone):
        assert np.array_equal(h.view(oracle.HSP_DTYPE), oracle.run(p.T, p.Q).hsps)

    results = [[], []]
    errors = []
    start = threading.Barrier(2)

    def worker(k):
        try:
            with pkg.Context(0) as ctx:
                start.wait()
                for _ in range(6):
                    h, st = ctx.run(pairs[k].T, pairs[k].Q, params)
                    results[k].append((h.copy(), {x: st[x] for x in KEYS}))
        except Exception as e:  # surfaced below
            errors.append(e)

    th = [threading.Thread(target=worker, args=(k,)) for k in (0, 1)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    for k in (0, 1):
        assert len(results[k]) == 6
        for h, st in results[k]:
            assert np.array_equal(h, alone[k][0])
            assert st == alone[k][1]
