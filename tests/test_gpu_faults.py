"""Error and recovery paths driven on the GPU without faulting it: a bounded
device wait that runs out (a hand-off queue slot nobody publishes), which the
follow-up launch absorbs so the call still returns the exact answer, and an
allocation that fails (injected on the host), which returns its error code
with the context usable for the next call."""
from __future__ import annotations

import time

import numpy as np
import pytest

import oracle
import synth
from synth.workloads import concat_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_06811_gb300 as P
    return P


def same(got, ref):
    a = np.ascontiguousarray(got).view(np.int32).reshape(-1, 5)
    b = np.ascontiguousarray(ref.hsps).view(np.int32).reshape(-1, 5)
    return a.shape == b.shape and np.array_equal(a, b)


def test_unanswered_queue_wait_is_left_to_the_follow_up_launch(pkg):
    """A hand-off entry that is never published (as if its producer's CTA could
    not become resident): the waiting warp gives up after wait_limit polls,
    the follow-up launch walks every published entry nobody finished, and the
    call returns the oracle's answer."""
    p = synth.tiny_pair(4, length=60_000, n_blocks=15)
    ref = oracle.run(p.T, p.Q)
    with pkg.Context(0) as ctx:
        late = pkg.default_params(input_codes=1, walk_mode=pkg.WALK_PERSISTENT, lane_cap=16,
                                  wait_limit=1 << 12,
                                  test_hooks=pkg.sfe.TEST_UNPUBLISHED_QUEUE_ENTRY)
        t0 = time.perf_counter()
        got, st = ctx.run(p.T, p.Q, late)
        assert time.perf_counter() - t0 < 30
        assert same(got, ref)
        assert (st["hits"], st["extended"], st["cells"]) == (ref.hits, ref.extended, ref.cells)
        assert st["deferred_tasks"] >= 1 and st["warp_tasks"] > 0
        got, st = ctx.run(p.T, p.Q, pkg.default_params(input_codes=1,
                                                       walk_mode=pkg.WALK_PERSISTENT,
                                                       lane_cap=16))
        assert same(got, ref) and st["deferred_tasks"] == 0


def test_unanswered_queue_wait_in_a_batch(pkg):
    pairs = synth.batch_pairs(seed=14, n_pairs=16, len_lo=2000, len_hi=20_000)
    T, toff, Q, qoff = concat_batch(pairs)
    with pkg.Context(0) as ctx:
        late = pkg.default_params(input_codes=1, walk_mode=pkg.WALK_PERSISTENT, lane_cap=16,
                                  wait_limit=1 << 12,
                                  test_hooks=pkg.sfe.TEST_UNPUBLISHED_QUEUE_ENTRY)
        h1, st1 = ctx.run_batch(T, toff, Q, qoff, late)
        h2, st2 = ctx.run_batch(T, toff, Q, qoff, pkg.default_params(input_codes=1,
                                                                      lane_cap=16))
        assert h1.shape[0] > 0 and np.array_equal(h1, h2)
        assert st1["cells"] == st2["cells"] and st1["deferred_tasks"] >= 1


def test_injected_allocation_failure(pkg):
    p = synth.tiny_pair(5, length=40_000, n_blocks=10)
    ref = oracle.run(p.T, p.Q)
    with pkg.Context(0) as ctx:
        ctx.fail_next_allocs(1)
        with pytest.raises(pkg.SfeError) as e:
            ctx.run(p.T, p.Q, pkg.default_params(input_codes=1))
        assert e.value.code == pkg.sfe.ENOMEM
        got, _ = ctx.run(p.T, p.Q, pkg.default_params(input_codes=1))
        assert same(got, ref)
        ctx.fail_next_allocs(3)  # a batch fails at its third allocation
        pairs = synth.batch_pairs(seed=15, n_pairs=8, len_lo=2000, len_hi=10_000)
        T, toff, Q, qoff = concat_batch(pairs)
        with pytest.raises(pkg.SfeError) as e:
            ctx.run_batch(T, toff, Q, qoff, pkg.default_params(input_codes=1))
        assert e.value.code == pkg.sfe.ENOMEM
        ctx.fail_next_allocs(0)
        h, _ = ctx.run_batch(T, toff, Q, qoff, pkg.default_params(input_codes=1))
        assert h.shape[0] >= 0
