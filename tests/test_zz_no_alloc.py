"""The allocation-free entry point, sfe_ungapped_xdrop_static.

It serves callers that cannot allocate device memory (code inside another
framework's memory pool or under a hard budget, plugins whose host owns all
device allocations, latency-critical paths). Its scratch is a fixed array in
the library, so it must give exactly what sfe_ungapped_xdrop gives, call after
call, with the array reused in between. This file is collected last so that a
run stopping at the first failure has run every other test first.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

import oracle
import synth
from tests import bruteforce as bf

pytestmark = pytest.mark.gpu

ELIMIT = -6


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_06811_gb300 as P
    L = P.lib()
    fn = L.sfe_ungapped_xdrop_static
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    fn.argtypes = [vp, i64, vp, i64, C.c_char_p, i32, vp, i64, C.POINTER(C.c_int32 * 16), i32, i32,
                   vp, i64, C.POINTER(i64), C.POINTER(P.Stats), vp]
    fn.restype = C.c_int
    ctx = P.Context(0)
    yield torch, P, fn, ctx
    ctx.close()


def _case(seed, n, m, nblocks):
    st = synth.Stream(seed, "static")
    T = synth.iid_bases(st.child("T"), n, 0.5)
    Q = synth.iid_bases(st.child("Q"), m, 0.5)
    synth.plant_blocks(st.child("b"), T, Q, nblocks, 300, 2000, 0.85, 0.97, 0.5, 0.01, 0.5)
    return T, Q


def _hits(T, Q, seed):
    recs = []
    for s, Qs in ((0, Q), (1, bf.revcomp(Q))):
        t, q = oracle.seed_hits(T, Qs)
        recs.append(np.stack([np.full(t.size, s), t, q], 1))
    H = np.concatenate(recs).astype(np.int32)
    order = synth.Stream(seed, "order").integers(0, 1 << 30, H.shape[0]).argsort(kind="stable")
    return np.ascontiguousarray(H[order])


def _static(env, T, Q, H, cap):
    torch, P, fn, _ = env
    dev = torch.device("cuda", 0)
    Td = torch.from_numpy(T.copy()).to(dev)
    Qd = torch.from_numpy(Q.copy()).to(dev)
    Hd = torch.from_numpy(H).to(dev)
    out = torch.full((max(cap, 1), 5), -7, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    nh = C.c_int64(0)
    st = P.Stats()
    sc = (C.c_int32 * 16)(*[int(x) for x in oracle.HOXD70.reshape(16)])
    code = fn(Td.data_ptr(), T.size, Qd.data_ptr(), Q.size, None, 1, Hd.data_ptr(), H.shape[0],
              C.byref(sc), 910, 3000, out.data_ptr(), cap, C.byref(nh), C.byref(st), None)
    return code, out[: nh.value].cpu().numpy(), st.as_dict()


def _existing(env, T, Q, H):
    torch, P, fn, ctx = env
    ix = ctx.index_build(T, P.default_params(input_codes=1))
    hsps, st = ctx.ungapped_xdrop(ix, Q, H, oracle.HOXD70, 910, 3000)
    ix.close()
    return np.ascontiguousarray(hsps).view(np.int32).reshape(-1, 5), st


def test_matches_the_allocating_entry_point_on_two_calls_in_a_row(env):
    cases = [_case(41, 60_000, 50_000, 12), _case(42, 30_000, 70_000, 8)]
    for k, (T, Q) in enumerate(cases):
        H = _hits(T, Q, k)
        ref, rst = _existing(env, T, Q, H)
        code, got, st = _static(env, T, Q, H, cap=4096)
        assert code == 0
        assert got.shape == ref.shape and np.array_equal(got, ref)
        assert (st["hits"], st["extended"], st["cells"], st["hsps"]) == \
            (rst["hits"], rst["extended"], rst["cells"], rst["hsps"])
        assert ref.shape[0] > 0


def test_reports_the_needed_capacity(env):
    T, Q = _case(43, 40_000, 40_000, 10)
    H = _hits(T, Q, 3)
    ref, _ = _existing(env, T, Q, H)
    code, _, st = _static(env, T, Q, H, cap=2)
    assert code == -5 and st["hsps"] == ref.shape[0]
    code, got, _ = _static(env, T, Q, H, cap=ref.shape[0])
    assert code == 0 and np.array_equal(got, ref)


def test_rejects_sizes_beyond_the_fixed_scratch(env):
    torch, P, fn, _ = env
    dev = torch.device("cuda", 0)
    big = torch.zeros((1 << 20) + 1, dtype=torch.uint8, device=dev)
    small = torch.zeros(1000, dtype=torch.uint8, device=dev)
    hits = torch.zeros(((1 << 17) + 1, 3), dtype=torch.int32, device=dev)
    out = torch.zeros((16, 5), dtype=torch.int32, device=dev)
    nh = C.c_int64(0)
    sc = (C.c_int32 * 16)(*[int(x) for x in oracle.HOXD70.reshape(16)])
    args = lambda t, tl, q, ql, h, nhits: (t.data_ptr(), tl, q.data_ptr(), ql, None, 1, h.data_ptr(),
                                            nhits, C.byref(sc), 910, 3000, out.data_ptr(), 16,
                                            C.byref(nh), None, None)
    assert fn(*args(big, big.numel(), small, small.numel(), hits, 0)) == ELIMIT
    assert fn(*args(small, small.numel(), big, big.numel(), hits, 0)) == ELIMIT
    assert fn(*args(small, small.numel(), small, small.numel(), hits, hits.shape[0])) == ELIMIT


def _raw(env, T, Q, H, cap, scores=None, stream=None, out_none=False):
    """One call with explicit scores and stream; returns (code, HSPs, needed count)."""
    torch, P, fn, _ = env
    dev = torch.device("cuda", 0)
    Td = torch.from_numpy(T.copy()).to(dev)
    Qd = torch.from_numpy(Q.copy()).to(dev)
    Hd = torch.from_numpy(H).to(dev)
    out = torch.full((max(cap, 1), 5), -7, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    nh = C.c_int64(-1)
    M = oracle.HOXD70.reshape(16) if scores is None else np.asarray(scores).reshape(16)
    sc = (C.c_int32 * 16)(*[int(x) for x in M])
    code = fn(Td.data_ptr(), T.size, Qd.data_ptr(), Q.size, None, 1, Hd.data_ptr(), H.shape[0],
              C.byref(sc), 910, 3000, None if out_none else out.data_ptr(), cap, C.byref(nh),
              None, stream)
    return code, out[: max(0, min(nh.value, cap))].cpu().numpy(), nh.value


def test_rejects_scores_outside_the_packed_window_range(env):
    """A score beyond 2^20 would overflow the walk's 64 x score window sums;
    the call refuses it before any GPU work, like every other entry point."""
    T, Q = _case(44, 20_000, 20_000, 4)
    H = _hits(T, Q, 4)
    for bad in ((1 << 20) + 1, -(1 << 20) - 1):
        M = oracle.HOXD70.reshape(16).copy()
        M[5] = bad
        code, _, _ = _raw(env, T, Q, H, cap=1024, scores=M)
        assert code == -1
    M = oracle.HOXD70.reshape(16).copy()
    M[5] = 1 << 20  # the bound itself is accepted
    code, _, _ = _raw(env, T, Q, H, cap=1 << 16, scores=M)
    assert code == 0


def test_a_hit_outside_the_sequences_is_rejected_and_the_next_call_is_exact(env):
    T, Q = _case(45, 30_000, 30_000, 6)
    H = _hits(T, Q, 5)
    bad = H.copy()
    bad[len(bad) // 2, 1] = T.size - 10  # the seed span would leave the target
    code, _, _ = _raw(env, T, Q, bad, cap=4096)
    assert code == -1
    ref, _ = _existing(env, T, Q, H)
    code, got, n = _raw(env, T, Q, H, cap=4096)
    assert code == 0 and n == ref.shape[0] and np.array_equal(got, ref)


def test_zero_capacity_without_a_buffer_reports_the_count(env):
    T, Q = _case(46, 30_000, 30_000, 6)
    H = _hits(T, Q, 6)
    ref, _ = _existing(env, T, Q, H)
    code, _, n = _raw(env, T, Q, H, cap=0, out_none=True)
    assert ref.shape[0] > 0 and code == -5 and n == ref.shape[0]


def test_runs_on_a_caller_stream(env):
    torch = env[0]
    T, Q = _case(47, 40_000, 30_000, 8)
    H = _hits(T, Q, 7)
    ref, _ = _existing(env, T, Q, H)
    s = torch.cuda.Stream(device=torch.device("cuda", 0))
    code, got, n = _raw(env, T, Q, H, cap=4096, stream=C.c_void_p(s.cuda_stream))
    assert code == 0 and n == ref.shape[0] and np.array_equal(got, ref)
