"""The device radix sort against numpy's stable sort: random 64-bit keys
ordered by a bit range, at sizes around the 4096-key tile and the ragged
tails, for 8-, 9- and 10-bit digit passes, with the key count on the host or
in device memory. Equal fields keep their input order (stability)."""
from __future__ import annotations

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_06811_gb300 as P
    ctx = P.Context(0)
    yield torch, ctx
    ctx.close()


def _keys(n, seed, lo, hi):
    st = synth.Stream(seed, "sort-keys")
    k = st.u64(n).astype(np.uint64)
    if n and hi - lo < 20:  # force many equal fields: stability is visible
        k &= ~np.uint64(((1 << (hi - lo)) - 1) << lo) | np.uint64(((1 << min(6, hi - lo)) - 1) << lo)
    return k


@pytest.mark.parametrize("n", [0, 1, 2, 4095, 4096, 4097, 100_003, 1_000_001])
@pytest.mark.parametrize("lo,hi", [(0, 8), (32, 57), (3, 31), (0, 64), (60, 64)])
@pytest.mark.parametrize("devn", [False, True])
def test_radix_sort_is_numpys_stable_sort(env, n, lo, hi, devn):
    torch, ctx = env
    k = _keys(n, n * 131 + lo, lo, hi)
    field = (k >> np.uint64(lo)) & np.uint64((1 << (hi - lo)) - 1)
    want = k[np.argsort(field, kind="stable")]
    t = torch.from_numpy(k.view(np.int64).copy()).cuda()
    ctx.test_radix_sort(t, lo, hi, device_count=devn)
    got = t.cpu().numpy().view(np.uint64)
    assert np.array_equal(got, want)
