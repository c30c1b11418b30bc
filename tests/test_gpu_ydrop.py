"""The gapped Y-drop stage on the GPU (sfe_gapped_extend) against the oracle's
or_gapped: the same committed alignments (box and score), the same counts of
skipped, extended and shadow anchors and of DP cells, for the serial order
(batch 1), speculative batches and one batch of every anchor."""
from __future__ import annotations

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


@pytest.fixture(scope="module")
def ctx(pkg):
    c = pkg.Context(0)
    yield c
    c.close()


def _ok(got, st, ref):
    a = np.ascontiguousarray(got).view(np.int32).reshape(-1, 6)
    b = np.ascontiguousarray(ref.aligns).view(np.int32).reshape(-1, 6)
    assert a.shape == b.shape and np.array_equal(a, b), (a.shape, b.shape)
    r = ref.stats
    assert (st["skipped"], st["extended"], st["cells"], st["shadow"], st["shadow_cells"],
            st["committed"], st["batches"]) == (r["skipped"], r["extended"], r["cells"],
                                                r["shadow"], r["shadow_cells"], r["committed"],
                                                r["batches"]), (st, r)


def _run(pkg, ctx, T, Q, H, batch, **kw):
    okw = {k: v for k, v in kw.items() if k != "band"}
    # the library's batch 0 is one batch of every anchor (the oracle's 0 is serial)
    ref = oracle.gapped(T, Q, H, batch=batch if batch > 0 else max(1, H.size),
                        band=kw.get("band", oracle.BAND), **okw)
    names = {"thresh": "gapped_thresh", "Y": "ydrop"}
    pp = pkg.ydrop_params(input_codes=1, batch=batch,
                          **{names.get(k, k): v for k, v in kw.items()})
    got, st = ctx.gapped_extend(T, Q, H, pp)
    return got, st, ref


@pytest.mark.parametrize("batch", [1, 3, 64, 0])
def test_gapped_stage_on_the_tiny_pair(pkg, ctx, batch):
    p = synth.tiny_pair(1)
    H = oracle.run(p.T, p.Q).hsps
    got, st, ref = _run(pkg, ctx, p.T, p.Q, H, batch)
    _ok(got, st, ref)
    assert ref.aligns.size > 0


@pytest.mark.parametrize("kw", [
    dict(gap_open=60, gap_extend=15, Y=2000), dict(Y=910), dict(band=8), dict(band=1),
    dict(thresh=8000), dict(scores=np.array([[100, -50, -20, -60], [-50, 90, -60, -20],
                                             [-20, -60, 95, -50], [-60, -20, -50, 100]],
                                            np.int32)),
])
def test_gapped_stage_parameters(pkg, ctx, kw):
    p = synth.plain_pair_10mb(4, scale=0.02)
    H = oracle.run(p.T, p.Q).hsps
    got, st, ref = _run(pkg, ctx, p.T, p.Q, H, 16, **kw)
    _ok(got, st, ref)


def test_gapped_stage_on_anchors_at_the_sequence_ends(pkg, ctx):
    st = synth.Stream(40, "yend")
    T = synth.iid_bases(st.child("T"), 3000, 0.5)
    Q = T.copy()
    H = np.zeros(4, dtype=oracle.HSP_DTYPE)
    H[0] = (0, 0, 0, 0, 5000)            # anchor at (0, 0): no backward half
    H[1] = (0, 3000, 3000, 0, 4000)      # anchor at the end: no forward half
    H[2] = (1, 10, 20, 40, 3000)
    H[3] = (0, 1500, 1490, 30, 2000)     # off the main diagonal
    got, sts, ref = _run(pkg, ctx, T, Q, H, 2)
    _ok(got, sts, ref)


def test_gapped_stage_with_an_alignment_larger_than_its_grid(pkg, ctx):
    """A query that copies 80 kb of the target: one alignment box spans more
    grid cells (1024 x 1024 bases each) than the committed-box index lists per
    box, so it is kept on the index's short list; every later anchor inside
    it must still be skipped, and anchors outside it extended."""
    st = synth.Stream(41, "ybig")
    T = synth.iid_bases(st.child("T"), 90_000, 0.45)
    Q = np.concatenate([T[5_000:85_000], synth.iid_bases(st.child("Q"), 6_000, 0.45)])
    H = np.zeros(5, dtype=oracle.HSP_DTYPE)
    H[0] = (0, 40_000, 35_000, 2_000, 190_000)  # on the copied diagonal, highest score first
    H[1] = (0, 10_000, 5_000, 500, 50_000)      # inside the copy's box: skipped
    H[2] = (0, 70_000, 65_000, 800, 80_000)     # inside as well
    H[3] = (1, 1_000, 2_000, 40, 3_500)         # other strand: extended
    H[4] = (0, 88_000, 83_000, 40, 3_000)       # past the copy's end on the target
    for batch in (1, 2, 0):
        got, sts, ref = _run(pkg, ctx, T, Q, H, batch)
        _ok(got, sts, ref)
    assert ref.stats["skipped"] + ref.stats["shadow"] >= 2


def test_gapped_stage_device_buffers_and_small_capacity(pkg, ctx):
    import torch
    p = synth.tiny_pair(3, length=100_000, n_blocks=20)
    H = oracle.run(p.T, p.Q).hsps
    ref = oracle.gapped(p.T, p.Q, H, batch=H.size)
    dev = torch.device("cuda", 0)
    Td = torch.from_numpy(p.T.copy()).to(dev)
    Qd = torch.from_numpy(p.Q.copy()).to(dev)
    Hd = torch.from_numpy(np.ascontiguousarray(H).view(np.int32).copy()).to(dev)
    got, st = ctx.gapped_extend(Td, Qd, Hd, pkg.ydrop_params(input_codes=1), cap=1)
    _ok(got, st, ref)


def test_gapped_stage_rejects_bad_input(pkg, ctx):
    p = synth.tiny_pair(2, length=5000, n_blocks=2)
    H = np.zeros(1, dtype=oracle.HSP_DTYPE)
    H[0] = (0, 4999, 10, 100, 5000)  # anchor past the target's end
    with pytest.raises(pkg.SfeError):
        ctx.gapped_extend(p.T, p.Q, H, pkg.ydrop_params(input_codes=1))
    with pytest.raises(pkg.SfeError):
        ctx.gapped_extend(p.T, p.Q, H[:0], pkg.ydrop_params(input_codes=1, band=300))


def hit_anchors(T, Q, span=19):
    """Seed hits of both strands as zero-score records of one seed span, the
    anchors of the Y-drop-as-filter stage (anchor at the seed's middle, taken
    in (strand, tpos, qpos) order)."""
    rows = []
    for s, Qs in ((0, Q), (1, oracle.revcomp(Q))):
        t, q = oracle.seed_hits(T, Qs)
        r = np.zeros(t.size, dtype=oracle.HSP_DTYPE)
        r["strand"], r["tpos"], r["qpos"], r["len"] = s, t, q, span
        rows.append(r)
    return np.concatenate(rows)


@pytest.mark.parametrize("batch", [0, 4096])
def test_ydrop_as_the_filter(pkg, ctx, batch):
    """Darwin-WGA's idea (the paper's closing section): the 2-D Y-drop applied
    to the seed hits themselves instead of the ungapped X-drop filter."""
    p = synth.tiny_pair(2, length=100_000, n_blocks=20)
    A = hit_anchors(p.T, p.Q)
    got, st, ref = _run(pkg, ctx, p.T, p.Q, A, batch, Y=910)
    _ok(got, st, ref)
    assert ref.stats["skipped"] + ref.stats["shadow"] > 0 and ref.aligns.size >= 15
