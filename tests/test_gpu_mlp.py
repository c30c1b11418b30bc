"""The learned schedule on the GPU: the extension log the predictor trains on,
its forward/backward/Adam kernels against the float64 oracle MLP, FP16
inference, training on one seed of a generator and evaluation on another,
and the schedule's output identity with the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
import synth
from synth.workloads import concat_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def pkg(torch):
    import paper_2606_06811_gb300 as P
    return P


@pytest.fixture(scope="module")
def ctx(pkg):
    c = pkg.Context(0)
    yield c
    c.close()


def ext_records(pkg, ctx, T, Q, every, cap=1 << 20, **kw):
    from paper_2606_06811_gb300 import predictor
    recs, st = predictor.collect(ctx, T, Q, every, cap, pkg.default_params(input_codes=1, **kw))
    return recs, st


def rec_set(a) -> set:
    return set(map(tuple, np.asarray(a).tolist()))


@pytest.fixture(scope="module")
def tiny(pkg, ctx):
    p = synth.tiny_pair(1)
    ref = oracle.run(p.T, p.Q, keep_log=True)
    return p, ref


def test_extension_log_is_every_extension_of_the_oracle(pkg, ctx, tiny):
    p, ref = tiny
    want = {(int(e["strand"]), int(e["t"]), int(e["q"]), int(e["rscored"]), int(e["lscored"]))
            for e in ref.ext}
    for kw in ({}, {"lane_cap": 1}, {"walk_mode": pkg.WALK_TWO_LAUNCHES},
               {"walk_mode": pkg.WALK_PERSISTENT, "walk_schedule": pkg.SCHED_RANDOM,
                "walk_chunk": 4}):
        recs, st = ext_records(pkg, ctx, p.T, p.Q, 1, **kw)
        r = recs.cpu().numpy()
        assert st["ext_logged"] == ref.extended == r.shape[0], kw
        assert (r[:, 0] == 0).all()
        assert rec_set(r[:, 1:]) == want, kw


def test_sampled_log_does_not_depend_on_the_schedule(pkg, ctx, tiny):
    p, ref = tiny
    base = None
    P_ = pkg.WALK_PERSISTENT
    for kw in ({}, {"walk_mode": pkg.WALK_TWO_LAUNCHES, "lane_cap": 8},
               {"walk_mode": P_, "walk_schedule": pkg.SCHED_LARGEST_FIRST},
               {"walk_mode": P_, "walk_schedule": pkg.SCHED_RANDOM}):
        recs, st = ext_records(pkg, ctx, p.T, p.Q, 7, **kw)
        s = rec_set(recs.cpu().numpy())
        assert len(s) == recs.shape[0]
        if base is None:
            base = s
            assert 0.08 * ref.extended < len(s) < 0.2 * ref.extended
        assert s == base, kw


def test_extension_log_cap_counts_beyond_the_buffer(pkg, ctx, tiny):
    p, ref = tiny
    recs, st = ext_records(pkg, ctx, p.T, p.Q, 1, cap=100)
    assert recs.shape[0] == 100 and st["ext_logged"] == ref.extended


def test_batch_extension_log_per_pair(pkg, ctx):
    pairs = synth.batch_pairs(seed=8, n_pairs=12, len_lo=2000, len_hi=30_000)
    T, toff, Q, qoff = concat_batch(pairs)
    import torch
    cap = 1 << 20
    log = torch.zeros((cap, 6), dtype=torch.int32, device="cuda:0")
    prm = pkg.default_params(input_codes=1, ext_log_every=1, ext_log=log.data_ptr(),
                             ext_log_cap=cap)
    _, st = ctx.run_batch(T, toff, Q, qoff, prm)
    r = log[: st["ext_logged"]].cpu().numpy()
    for i, pr in enumerate(pairs):
        ref = oracle.run(pr.T, pr.Q, keep_log=True)
        want = {(int(e["strand"]), int(e["t"]), int(e["q"]), int(e["rscored"]),
                 int(e["lscored"])) for e in ref.ext}
        assert rec_set(r[r[:, 0] == i][:, 1:]) == want, i


@pytest.fixture(scope="module")
def grad_case(pkg, ctx, torch, tiny):
    p, _ = tiny
    recs, _ = ext_records(pkg, ctx, p.T, p.Q, 1)
    sel = recs[:: max(1, recs.shape[0] // 3000)].contiguous()
    data = ctx.mlp_data(p.T, [0, p.tlen], p.Q, [0, p.qlen], sel, input_codes=1)
    params = torch.zeros(pkg.mlp_param_count(), dtype=torch.float32, device="cuda:0")
    ctx.mlp_init(params, 123)
    rn = sel.cpu().numpy()
    rs = np.zeros(rn.shape[0], dtype=pkg.EXT_DTYPE)
    for j, name in enumerate(pkg.EXT_DTYPE.names):
        rs[name] = rn[:, j]
    X = omlp.feature_matrix([p.T], [p.Q], rs)
    y = omlp.targets_of(rs)
    return data, params, X, y


def _group_errors(a, b):
    A, B = omlp.unpack(a), omlp.unpack(b)
    return {k: float(np.linalg.norm(np.ravel(A[k] - B[k])) / max(np.linalg.norm(np.ravel(B[k])),
                                                                  1e-30)) for k in A}


def test_init_is_bounded_and_b3_is_three(pkg, ctx, grad_case):
    _, params, _, _ = grad_case
    P = omlp.unpack(params.double().cpu().numpy())
    assert P["b3"] == 3.0
    assert np.abs(P["W1"]).max() <= np.sqrt(6 / 64) and P["W1"].std() > 0.15
    assert np.abs(P["W2"]).max() <= np.sqrt(6 / 64)
    assert not P["b1"].any() and not P["b2"].any()


def test_loss_gradient_and_predictions_match_the_oracle(pkg, ctx, torch, grad_case):
    data, params, X, y = grad_case
    theta = params.double().cpu().numpy()
    grad = torch.zeros_like(params)
    preds = torch.zeros(data.n, dtype=torch.float32, device="cuda:0")
    loss = ctx.mlp_loss_grad(data, params, grad, preds)
    ref_pred, _ = omlp.forward(theta, X)
    assert np.abs(preds.cpu().numpy() - ref_pred).max() < 1e-4
    ref_loss = omlp.loss(theta, X, y)
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    errs = _group_errors(grad.double().cpu().numpy(), omlp.grad(theta, X, y))
    assert max(errs.values()) < 1e-4, errs
    # loss without a gradient buffer is the same number
    assert ctx.mlp_loss_grad(data, params) == pytest.approx(loss, rel=1e-6)


def test_fp16_inference_matches_the_oracle_with_half_weights(pkg, ctx, torch, grad_case):
    data, params, X, _ = grad_case
    model = torch.zeros(pkg.mlp_model_bytes(), dtype=torch.uint8, device="cuda:0")
    ctx.mlp_pack(params, model)
    preds = torch.zeros(data.n, dtype=torch.float32, device="cuda:0")
    ctx.mlp_predict(data, model, preds)
    ref = omlp.forward_fp16(params.double().cpu().numpy(), X)
    err = np.abs(preds.cpu().numpy() - ref)
    # float32 sums in another order can round a hidden unit to the next half
    assert err.max() < 2e-3 and np.median(err) < 1e-5, (err.max(), np.median(err))


def test_one_adam_step_matches_the_oracle(pkg, ctx, torch, grad_case):
    data, params0, X, y = grad_case
    params = params0.clone()
    lr = 1e-3
    ctx.mlp_train(data, params, epochs=1, batch=int(data.n), lr=lr, seed=5)
    theta0 = params0.double().cpu().numpy()
    g = omlp.grad(theta0, X, y)
    want, _, _ = omlp.adam_step(theta0, g, np.zeros_like(g), np.zeros_like(g), lr, 1)
    got = params.double().cpu().numpy()
    clear = np.abs(g) > 1e-5 * np.abs(g).max()
    assert np.abs(got - want)[clear].max() < 1e-6 * lr + 1e-7
    assert (np.abs(got - theta0) <= lr * (1 + 1e-5) + 1e-7).all()
    assert np.array_equal(got[g == 0], theta0[g == 0])


def test_bad_records_and_missing_model_are_rejected(pkg, ctx, torch, tiny):
    p, _ = tiny
    bad = torch.tensor([[1, 0, 10, 10, 5, 5]], dtype=torch.int32, device="cuda:0")
    with pytest.raises(pkg.SfeError):
        ctx.mlp_data(p.T, [0, p.tlen], p.Q, [0, p.qlen], bad, input_codes=1)
    with pytest.raises(pkg.SfeError):
        ctx.run(p.T, p.Q, pkg.default_params(input_codes=1, walk_mode=pkg.WALK_PERSISTENT,
                                             walk_schedule=pkg.SCHED_PREDICTED))
    with pytest.raises(pkg.SfeError):  # a schedule orders the persistent walk only
        ctx.run(p.T, p.Q, pkg.default_params(input_codes=1, walk_mode=pkg.WALK_TWO_LAUNCHES,
                                             walk_schedule=pkg.SCHED_RANDOM))


@pytest.fixture(scope="module")
def trained(pkg, ctx):
    """Trained on two pairs of the 10 Mb generator at 1/5 size (seeds 100, 101)."""
    from paper_2606_06811_gb300 import predictor
    runs = []
    for seed in (100, 101):
        pr = synth.plain_pair_10mb(seed, scale=0.2)
        recs, _ = ext_records(pkg, ctx, pr.T, pr.Q, 4, cap=1 << 22)
        runs.append((pr.T, pr.Q, recs))
    data = predictor.training_data(ctx, runs)
    return predictor.train(ctx, data, epochs=3, batch=4096, lr=2e-3, seed=7)


def test_training_beats_the_mean_on_a_fresh_seed(pkg, ctx, torch, trained):
    from paper_2606_06811_gb300 import predictor
    assert trained.history[-1] < trained.history[0]
    ev = synth.plain_pair_10mb(5, scale=0.2)
    recs, _ = ext_records(pkg, ctx, ev.T, ev.Q, 4, cap=1 << 22)
    data = predictor.training_data(ctx, [(ev.T, ev.Q, recs)])
    preds = torch.zeros(data.n, dtype=torch.float32, device="cuda:0")
    ctx.mlp_predict(data, trained.model, preds)
    r = recs.double().cpu().numpy()
    y = np.log1p(r[:, 4] + r[:, 5])
    mse = float(np.mean((preds.double().cpu().numpy() - y) ** 2))
    var = float(np.var(y))
    print(f"eval: n={y.size} mse={mse:.4f} var={var:.4f} r2={1 - mse / var:.3f} "
          f"history={trained.history}")
    assert mse < 0.5 * var  # R^2 above 0.5 (0.87 measured)


def test_predicted_schedule_keeps_the_oracle_output(pkg, ctx, trained):
    for seed, kw in ((1, {}), (2, {"walk_chunk": 4, "lane_cap": 16}), (3, {"walk_chunk": 200})):
        p = synth.tiny_pair(seed, length=80_000, n_blocks=20)
        ref = oracle.run(p.T, p.Q)
        prm = pkg.default_params(input_codes=1, walk_mode=pkg.WALK_PERSISTENT,
                                 walk_schedule=pkg.SCHED_PREDICTED,
                                 model=trained.model.data_ptr(), **kw)
        got, st = ctx.run(p.T, p.Q, prm)
        a = np.ascontiguousarray(got).view(np.int32).reshape(-1, 5)
        b = np.ascontiguousarray(ref.hsps).view(np.int32).reshape(-1, 5)
        assert np.array_equal(a, b)
        assert (st["hits"], st["extended"], st["cells"]) == (ref.hits, ref.extended, ref.cells)


def test_predicted_schedule_on_a_batch(pkg, ctx, trained):
    pairs = synth.batch_pairs(seed=9, n_pairs=16, len_lo=2000, len_hi=40_000)
    T, toff, Q, qoff = concat_batch(pairs)
    prm = pkg.default_params(input_codes=1, walk_mode=pkg.WALK_PERSISTENT,
                             walk_schedule=pkg.SCHED_PREDICTED, model=trained.model.data_ptr(),
                             walk_chunk=8)
    got, st = ctx.run_batch(T, toff, Q, qoff, prm)
    H = np.ascontiguousarray(got).view(np.int32).reshape(-1, 6)
    for i, pr in enumerate(pairs):
        ref = np.ascontiguousarray(oracle.run(pr.T, pr.Q).hsps).view(np.int32).reshape(-1, 5)
        assert np.array_equal(H[H[:, 0] == i][:, 1:], ref), i


def test_predictor_file_round_trip(pkg, ctx, torch, trained, tmp_path):
    from paper_2606_06811_gb300 import predictor
    f = tmp_path / "model.sfemlp"
    trained.save(str(f))
    back = predictor.Predictor.load(ctx, str(f))
    assert torch.equal(back.params, trained.params)
    assert torch.equal(back.model, trained.model)
