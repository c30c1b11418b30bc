"""Pins of the work-predictor oracle (oracle/mlp.py) against facts that do not
come from the oracle itself: the inverse of the one-hot encoding, networks
whose output is a count computed by string methods, central finite
differences, Adam's closed-form first step and IEEE half rounding."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import mlp
import synth


def _seq(n, seed):
    return synth.Stream(seed, "mlp-seq").integers(0, 4, n).astype(np.uint8)


def _columns(T, Qs, t0, q0):
    """Substitution classes of the 32 columns from (t0, q0), -1 where a column
    leaves a sequence: padded slices of both sequences, XOR of the codes."""
    Tp = np.concatenate([np.full(80, -1), np.asarray(T, dtype=np.int64), np.full(80, -1)])
    Qp = np.concatenate([np.full(80, -1), np.asarray(Qs, dtype=np.int64), np.full(80, -1)])
    a, b = Tp[t0 + 80: t0 + 112], Qp[q0 + 80: q0 + 112]
    return np.where((a >= 0) & (b >= 0), a ^ b, -1)


def _decode(x):
    """Column classes of a feature vector: the one-hot inverted (-1 for an empty column)."""
    H = x.reshape(64, 4)
    assert set(np.unique(H)) <= {0.0, 1.0}
    assert (H.sum(axis=1) <= 1).all()
    return np.where(H.sum(axis=1) == 1, H.argmax(axis=1), -1)


def test_substitution_classes_follow_the_biology():
    """XOR of the codes A=0, C=1, G=2, T=3: 0 exactly for a match, 2 exactly for
    the transitions A<->G and C<->T, 1 or 3 for the transversions."""
    code = {"A": 0, "C": 1, "G": 2, "T": 3}
    transitions = {frozenset("AG"), frozenset("CT")}
    for x in "ACGT":
        for y in "ACGT":
            T = np.full(100, code[x], np.uint8)
            Q = np.full(100, code[y], np.uint8)
            cls = set(_decode(mlp.features(T, Q, 50, 50))) - {-1}
            assert len(cls) == 1
            c = cls.pop()
            assert (c == 0) == (x == y)
            assert (c == 2) == (frozenset((x, y)) in transitions)


@pytest.mark.parametrize("t,q", [(0, 0), (3, 50), (32, 32), (100, 90), (280, 270), (299, 0),
                                 (150, 298), (-3, 5), (60, 13)])
def test_features_invert_to_the_flank_columns(t, q):
    T, Qs = _seq(300, 1), _seq(300, 2)
    cols = _decode(mlp.features(T, Qs, t, q))
    assert np.array_equal(cols[:32], _columns(T, Qs, t - 32, q - 32))
    assert np.array_equal(cols[32:], _columns(T, Qs, t + 19, q + 19))
    cols = _decode(mlp.features(T, Qs, t, q, span=11))
    assert np.array_equal(cols[32:], _columns(T, Qs, t + 11, q + 11))


def test_feature_matrix_reads_the_reverse_complement_on_strand_1():
    T, Q = _seq(200, 3), _seq(150, 4)
    rc = np.array([3 - b for b in Q[::-1]])
    recs = np.zeros(2, dtype=[("pair", "<i4"), ("strand", "<i4"), ("t", "<i4"), ("q", "<i4"),
                              ("right", "<i4"), ("left", "<i4")])
    recs[0] = (0, 0, 40, 60, 0, 0)
    recs[1] = (0, 1, 40, 60, 0, 0)
    X = mlp.feature_matrix([T], [Q], recs)
    assert np.array_equal(_decode(X[0]), np.concatenate([_columns(T, Q, 8, 28),
                                                         _columns(T, Q, 59, 79)]))
    assert np.array_equal(_decode(X[1]), np.concatenate([_columns(T, rc, 8, 28),
                                                         _columns(T, rc, 59, 79)]))


def _counting_net(shift=0.0):
    """Unit 0 counts the matches right of the seed, unit 1 the transitions left
    of it (minus `shift` each, through the ReLU); the output is their sum + 0.5."""
    P = {k: np.array(v, dtype=np.float64) for k, v in mlp.unpack(np.zeros(mlp.N_PARAM)).items()}
    for i in range(32):
        P["W1"][(32 + i) * 4 + 0, 0] = 1.0
        P["W1"][i * 4 + 2, 1] = 1.0
    P["b1"][:2] = -shift
    P["W2"][0, 0] = P["W2"][1, 1] = 1.0
    P["W3"][:2] = 1.0
    P["b3"] = 0.5
    return mlp.pack(P)


@pytest.mark.parametrize("shift", [0.0, 6.0])
def test_forward_of_a_counting_network(shift):
    T, Qs = _seq(500, 5), _seq(500, 6)
    for k in range(0, 500, 40):  # plant some matching stretches
        Qs[k:k + 12] = T[k:k + 12]
    theta = _counting_net(shift)
    pos = [(40, 20), (200, 3), (480, 490), (2, 2), (100, 100), (90, 90)]
    X = np.stack([mlp.features(T, Qs, t, q) for t, q in pos])
    y, _ = mlp.forward(theta, X)
    ts, qs = "".join("ACGT"[b] for b in T), "".join("ACGT"[b] for b in Qs)
    pairs = {("A", "G"), ("G", "A"), ("C", "T"), ("T", "C")}
    for k, (t, q) in enumerate(pos):
        right = sum(1 for i in range(32) if t + 19 + i < 500 and q + 19 + i < 500
                    and ts[t + 19 + i] == qs[q + 19 + i])
        left = sum(1 for i in range(32) if t - 32 + i >= 0 and q - 32 + i >= 0
                   and (ts[t - 32 + i], qs[q - 32 + i]) in pairs)
        assert y[k] == max(right - shift, 0) + max(left - shift, 0) + 0.5


def _random_problem(n=40, seed=7):
    st = synth.Stream(seed, "mlp-theta")
    theta = (st.uniform(mlp.N_PARAM) * 2.0 - 1.0) * 0.5
    T, Qs = _seq(400, seed), _seq(400, seed + 1)
    pos = st.integers(0, 400, 2 * n).reshape(n, 2)
    X = np.stack([mlp.features(T, Qs, int(t), int(q)) for t, q in pos])
    target = st.uniform(n) * 6.0
    return theta, X, target


def test_gradient_matches_central_differences():
    theta, X, target = _random_problem()
    g = mlp.grad(theta, X, target)
    # coordinates of every parameter group, plus all of W3 and b3
    st = synth.Stream(11, "mlp-coords")
    idx = np.concatenate([st.integers(0, 256 * 64, 60), 256 * 64 + st.integers(0, 64, 10),
                          256 * 64 + 64 + st.integers(0, 64 * 64, 60),
                          256 * 64 + 64 + 4096 + st.integers(0, 64, 10),
                          np.arange(mlp.N_PARAM - 65, mlp.N_PARAM)])
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.N_PARAM)
        e[i] = h
        fd = (mlp.loss(theta + e, X, target) - mlp.loss(theta - e, X, target)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), i


def test_gradient_of_inactive_inputs_and_dead_units_is_zero():
    theta, X, target = _random_problem(n=3)
    g = mlp.unpack(mlp.grad(theta, X, target))
    unused = X.sum(axis=0) == 0
    assert unused.any()
    assert (g["W1"][unused] == 0).all()
    _, A = mlp.forward(theta, X)
    dead = (A["z1"] <= 0).all(axis=0)
    if dead.any():
        assert (g["b1"][dead] == 0).all() and (g["W2"][dead] == 0).all()


def test_loss_and_gradient_vanish_at_an_exact_fit():
    P = {k: np.zeros(s) for k, s in mlp.SIZES}
    P["b3"] = 2.25
    theta = mlp.pack(P)
    _, X, _ = _random_problem()
    target = np.full(X.shape[0], 2.25)
    assert mlp.loss(theta, X, target) == 0.0
    assert not mlp.grad(theta, X, target).any()


def test_adam_first_step_is_lr_times_sign():
    g = np.array([3.0, -0.5, 1e-3, -2e4, 0.0])
    theta = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    new, m, v = mlp.adam_step(theta, g, np.zeros(5), np.zeros(5), lr=0.01, step=1)
    # m_hat = g, v_hat = g^2 on the first step: the update is lr * g / (|g| + eps)
    assert np.allclose(new, theta - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_fp16_weights_round_to_nearest_half_and_keep_biases():
    P = {k: np.zeros(s) for k, s in mlp.SIZES}
    P["W1"][0, 0] = 1.0 / 3.0       # nearest half: 0.333251953125 (0x3555)
    P["W2"][1, 2] = 65519.0         # rounds to the largest half, 65504
    P["W3"][5] = 1.0 + 2.0 ** -11   # a tie: to even, 1.0
    P["b1"][3] = 1.0 / 3.0
    P["b3"] = 0.1
    Q = mlp.unpack(mlp.fp16_weights(mlp.pack(P)))
    assert Q["W1"][0, 0] == 0.333251953125
    assert Q["W2"][1, 2] == 65504.0
    assert Q["W3"][5] == 1.0
    assert Q["b1"][3] == 1.0 / 3.0 and Q["b3"] == 0.1


def test_parameter_layout():
    assert mlp.N_PARAM == 256 * 64 + 64 + 64 * 64 + 64 + 64 + 1 == 20673
    theta = np.arange(mlp.N_PARAM, dtype=np.float64)
    P = mlp.unpack(theta)
    assert P["W1"][1, 0] == 64 and P["b1"][0] == 16384 and P["W2"][0, 1] == 16449
    assert P["b3"] == 20672
    assert np.array_equal(mlp.pack(P), theta)


def test_fp16_forward_rounds_weights_and_hidden_units():
    """forward_fp16 equals forward on half-rounded weights when the hidden
    units are exact halves (small integers), and differs from it otherwise by
    at most the rounding of the hidden units."""
    theta = _counting_net(0.0)  # integer weights and biases
    T, Qs = _seq(500, 5), _seq(500, 6)
    X = np.stack([mlp.features(T, Qs, t, q) for t, q in [(40, 20), (200, 3), (90, 90)]])
    assert np.array_equal(mlp.forward_fp16(theta, X), mlp.forward(theta, X)[0])
    th, X2, _ = _random_problem(n=8, seed=3)
    a, b = mlp.forward_fp16(th, X2), mlp.forward(mlp.fp16_weights(th), X2)[0]
    assert not np.array_equal(a, b) and np.abs(a - b).max() < 0.05
