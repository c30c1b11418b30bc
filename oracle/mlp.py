"""Oracle of the work predictor (the learned schedule's MLP), in float64 numpy.

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the library.

The paper learns nothing; it names the problem the predictor serves. Section 8
describes extensions whose lengths vary so widely that a synchronous warp
waits for its longest lane, and cites length pre-sorting with persistent
queues as the known remedy when lengths are known in advance. The predictor
estimates an X-drop extension's length from the seed's sequence context so
that independent work can be ordered by it; it never changes which HSPs are
reported. Its definition (inputs, layers, target) is fixed by the library's
interface, restated here from that definition:

* inputs: for a hit at (t, q) on a strand-oriented query Qs and a seed of
  span s, the diagonal columns (T[t - 32 + i], Qs[q - 32 + i]) (columns
  0..31, left of the seed) and (T[t + s + i], Qs[q + s + i]) (columns 32..63,
  right of it), i = 0..31, each one-hot over its substitution class, the XOR
  of the 2-bit codes (A=0, C=1, G=2, T=3: 0 is a match, 2 a transition, 1 and
  3 the two transversion kinds): input index column * 4 + class; a column
  with either position outside its sequence sets none of its inputs;
* layers: z1 = x W1 + b1, a1 = relu(z1), z2 = a1 W2 + b2, a2 = relu(z2),
  y = a2 . W3 + b3, with W1 256 x 64 and W2 64 x 64 stored row = input unit;
* parameter vector: W1 (row-major), b1, W2 (row-major), b2, W3, b3;
* target: log(1 + right + left), the bases the X-drop scored on the two
  sides of the seed (Section 1's ungapped extension);
* loss: mean squared error over the samples;
* Adam (Kingma and Ba, 2015): beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected.

Everything is dense float64 and unblocked: the features are built as a
matrix, the layers are matrix products, and the gradient is written out by
the chain rule, layer by layer.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, CTX = 256, 64, 32
SPAN = 19  # the default 12of19 seed
SIZES = (("W1", (N_IN, N_HID)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
         ("W3", (N_HID,)), ("b3", ()))
N_PARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta) -> dict:
    """The parameter vector split into named arrays (views)."""
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (N_PARAM,)
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = theta[o:o + k].reshape(shape) if shape else theta[o]
        o += k
    return out


def pack(parts: dict) -> np.ndarray:
    return np.concatenate([np.asarray(parts[n], dtype=np.float64).reshape(-1) for n, _ in SIZES])


def features(T, Qs, t: int, q: int, span: int = SPAN) -> np.ndarray:
    """The 256 one-hot inputs of a hit at (t, q); T and Qs hold codes 0..3."""
    x = np.zeros(N_IN)
    starts = [(t - CTX, q - CTX), (t + span, q + span)]  # left flank, right flank
    for side, (t0, q0) in enumerate(starts):
        for i in range(CTX):
            pt, pq = t0 + i, q0 + i
            if 0 <= pt < len(T) and 0 <= pq < len(Qs):
                cls = int(T[pt]) ^ int(Qs[pq])
                x[(side * CTX + i) * 4 + cls] = 1.0
    return x


def feature_matrix(targets, queries, recs, span: int = SPAN) -> np.ndarray:
    """Features of extension records (fields pair, strand, t, q): targets[p] and
    queries[p] are pair p's sequences (codes); strand 1 reads the reverse
    complement of the query."""
    rc = {}
    X = np.zeros((len(recs), N_IN))
    for i, r in enumerate(recs):
        p, s = int(r["pair"]), int(r["strand"])
        Q = queries[p]
        if s:
            if p not in rc:
                rc[p] = (3 - np.asarray(Q, dtype=np.int64))[::-1]
            Q = rc[p]
        X[i] = features(targets[p], Q, int(r["t"]), int(r["q"]), span)
    return X


def targets_of(recs) -> np.ndarray:
    return np.log1p(np.asarray(recs["right"], dtype=np.float64) +
                    np.asarray(recs["left"], dtype=np.float64))


def forward(theta, X) -> tuple[np.ndarray, dict]:
    """Predictions for the rows of X, and the activations the gradient needs."""
    P = unpack(theta)
    z1 = X @ P["W1"] + P["b1"]
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ P["W2"] + P["b2"]
    a2 = np.maximum(z2, 0.0)
    y = a2 @ P["W3"] + P["b3"]
    return y, {"z1": z1, "a1": a1, "z2": z2, "a2": a2}


def loss(theta, X, target) -> float:
    y, _ = forward(theta, X)
    return float(np.mean((y - target) ** 2))


def grad(theta, X, target) -> np.ndarray:
    """Gradient of the mean squared error, by the chain rule."""
    P = unpack(theta)
    y, A = forward(theta, X)
    n = X.shape[0]
    dy = 2.0 * (y - target) / n                  # d loss / d y
    g = {"b3": dy.sum(), "W3": A["a2"].T @ dy}
    dz2 = np.outer(dy, P["W3"]) * (A["z2"] > 0)  # through the output layer and ReLU
    g["b2"] = dz2.sum(axis=0)
    g["W2"] = A["a1"].T @ dz2
    dz1 = (dz2 @ P["W2"].T) * (A["z1"] > 0)
    g["b1"] = dz1.sum(axis=0)
    g["W1"] = X.T @ dz1
    return pack(g)


def adam_step(theta, g, m, v, lr: float, step: int, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update; returns (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def forward_fp16(theta, X) -> np.ndarray:
    """The inference model as the tensor cores compute it: weights rounded to
    IEEE half, and the hidden units of the first layer rounded to half after
    the ReLU (they are the half-precision inputs of the second product); sums
    in float64 here (float32 on the device)."""
    P = unpack(fp16_weights(theta))
    h1 = np.maximum(X @ P["W1"] + P["b1"], 0.0).astype(np.float16).astype(np.float64)
    h2 = np.maximum(h1 @ P["W2"] + P["b2"], 0.0)
    return h2 @ P["W3"] + P["b3"]


def fp16_weights(theta) -> np.ndarray:
    """The inference model's parameters: weights rounded to IEEE half (nearest,
    ties to even), biases kept."""
    P = unpack(theta)
    for name in ("W1", "W2", "W3"):
        P[name] = P[name].astype(np.float16).astype(np.float64)
    return pack(P)
