"""The pins of the oracle MLP must reject an oracle with a plausible mistake
planted in it: each mutant is oracle/mlp.py with one textual change, loaded
as a separate module on the CPU, and at least one pin of
tests/test_oracle_mlp.py must fail on it while all pass on the real one."""
from __future__ import annotations

import importlib.util
import os
import sys

import numpy as np
import pytest

from tests import test_oracle_mlp as pins

SRC = os.path.join(os.path.dirname(os.path.dirname(__file__)), "oracle", "mlp.py")

# (name, old text, new text)
MUTANTS = [
    ("relu_mask_dropped_in_backward", "dz2 = np.outer(dy, P[\"W3\"]) * (A[\"z2\"] > 0)",
     "dz2 = np.outer(dy, P[\"W3\"])"),
    ("w2_not_transposed_in_backward", "dz1 = (dz2 @ P[\"W2\"].T)", "dz1 = (dz2 @ P[\"W2\"])"),
    ("loss_gradient_factor", "dy = 2.0 * (y - target) / n", "dy = (y - target) / n"),
    ("left_flank_off_by_one", "starts = [(t - CTX, q - CTX), (t + span, q + span)]",
     "starts = [(t - CTX + 1, q - CTX + 1), (t + span, q + span)]"),
    ("right_flank_without_span", "starts = [(t - CTX, q - CTX), (t + span, q + span)]",
     "starts = [(t - CTX, q - CTX), (t, q)]"),
    ("class_is_target_base", "cls = int(T[pt]) ^ int(Qs[pq])", "cls = int(T[pt])"),
    ("flank_column_order", "x[(side * CTX + i) * 4 + cls] = 1.0", "x[(i * 2 + side) * 4 + cls] = 1.0"),
    ("rc_without_complement", "rc[p] = (3 - np.asarray(Q, dtype=np.int64))[::-1]",
     "rc[p] = np.asarray(Q, dtype=np.int64)[::-1]"),
    ("adam_without_bias_correction", "mh = m / (1 - b1 ** step)", "mh = m"),
    ("bias_b1_dropped", "z1 = X @ P[\"W1\"] + P[\"b1\"]", "z1 = X @ P[\"W1\"]"),
    ("fp16_hidden_not_rounded", ".astype(np.float16).astype(np.float64)\n    h2",
     "\n    h2"),
]


def _load(path: str, name: str):
    spec = importlib.util.spec_from_file_location(name, path)
    mod = importlib.util.module_from_spec(spec)
    sys.modules[name] = mod
    spec.loader.exec_module(mod)
    return mod


def _pins() -> list:
    out = []
    for n in dir(pins):
        if n.startswith("test_"):
            f = getattr(pins, n)
            marks = getattr(f, "pytestmark", [])
            params = [m for m in marks if m.name == "parametrize"]
            if params:
                names = [s.strip() for s in params[0].args[0].split(",")]
                for vals in params[0].args[1]:
                    vals = vals if isinstance(vals, tuple) else (vals,)
                    out.append((n, lambda f=f, kw=dict(zip(names, vals)): f(**kw)))
            else:
                out.append((n, f))
    return out


def _rejects(mod) -> list:
    failed = []
    saved = pins.mlp
    pins.mlp = mod
    try:
        for name, fn in _pins():
            try:
                fn()
            except Exception:
                failed.append(name)
    finally:
        pins.mlp = saved
    return failed


def test_the_real_oracle_passes_every_pin():
    assert _rejects(pins.mlp) == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_rejected(name, old, new, tmp_path):
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / f"mlp_{name}.py"
    path.write_text(src.replace(old, new))
    mod = _load(str(path), f"mlp_mutant_{name}")
    assert _rejects(mod), f"no pin rejects the mutant {name}"
