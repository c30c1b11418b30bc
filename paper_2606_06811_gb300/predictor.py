"""The work predictor of the learned schedule: collecting its training data
from runs of the filter stage, training it with the library's kernels, and
storing it.

The filter stage logs (seed hit, bases scored on each side) for a hashed
sample of its extensions (sfe_params.ext_log_every); those records and the
sequences they refer to are the training set. Training, inference and the
schedule all run in libsfe (include/sfe.h); this module only arranges the
buffers. A trained model changes the order in which the persistent walk
takes its chunks of hits (SFE_SCHED_PREDICTED), never the HSPs it reports.
"""
from __future__ import annotations

import json
import struct
from dataclasses import dataclass, field

import numpy as np

from . import sfe

_MAGIC = b"SFEMLP01"


def collect(ctx: "sfe.Context", target, query, every: int, cap: int = 1 << 22, params=None):
    """Run the filter stage on one pair with the extension log on. Returns
    (records as an int32 device tensor of shape (n, 6): pair, strand, t, q,
    right, left; the run's stats)."""
    import torch
    log = torch.zeros((int(cap), 6), dtype=torch.int32, device=f"cuda:{ctx.device}")
    p = params if params is not None else sfe.default_params()
    p.ext_log_every = int(every)
    p.ext_log = log.data_ptr()
    p.ext_log_cap = int(cap)
    _, st = ctx.run(target, query, p)
    n = min(int(st["ext_logged"]), int(cap))
    p.ext_log = None
    p.ext_log_every = 0
    return log[:n], st


@dataclass
class Predictor:
    """FP32 parameters (device tensor) and the FP16 inference blob made from them."""
    params: object
    model: object
    history: list = field(default_factory=list)  # per-epoch training loss
    meta: dict = field(default_factory=dict)

    def save(self, path: str) -> None:
        """Flat file: magic, 8-byte header length, JSON header, float32 parameters."""
        theta = self.params.detach().cpu().numpy().astype("<f4")
        head = json.dumps({"param_count": int(theta.size), "dtype": "float32",
                           "layout": ["W1[256][64]", "b1[64]", "W2[64][64]", "b2[64]", "W3[64]",
                                      "b3"],
                           "inputs": "32 + 32 flank columns x substitution class (T xor Q)",
                           "history": [float(x) for x in self.history],
                           "meta": self.meta}).encode()
        with open(path, "wb") as f:
            f.write(_MAGIC)
            f.write(struct.pack("<Q", len(head)))
            f.write(head)
            f.write(theta.tobytes())

    @staticmethod
    def load(ctx: "sfe.Context", path: str) -> "Predictor":
        import torch
        with open(path, "rb") as f:
            if f.read(8) != _MAGIC:
                raise ValueError(f"{path} is not a predictor file")
            (hl,) = struct.unpack("<Q", f.read(8))
            head = json.loads(f.read(hl))
            theta = np.frombuffer(f.read(), dtype="<f4")
        if head.get("param_count") != sfe.mlp_param_count() or theta.size != head["param_count"]:
            raise ValueError(f"{path}: parameter count does not match the library")
        dev = f"cuda:{ctx.device}"
        params = torch.from_numpy(theta.copy()).to(dev)
        model = torch.zeros(sfe.mlp_model_bytes(), dtype=torch.uint8, device=dev)
        ctx.mlp_pack(params, model)
        return Predictor(params, model, head.get("history", []), head.get("meta", {}))


def training_data(ctx: "sfe.Context", runs, span: int = 19) -> "sfe.MlpData":
    """One MlpData over several runs: `runs` is a list of (target, query, records)
    with codes 0..3 (numpy) and the records of collect(); run i becomes pair i.
    span: the seed span of those runs."""
    import torch
    ts = [np.asarray(r[0], dtype=np.uint8) for r in runs]
    qs = [np.asarray(r[1], dtype=np.uint8) for r in runs]
    toff = np.concatenate([[0], np.cumsum([t.size for t in ts])]).astype(np.int64)
    qoff = np.concatenate([[0], np.cumsum([q.size for q in qs])]).astype(np.int64)
    recs = []
    for i, r in enumerate(runs):
        x = r[2].clone()
        x[:, 0] = i
        recs.append(x)
    recs = torch.cat(recs).contiguous() if recs else torch.zeros((0, 6), dtype=torch.int32)
    return ctx.mlp_data(np.concatenate(ts), toff, np.concatenate(qs), qoff, recs, input_codes=1,
                        span=span)


def train(ctx: "sfe.Context", data: "sfe.MlpData", epochs: int = 4, batch: int = 4096,
          lr: float = 1e-3, seed: int = 0, init_seed: int = 1) -> Predictor:
    """Initialise, train with Adam on the device and pack the FP16 model."""
    import torch
    dev = f"cuda:{ctx.device}"
    params = torch.zeros(sfe.mlp_param_count(), dtype=torch.float32, device=dev)
    ctx.mlp_init(params, init_seed)
    hist = ctx.mlp_train(data, params, epochs, batch, lr, seed)
    model = torch.zeros(sfe.mlp_model_bytes(), dtype=torch.uint8, device=dev)
    ctx.mlp_pack(params, model)
    return Predictor(params, model, hist, {"epochs": epochs, "batch": batch, "lr": lr,
                                           "samples": int(data.n)})
