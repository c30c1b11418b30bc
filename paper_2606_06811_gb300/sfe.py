"""Python binding of libsfe: argument marshalling only.

Every step of the filter stage runs in the library's CUDA kernels; this module
converts numpy arrays, bytes and PyTorch tensors into pointers and sizes,
calls the C ABI declared in include/sfe.h and wraps the results. It fails
loudly when the library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsfe.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EOVERFLOW = 0, -1, -2, -3, -4, -5
SKIP_PASSING_ONLY = 1
TIME_STAGES = 2
NO_CELL_PLANES = 4
WALK_TWO_LAUNCHES, WALK_PERSISTENT, WALK_SPECULATIVE = 0, 1, 2
SCHED_NATURAL, SCHED_LARGEST_FIRST, SCHED_PREDICTED, SCHED_RANDOM = 0, 1, 2, 3
TEST_UNPUBLISHED_QUEUE_ENTRY = 1
TEST_DENSE_INDEX = 2
EXT_DTYPE = np.dtype([("pair", "<i4"), ("strand", "<i4"), ("t", "<i4"), ("q", "<i4"),
                      ("right", "<i4"), ("left", "<i4")])
STAGES = ("pack", "index", "count", "write", "sort", "schedule", "walk_lanes", "walk_warps",
          "output")

HIT_DTYPE = np.dtype([("strand", "<i4"), ("tpos", "<i4"), ("qpos", "<i4")])
HSP_DTYPE = np.dtype([("strand", "<i4"), ("tpos", "<i4"), ("qpos", "<i4"), ("len", "<i4"),
                      ("score", "<i4")])
BATCH_HSP_DTYPE = np.dtype([("pair", "<i4"), ("strand", "<i4"), ("tpos", "<i4"), ("qpos", "<i4"),
                            ("len", "<i4"), ("score", "<i4")])


class SfeError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class Params(C.Structure):
    _fields_ = [("seed_pattern", C.c_char_p), ("transition", C.c_int32),
                ("strands", C.c_int32), ("scores", C.c_int32 * 16), ("xdrop", C.c_int32),
                ("hsp_thresh", C.c_int32), ("flags", C.c_int32), ("input_codes", C.c_int32),
                ("lane_cap", C.c_int32), ("lanes_per_sm", C.c_int32), ("tile_hits", C.c_int64),
                ("walk_chunk", C.c_int32), ("walk_mode", C.c_int32), ("walk_schedule", C.c_int32),
                ("ext_log_every", C.c_int32), ("ext_log", C.c_void_p), ("ext_log_cap", C.c_int64),
                ("model", C.c_void_p), ("wait_limit", C.c_int32), ("test_hooks", C.c_int32),
                ("step", C.c_int32), ("spec_window", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("hits", C.c_int64), ("extended", C.c_int64), ("cells", C.c_int64),
                ("hsps", C.c_int64), ("lane_tasks", C.c_int64), ("warp_tasks", C.c_int64),
                ("warp_cells", C.c_int64), ("tiles", C.c_int64), ("launches", C.c_int64),
                ("ext_logged", C.c_int64), ("shadow_cells", C.c_int64),
                ("stage_ms", C.c_double * len(STAGES)),
                ("stage_launches", C.c_int64 * len(STAGES)),
                ("deferred_tasks", C.c_int64)]

    def as_dict(self) -> dict:
        d = {k: int(getattr(self, k)) for k, _ in self._fields_[:11]}
        d["stage_ms"] = {n: float(self.stage_ms[i]) for i, n in enumerate(STAGES)}
        d["stage_launches"] = {n: int(self.stage_launches[i]) for i, n in enumerate(STAGES)}
        d["deferred_tasks"] = int(self.deferred_tasks)
        return d


class YdropParams(C.Structure):
    _fields_ = [("scores", C.c_int32 * 16), ("gap_open", C.c_int32), ("gap_extend", C.c_int32),
                ("ydrop", C.c_int32), ("gapped_thresh", C.c_int32), ("band", C.c_int32),
                ("input_codes", C.c_int32), ("batch", C.c_int64)]


class YdropStats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("anchors", "skipped", "extended", "cells", "shadow",
                                          "shadow_cells", "committed", "batches")] + \
               [("device_ms", C.c_double), ("total_ms", C.c_double)]

    def as_dict(self) -> dict:
        return {k: (float if k.endswith("_ms") else int)(getattr(self, k))
                for k, _ in self._fields_}


GALIGN_DTYPE = np.dtype([("strand", "<i4"), ("tstart", "<i4"), ("tend", "<i4"),
                         ("qstart", "<i4"), ("qend", "<i4"), ("score", "<i4")])

_lib = None


def lib() -> C.CDLL:
    """The loaded libsfe (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libsfe.so is not built ({LIB_PATH}); run "
                              "paper_2606_06811_gb300.build.build() or __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        L.sfe_params_default.argtypes = [C.POINTER(Params)]
        L.sfe_strerror.argtypes = [C.c_int]
        L.sfe_strerror.restype = C.c_char_p
        L.sfe_last_error.argtypes = []
        L.sfe_last_error.restype = C.c_char_p
        L.sfe_ctx_create.argtypes = [C.c_int, C.POINTER(vp)]
        L.sfe_ctx_set_stream.argtypes = [vp, vp]
        L.sfe_ctx_fail_next_allocs.argtypes = [vp, i32]
        L.sfe_ctx_set_walk.argtypes = [vp, C.POINTER(Params)]
        L.sfe_ydrop_params_default.argtypes = [C.POINTER(YdropParams)]
        L.sfe_gapped_extend.argtypes = [vp, vp, i64, vp, i64, vp, i64, C.POINTER(YdropParams), vp,
                                        i64, C.POINTER(i64), C.POINTER(YdropStats)]
        L.sfe_test_radix_sort.argtypes = [vp, vp, i64, i32, i32, i32]
        L.sfe_test_radix_sort.restype = C.c_int
        L.sfe_test_committed_boxes.argtypes = [vp, i64, vp, i64, vp]
        L.sfe_test_committed_boxes.restype = C.c_int
        L.sfe_ctx_fail_next_allocs.restype = C.c_int
        L.sfe_ctx_destroy.argtypes = [vp]
        L.sfe_ctx_destroy.restype = None
        L.sfe_index_build.argtypes = [vp, vp, i64, C.POINTER(Params), C.POINTER(vp)]
        L.sfe_index_free.argtypes = [vp]
        L.sfe_index_free.restype = None
        L.sfe_seed_hits.argtypes = [vp, vp, vp, i64, i32, vp, i64, C.POINTER(i64)]
        L.sfe_ungapped_xdrop.argtypes = [vp, vp, vp, i64, vp, i64, C.POINTER(C.c_int32 * 16), i32,
                                         i32, vp, i64, C.POINTER(i64), C.POINTER(Stats)]
        L.sfe_run.argtypes = [vp, vp, i64, vp, i64, C.POINTER(Params), vp, i64, C.POINTER(i64),
                              C.POINTER(Stats)]
        L.sfe_run_batch.argtypes = [vp, vp, vp, vp, vp, i32, C.POINTER(Params), vp, i64,
                                    C.POINTER(i64), C.POINTER(Stats)]
        L.sfe_batch_plan_create.argtypes = [vp, vp, vp, i32, C.POINTER(Params), i64,
                                            C.POINTER(vp)]
        L.sfe_batch_plan_run.argtypes = [vp, vp, vp, vp, i64, C.POINTER(i64), C.POINTER(Stats)]
        L.sfe_batch_plan_free.argtypes = [vp]
        L.sfe_batch_plan_free.restype = None
        L.sfe_mlp_param_count.argtypes = []
        L.sfe_mlp_param_count.restype = i32
        L.sfe_mlp_model_bytes.argtypes = []
        L.sfe_mlp_model_bytes.restype = i64
        L.sfe_mlp_init.argtypes = [vp, vp, C.c_uint64]
        L.sfe_mlp_pack.argtypes = [vp, vp, vp]
        L.sfe_mlp_data_create.argtypes = [vp, vp, vp, vp, vp, i32, i32, i32, vp, i64,
                                          C.POINTER(vp)]
        L.sfe_mlp_data_free.argtypes = [vp]
        L.sfe_mlp_data_free.restype = None
        L.sfe_mlp_loss_grad.argtypes = [vp, vp, vp, vp, vp, C.POINTER(C.c_double)]
        L.sfe_mlp_predict.argtypes = [vp, vp, vp, vp]
        L.sfe_mlp_train.argtypes = [vp, vp, vp, i32, i32, C.c_float, C.c_uint64,
                                    C.POINTER(C.c_double)]
        for f in ("sfe_params_default", "sfe_ctx_create", "sfe_ctx_set_stream", "sfe_index_build",
                  "sfe_seed_hits", "sfe_ungapped_xdrop", "sfe_run", "sfe_run_batch",
                  "sfe_mlp_init", "sfe_mlp_pack", "sfe_mlp_data_create", "sfe_mlp_loss_grad",
                  "sfe_mlp_predict", "sfe_mlp_train", "sfe_batch_plan_create",
                  "sfe_batch_plan_run"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def _check(code: int) -> int:
    if code != OK:
        raise SfeError(code, lib().sfe_last_error().decode(errors="replace") or
                       lib().sfe_strerror(code).decode())
    return code


def ydrop_params(**kw) -> YdropParams:
    """sfe_ydrop_params_default(), then the given fields."""
    p = YdropParams()
    _check(lib().sfe_ydrop_params_default(C.byref(p)))
    for k, v in kw.items():
        if k == "scores":
            p.scores[:] = [int(x) for x in np.asarray(v, dtype=np.int64).reshape(16)]
        else:
            setattr(p, k, v)
    return p


def default_params(**kw) -> Params:
    """sfe_params_default(), then the given fields (scores may be a 4x4 or 16 array)."""
    p = Params()
    _check(lib().sfe_params_default(C.byref(p)))
    for k, v in kw.items():
        if k == "scores":
            p.scores[:] = [int(x) for x in np.asarray(v, dtype=np.int64).reshape(16)]
        elif k == "seed_pattern":
            p._pattern_keep = v.encode() if isinstance(v, str) else v
            p.seed_pattern = p._pattern_keep
        else:
            setattr(p, k, v)
    return p


def _buf(x):
    """(pointer, size in bytes, keep-alive) of a torch tensor, numpy array or bytes."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if not x.is_contiguous():
                raise ValueError("tensor must be contiguous")
            return x.data_ptr(), x.numel() * x.element_size(), x
    except ImportError:
        pass
    if isinstance(x, (bytes, bytearray, memoryview)):
        x = np.frombuffer(x, dtype=np.uint8)
    a = np.ascontiguousarray(x)
    if a.size == 0:
        a = np.zeros(1, dtype=a.dtype)
        return a.ctypes.data, 0, a
    return a.ctypes.data, a.nbytes, a


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class Context:
    """A device context (stream + scratch arena) of libsfe."""

    def __init__(self, device: int = 0, stream=None):
        h = C.c_void_p()
        _check(lib().sfe_ctx_create(int(device), C.byref(h)))
        self.h = h
        self.device = int(device)
        if stream is not None:
            self.set_stream(stream)

    def set_stream(self, stream) -> None:
        _check(lib().sfe_ctx_set_stream(self.h, _stream_handle(stream)))

    def test_radix_sort(self, keys, lo: int, hi: int, device_count: bool = False) -> None:
        """Test hook: the library's stable radix sort of a device tensor of int64 keys
        by bits [lo, hi), in place."""
        ptr, nbytes, keep = _buf(keys)
        _check(lib().sfe_test_radix_sort(self.h, ptr, nbytes // 8, int(lo), int(hi),
                                         int(bool(device_count))))

    def gapped_extend(self, target, query, hsps, params: YdropParams | None = None,
                      cap: int | None = None):
        """Gapped Y-drop extension of the HSPs (sfe_gapped_extend): (alignments as numpy
        GALIGN_DTYPE sorted, stats dict)."""
        p = params or ydrop_params()
        tptr, tn, tkeep = _buf(target)
        qptr, qn, qkeep = _buf(query)
        if isinstance(hsps, np.ndarray) and hsps.dtype != np.int32:
            hsps = np.ascontiguousarray(hsps).view(np.int32).reshape(-1)
        hptr, hn, hkeep = _buf(hsps)
        n = C.c_int64(0)
        st = YdropStats()
        cap = 1 << 16 if cap is None else int(cap)
        while True:
            buf = np.zeros(max(cap, 1), dtype=GALIGN_DTYPE)
            code = lib().sfe_gapped_extend(self.h, tptr, tn, qptr, qn, hptr, hn // 20, C.byref(p),
                                           buf.ctypes.data, cap, C.byref(n), C.byref(st))
            if code == EOVERFLOW and n.value > cap:
                cap = int(n.value)
                continue
            _check(code)
            return buf[: n.value], st.as_dict()

    def set_walk(self, params: Params | None) -> None:
        """Walk settings for later ungapped_xdrop calls (sfe_ctx_set_walk); None: defaults."""
        _check(lib().sfe_ctx_set_walk(self.h, C.byref(params) if params is not None else None))

    def fail_next_allocs(self, n: int) -> None:
        """Test hook: the next n scratch allocations fail with SFE_ENOMEM."""
        _check(lib().sfe_ctx_fail_next_allocs(self.h, int(n)))

    def close(self) -> None:
        if getattr(self, "h", None):
            lib().sfe_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------ calls

    def index_build(self, target, params: Params | None = None) -> "Index":
        p = params or default_params()
        ptr, n, keep = _buf(target)
        h = C.c_void_p()
        _check(lib().sfe_index_build(self.h, ptr, n, C.byref(p), C.byref(h)))
        return Index(h, n)

    def seed_hits(self, index: "Index", query, strands: int = 3, cap: int | None = None,
                  out=None):
        """Hits sorted by (strand, diagonal, tpos); numpy HIT_DTYPE unless `out` is given."""
        ptr, n, keep = _buf(query)
        nh = C.c_int64(0)
        if out is not None:
            optr, ocap, _ = _buf(out)
            _check(lib().sfe_seed_hits(self.h, index.h, ptr, n, int(strands), optr,
                                       ocap // HIT_DTYPE.itemsize, C.byref(nh)))
            return out, int(nh.value)
        cap = 1 << 16 if cap is None else int(cap)
        while True:
            buf = np.zeros(max(cap, 1), dtype=HIT_DTYPE)
            code = lib().sfe_seed_hits(self.h, index.h, ptr, n, int(strands), buf.ctypes.data,
                                       cap, C.byref(nh))
            if code == EOVERFLOW and nh.value > cap:
                cap = int(nh.value)
                continue
            _check(code)
            return buf[: nh.value]

    def ungapped_xdrop(self, index: "Index", query, hits, scores, X: int, thresh: int,
                       cap: int | None = None):
        """(HSPs as numpy HSP_DTYPE sorted, stats dict) for a hit list."""
        qptr, qn, qkeep = _buf(query)
        if isinstance(hits, np.ndarray) and hits.dtype == HIT_DTYPE:
            hits = hits.view(np.int32).reshape(-1)
        hptr, hn, hkeep = _buf(hits)
        nhits = hn // HIT_DTYPE.itemsize
        sc = (C.c_int32 * 16)(*[int(x) for x in np.asarray(scores, dtype=np.int64).reshape(16)])
        return self._retry(cap, lambda buf, cp, nout, st: lib().sfe_ungapped_xdrop(
            self.h, index.h, qptr, qn, hptr, nhits, C.byref(sc), int(X), int(thresh), buf, cp,
            nout, st))

    def run(self, target, query, params: Params | None = None, cap: int | None = None,
            out=None):
        """The whole filter stage. Returns (HSPs, stats); HSPs are numpy HSP_DTYPE, or the
        first rows of `out` (an int32 tensor of shape (cap, 5)) when it is given."""
        p = params or default_params()
        tptr, tn, tkeep = _buf(target)
        qptr, qn, qkeep = _buf(query)
        if out is not None:
            optr, on, _ = _buf(out)
            nout = C.c_int64(0)
            st = Stats()
            _check(lib().sfe_run(self.h, tptr, tn, qptr, qn, C.byref(p), optr,
                                 on // HSP_DTYPE.itemsize, C.byref(nout), C.byref(st)))
            return out[: nout.value], st.as_dict()
        return self._retry(cap, lambda buf, cp, nout, st: lib().sfe_run(
            self.h, tptr, tn, qptr, qn, C.byref(p), buf, cp, nout, st))

    def run_batch(self, targets, toff, queries, qoff, params: Params | None = None,
                  cap: int | None = None, out=None):
        """Filter stage over a batch of pairs given back to back with int64 offsets (host).
        Returns (HSPs as numpy BATCH_HSP_DTYPE sorted by pair first, stats), or the first
        rows of `out` (int32 tensor of shape (cap, 6)) when it is given."""
        p = params or default_params()
        tptr, _, tkeep = _buf(targets)
        qptr, _, qkeep = _buf(queries)
        to = np.ascontiguousarray(toff, dtype=np.int64)
        qo = np.ascontiguousarray(qoff, dtype=np.int64)
        npairs = int(to.size - 1)
        nout = C.c_int64(0)
        st = Stats()
        if out is not None:
            optr, on, _ = _buf(out)
            _check(lib().sfe_run_batch(self.h, tptr, to.ctypes.data, qptr, qo.ctypes.data, npairs,
                                       C.byref(p), optr, on // BATCH_HSP_DTYPE.itemsize,
                                       C.byref(nout), C.byref(st)))
            return out[: nout.value], st.as_dict()
        cap = 1 << 16 if cap is None else int(cap)
        while True:
            buf = np.zeros(max(cap, 1), dtype=BATCH_HSP_DTYPE)
            code = lib().sfe_run_batch(self.h, tptr, to.ctypes.data, qptr, qo.ctypes.data, npairs,
                                       C.byref(p), buf.ctypes.data, cap, C.byref(nout),
                                       C.byref(st))
            if code == EOVERFLOW and nout.value > cap:
                cap = int(nout.value)
                continue
            _check(code)
            return buf[: nout.value], st.as_dict()

    def batch_plan(self, toff, qoff, params: Params | None = None,
                   hit_cap: int = 0) -> "BatchPlan":
        """A batch of fixed pair lengths captured as a CUDA graph (sfe_batch_plan_create)."""
        p = params or default_params()
        to = np.ascontiguousarray(toff, dtype=np.int64)
        qo = np.ascontiguousarray(qoff, dtype=np.int64)
        h = C.c_void_p()
        _check(lib().sfe_batch_plan_create(self.h, to.ctypes.data, qo.ctypes.data,
                                           int(to.size - 1), C.byref(p), int(hit_cap),
                                           C.byref(h)))
        return BatchPlan(h, p)

    # ------------------------------------------------ work predictor (MLP)

    def mlp_init(self, params, seed: int) -> None:
        """Random initial FP32 parameters into the device tensor `params`."""
        ptr, n, keep = _buf(params)
        if n < 4 * mlp_param_count():
            raise ValueError("params holds fewer than sfe_mlp_param_count() floats")
        _check(lib().sfe_mlp_init(self.h, ptr, int(seed)))

    def mlp_pack(self, params, model) -> None:
        """FP16 inference blob (device tensor of sfe_mlp_model_bytes() bytes) of `params`."""
        pptr, pn, pk = _buf(params)
        mptr, mn, mk = _buf(model)
        if pn < 4 * mlp_param_count() or mn < mlp_model_bytes():
            raise ValueError("params or model buffer too small")
        _check(lib().sfe_mlp_pack(self.h, pptr, mptr))

    def mlp_data(self, targets, toff, queries, qoff, recs, input_codes: int = 0,
                 span: int = 19) -> "MlpData":
        """Training samples: extension records (EXT_DTYPE, host or device) and their pairs'
        sequences back to back with int64 offsets, as for run_batch; span is the seed span
        of the run that logged them."""
        tptr, _, tkeep = _buf(targets)
        qptr, _, qkeep = _buf(queries)
        to = np.ascontiguousarray(toff, dtype=np.int64)
        qo = np.ascontiguousarray(qoff, dtype=np.int64)
        rptr, rn, rkeep = _buf(recs)
        n = rn // EXT_DTYPE.itemsize
        h = C.c_void_p()
        _check(lib().sfe_mlp_data_create(self.h, tptr, to.ctypes.data, qptr, qo.ctypes.data,
                                         int(to.size - 1), int(input_codes), int(span), rptr,
                                         n, C.byref(h)))
        return MlpData(h, n)

    def mlp_loss_grad(self, data: "MlpData", params, grad=None, preds=None) -> float:
        """Mean squared error of the FP32 network; fills the device tensors grad / preds."""
        pptr, _, pk = _buf(params)
        gptr = _buf(grad)[0] if grad is not None else None
        optr = _buf(preds)[0] if preds is not None else None
        loss = C.c_double(0.0)
        _check(lib().sfe_mlp_loss_grad(self.h, data.h, pptr, gptr, optr, C.byref(loss)))
        return float(loss.value)

    def mlp_predict(self, data: "MlpData", model, preds) -> None:
        """Predictions of the FP16 model into the device tensor preds (one per record)."""
        _check(lib().sfe_mlp_predict(self.h, data.h, _buf(model)[0], _buf(preds)[0]))

    def mlp_train(self, data: "MlpData", params, epochs: int, batch: int = 4096,
                  lr: float = 1e-3, seed: int = 0) -> list[float]:
        """Adam on minibatches, in place on `params`; returns each epoch's loss."""
        pptr, _, pk = _buf(params)
        out = (C.c_double * max(int(epochs), 1))()
        _check(lib().sfe_mlp_train(self.h, data.h, pptr, int(epochs), int(batch), float(lr),
                                   int(seed), out))
        return [float(out[i]) for i in range(int(epochs))]

    def _retry(self, cap, call):
        cap = 1 << 16 if cap is None else int(cap)
        nout = C.c_int64(0)
        st = Stats()
        while True:
            buf = np.zeros(max(cap, 1), dtype=HSP_DTYPE)
            code = call(buf.ctypes.data, cap, C.byref(nout), C.byref(st))
            if code == EOVERFLOW and nout.value > cap:
                cap = int(nout.value)
                continue
            _check(code)
            return buf[: nout.value], st.as_dict()


class Index:
    """A seeding index over one target (owned device memory)."""

    def __init__(self, h, tlen: int):
        self.h = h
        self.tlen = tlen

    def close(self) -> None:
        if getattr(self, "h", None):
            lib().sfe_index_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchPlan:
    """A captured batch (owned device memory and CUDA graph); run() replays it."""

    def __init__(self, h, params):
        self.h = h
        self._params = params  # pointers in it were captured

    def run(self, targets, queries, cap: int | None = None, out=None):
        """Replay on new sequences of the plan's lengths. Returns (HSPs as numpy
        BATCH_HSP_DTYPE, stats), or the first rows of `out` (int32, shape (cap, 6))."""
        tptr, _, tkeep = _buf(targets)
        qptr, _, qkeep = _buf(queries)
        nout = C.c_int64(0)
        st = Stats()
        if out is not None:
            optr, on, _ = _buf(out)
            _check(lib().sfe_batch_plan_run(self.h, tptr, qptr, optr,
                                            on // BATCH_HSP_DTYPE.itemsize, C.byref(nout),
                                            C.byref(st)))
            return out[: nout.value], st.as_dict()
        cap = 1 << 16 if cap is None else int(cap)
        while True:
            buf = np.zeros(max(cap, 1), dtype=BATCH_HSP_DTYPE)
            code = lib().sfe_batch_plan_run(self.h, tptr, qptr, buf.ctypes.data, cap,
                                            C.byref(nout), C.byref(st))
            if code == EOVERFLOW and nout.value > cap:
                cap = int(nout.value)
                continue
            _check(code)
            return buf[: nout.value], st.as_dict()

    def close(self) -> None:
        if getattr(self, "h", None):
            lib().sfe_batch_plan_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MlpData:
    """Training samples of the work predictor (owned device memory)."""

    def __init__(self, h, n: int):
        self.h = h
        self.n = n

    def close(self) -> None:
        if getattr(self, "h", None):
            lib().sfe_mlp_data_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def test_committed_boxes(boxes, queries):
    """Test hook (host only): for each (strand, t, q) row of `queries`, whether
    one of the committed alignment boxes (rows of GALIGN_DTYPE fields, added in
    order) contains it, through the gapped stage's own box index."""
    b = np.ascontiguousarray(boxes, dtype=np.int32).reshape(-1, 6)
    q = np.ascontiguousarray(queries, dtype=np.int32).reshape(-1, 3)
    out = np.zeros(q.shape[0], dtype=np.uint8)
    _check(lib().sfe_test_committed_boxes(b.ctypes.data if b.size else None, b.shape[0],
                                          q.ctypes.data if q.size else None, q.shape[0],
                                          out.ctypes.data if out.size else None))
    return out.astype(bool)


def mlp_param_count() -> int:
    return int(lib().sfe_mlp_param_count())


def mlp_model_bytes() -> int:
    return int(lib().sfe_mlp_model_bytes())


def exported_symbols() -> list[str]:
    """Names of the functions declared in include/sfe.h."""
    import re
    hdr = os.path.join(os.path.dirname(_HERE), "include", "sfe.h")
    txt = open(hdr).read()
    return sorted(set(re.findall(r"\b(sfe_[a-z_]+)\s*\(", txt)))
