"""Python binding of the RotorMap C ABI (``include/rotormap.h``).

Argument marshalling only: every step runs in ``librotormap.so``. Functions
keep the C names; they take torch tensors (device memory) and enqueue work on
torch's current CUDA stream. PyTorch supplies memory and streams, nothing else.
Loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librotormap.so")
_lib = None

ROPE_PREC_FP32 = 0
ROPE_PREC_BF16 = 1
ROPE_PREC_FP8 = 2
_PREC = {"fp32": ROPE_PREC_FP32, "bf16": ROPE_PREC_BF16, "fp8": ROPE_PREC_FP8}
_STATUS = {0: "ROPE_OK", 1: "ROPE_ERR_INVALID_ARG", 2: "ROPE_ERR_INVALID_BASE", 3: "ROPE_ERR_OOM",
           4: "ROPE_ERR_CUDA", 5: "ROPE_ERR_TIMEOUT", 6: "ROPE_ERR_UNSUPPORTED"}


class RopeError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class rope_params(ctypes.Structure):
    _fields_ = [("s", ctypes.c_int32), ("m", ctypes.c_int32), ("t", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("score_mode", ctypes.c_int32), ("window_len", ctypes.c_int32), ("stride", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("bin_of_mer_host", ctypes.c_void_p)]


class rope_score_opts(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("sep", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("rescore", ctypes.c_int32), ("cand_depth", ctypes.c_int32), ("rescore_depth", ctypes.c_int32),
                ("n_ranges", ctypes.c_int32), ("reserved0", ctypes.c_int32), ("j_begin", ctypes.c_int64),
                ("j_end", ctypes.c_int64)]


# (name, argtypes, restype) of every exported function
_P, _I32, _I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
EXPORTS = {
    "rope_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "rope_last_error": ([], ctypes.c_char_p),
    "rope_dim": ([_P], _I32),
    "rope_sync_status": ([_P], ctypes.c_int),
    "rope_set_wait_limit": ([ctypes.c_double], ctypes.c_int),
    "rope_noalloc_sync_status": ([_P], ctypes.c_int),
    "rope_pack_2bit": ([_P, _I64, _P, _P], ctypes.c_int),
    "rope_mer_bins": ([_P, _P, _I64, _P, _P], ctypes.c_int),
    "rope_encode_reference": ([_P, _P, _I64, _P, _P], ctypes.c_int),
    "rope_encode_reference_dense": ([_P, _P, _I64, _P, _P], ctypes.c_int),
    "rope_index_free": ([_P], None),
    "rope_index_info": ([_P, _P, _P, _P, _P, _P], ctypes.c_int),
    "rope_window_embeddings": ([_P, _I64, _I64, _P, _P], ctypes.c_int),
    "rope_encode_reads": ([_P, _P, _P, _I64, _P, _P, _P, _P], ctypes.c_int),
    "rope_score_topk": ([_P, _P, _P, _P, _I64, _P, _P, _P, _P], ctypes.c_int),
    "rope_score_topk_noalloc": ([_P, _P, _P, _P, _I64, _P, _P, _P, _P], ctypes.c_int),
    "rope_score_dense": ([_P, _P, _P, _P, _I64, _I32, _I64, _I64, _P, _P], ctypes.c_int),
    "rope_map": ([_P, _P, _P, _I64, _P, _P, _P, _P], ctypes.c_int),
    "rope_map_strands": ([_P, _P, _P, _I64, _P, _P, _P, _P, _P], ctypes.c_int),
    "rope_pair_fidelities": ([_P, _P, _P, _I64, _P, ctypes.c_uint64, _P, _P], ctypes.c_int),
    "rope_refine": ([_P, _P, _P, _P, _I64, _P, _I32, _I32, _P, _P, _P], ctypes.c_int),
    "rope_fragment_thresholds": ([_P, ctypes.c_double, _I32, ctypes.c_uint64, _I64, _I64, _P, _P], ctypes.c_int),
    "rope_score_threshold": ([_P, _P, _I64, _P, _I64, _I64, _I64, _P, _P, _P, _P, _P], ctypes.c_int),
    "rope_reranker_create": ([_I32, _I32, ctypes.c_uint64, _P], ctypes.c_int),
    "rope_reranker_free": ([_P], None),
    "rope_reranker_get": ([_P, _P, _P], ctypes.c_int),
    "rope_reranker_set": ([_P, _P, _I32], ctypes.c_int),
    "rope_reranker_grad": ([_P, _P, _P, _P, _I64, _P, _P, _P], ctypes.c_int),
    "rope_reranker_train_step": ([_P, _P, _P, _P, _I64, ctypes.c_float, ctypes.c_float, _P, _P], ctypes.c_int),
    "rope_reranker_predict": ([_P, _P, _I64, _P, _P], ctypes.c_int),
    "rope_reranker_save": ([_P, ctypes.c_char_p], ctypes.c_int),
    "rope_reranker_load": ([_P, ctypes.c_char_p], ctypes.c_int),
    "rope_levenshtein": ([_P, _P, _P, _P, _P, _I64, _P, _P, _P], ctypes.c_int),
    "rope_rerank_features": ([_P, _P, _P, _P, _P, _P, _P, _I64, _I32, _P, _P], ctypes.c_int),
    "rope_rerank_prune": ([_P, _P, _P, _I64, _I32, _I32, _P, _P, _P, _P], ctypes.c_int),
    "rope_map_rerank": ([_P, _P, _P, _I64, _P, _P, _I32, _P, _P, _P, _P], ctypes.c_int),
    "rope_autotune_enable": ([_I32], ctypes.c_int),
    "rope_autotune_query": ([_P, _I64, _P, _P, _P, _P], ctypes.c_int),
    "rope_autotune_set": ([_P, _I64, _P, _I32, _I32], ctypes.c_int),
    "rope_ladder_lengths": ([_I32, _I32, _I32, _P, _I32], _I32),
    "rope_ladder_create": ([_P, _P, _I64, _I32, _I32, _I32, _P, _P], ctypes.c_int),
    "rope_ladder_free": ([_P], None),
    "rope_ladder_size": ([_P], _I32),
    "rope_ladder_graph_count": ([_P], _I32),
    "rope_ladder_bucket": ([_P, _I32], _P),
    "rope_ladder_map": ([_P, _P, _P, _I64, _P, _P, _P, _P, _P], ctypes.c_int),
    "rope_merge_shards_host": ([_P, _P, _I32, _I64, _I32, _I32, _I32, _P, _P], ctypes.c_int),
    "rope_profile_enable": ([_I32], ctypes.c_int),
    "rope_profile_read": ([_P, _I32, _P], ctypes.c_int),
}


def load(path: str = LIB_PATH):
    """Load librotormap.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        for name, (args, res) in EXPORTS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def _check(st: int):
    if st != 0:
        raise RopeError(st, load().rope_last_error().decode())


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t: torch.Tensor | None) -> int | None:
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device tensors must be contiguous CUDA tensors"
    return t.data_ptr()


@dataclass
class Params:
    """Encoding parameters (see ``rope_params`` in include/rotormap.h)."""
    s: int = 4
    m: int = 2
    t: int = 2
    variant: int = 1
    score_mode: int = 0
    window_len: int = 150
    stride: int = 1
    bin_map: np.ndarray | None = None

    @property
    def dim(self) -> int:
        return self.m << (2 * self.t)

    def c(self) -> rope_params:
        p = rope_params(self.s, self.m, self.t, self.variant, self.score_mode, self.window_len, self.stride, 0, None)
        if self.bin_map is not None:
            self._keep = np.ascontiguousarray(self.bin_map, dtype=np.uint16)
            p.bin_of_mer_host = self._keep.ctypes.data
        return p


def rope_dim(p: Params) -> int:
    return load().rope_dim(ctypes.byref(p.c()))


def rope_sync_status(stream=None):
    _check(load().rope_sync_status(_stream(stream)))


def rope_set_wait_limit(seconds: float):
    """Bound of every in-kernel wait of later launches (0 restores the default)."""
    _check(load().rope_set_wait_limit(float(seconds)))


def rope_noalloc_sync_status(stream=None):
    """Raises the status recorded by rope_score_topk_noalloc calls since the last read."""
    _check(load().rope_noalloc_sync_status(_stream(stream)))


def rope_pack_2bit(seq: torch.Tensor, stream=None) -> torch.Tensor:
    out = torch.empty((seq.numel() + 15) // 16, dtype=torch.int32, device=seq.device)
    _check(load().rope_pack_2bit(_ptr(seq), seq.numel(), _ptr(out), _stream(stream)))
    return out


def rope_mer_bins(p: Params, packed: torch.Tensor, length: int, stream=None) -> torch.Tensor:
    out = torch.empty(max(length - p.s + 1, 0), dtype=torch.int16, device=packed.device)
    pc = p.c()
    _check(load().rope_mer_bins(ctypes.byref(pc), _ptr(packed), length, _ptr(out), _stream(stream)))
    return out


class _CudaArray:
    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = dict(shape=(n,), typestr=typestr, data=(ptr, False), version=3)


def _device_view(ptr: int, n: int, typestr: str, dtype) -> torch.Tensor:
    t = torch.as_tensor(_CudaArray(ptr, n, typestr), device="cuda")
    return t.view(dtype) if t.dtype != dtype else t


class Index:
    """Owner of a ``rope_index`` (freed with rope_index_free), or a borrowed
    view of one that another object owns (``owner`` set; free() is a no-op)."""

    def __init__(self, handle: int, params: Params, owner=None):
        self.handle = handle
        self.params = params
        self.owner = owner

    def info(self) -> dict:
        nw, rl, ap = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        pk, inv = ctypes.c_void_p(), ctypes.c_void_p()
        _check(load().rope_index_info(self.handle, ctypes.byref(nw), ctypes.byref(rl), ctypes.byref(ap),
                                      ctypes.byref(pk), ctypes.byref(inv)))
        return dict(n_windows=nw.value, ref_len=rl.value, anchor_period=ap.value, packed=pk.value,
                    inv_norm=inv.value)

    @property
    def n_windows(self) -> int:
        return self.info()["n_windows"]

    def inv_norm(self) -> torch.Tensor:
        """Zero-copy view of the stored 1/sqrt(C_j), j < W (owned by the index)."""
        inf = self.info()
        return _device_view(inf["inv_norm"], inf["n_windows"], "<f4", torch.float32)

    def packed(self) -> torch.Tensor:
        """Zero-copy view of the 2-bit packed reference words (owned by the index)."""
        inf = self.info()
        return _device_view(inf["packed"], (inf["ref_len"] + 15) // 16, "<u4", torch.int32)

    def free(self):
        if self.handle and self.owner is None:
            load().rope_index_free(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def rope_encode_reference(p: Params, ref: torch.Tensor, stream=None) -> Index:
    h = ctypes.c_void_p()
    pc = p.c()
    _check(load().rope_encode_reference(ctypes.byref(pc), _ptr(ref), ref.numel(), ctypes.byref(h), _stream(stream)))
    return Index(h.value, p)


def rope_encode_reference_dense(p: Params, ref: torch.Tensor, stream=None) -> Index:
    """The materialised index (every window's FP32 and BF16 encoding stored)."""
    h = ctypes.c_void_p()
    pc = p.c()
    _check(load().rope_encode_reference_dense(ctypes.byref(pc), _ptr(ref), ref.numel(), ctypes.byref(h),
                                              _stream(stream)))
    return Index(h.value, p)


def rope_index_free(idx: Index):
    idx.free()


def rope_window_embeddings(idx: Index, j_begin: int, count: int, stream=None) -> torch.Tensor:
    out = torch.empty((count, 2 * idx.params.dim), dtype=torch.float32, device="cuda")
    _check(load().rope_window_embeddings(idx.handle, j_begin, count, _ptr(out), _stream(stream)))
    return out


def rope_encode_reads(p: Params, seqs: torch.Tensor, offsets: torch.Tensor, want_f32: bool = True,
                      want_bf16: bool = True, stream=None):
    """Returns (emb_f32 [n, 2D] or None, emb_bf16 [n, 2D] or None, norms [n, 1+m])."""
    n = offsets.numel() - 1
    D = p.dim
    f32 = torch.empty((n, 2 * D), dtype=torch.float32, device=seqs.device) if want_f32 else None
    bf16 = torch.empty((n, 2 * D), dtype=torch.bfloat16, device=seqs.device) if want_bf16 else None
    norms = torch.empty((n, 1 + p.m), dtype=torch.float32, device=seqs.device)
    pc = p.c()
    _check(load().rope_encode_reads(ctypes.byref(pc), _ptr(seqs), _ptr(offsets), n, _ptr(f32), _ptr(bf16),
                                    _ptr(norms), _stream(stream)))
    return f32, bf16, norms


def _opts(k, sep, precision, rescore, cand_depth, rescore_depth, n_ranges, j_begin, j_end) -> rope_score_opts:
    prec = _PREC.get(precision, precision)
    if rescore is None:
        rescore = 1 if prec in (ROPE_PREC_BF16, ROPE_PREC_FP8) else 0
    return rope_score_opts(k, sep, prec, int(rescore), cand_depth, rescore_depth, n_ranges, 0, j_begin, j_end)


def rope_score_topk(idx: Index, emb_f32: torch.Tensor, emb_bf16: torch.Tensor | None, norms: torch.Tensor, k: int = 8,
                    sep: int = 0, precision="bf16", rescore=None, cand_depth: int = 0, rescore_depth: int = 0,
                    n_ranges: int = 0, j_begin: int = 0, j_end: int = 0, out=None, stream=None):
    """Per-read top-k: (window starts int64 [n, k], fidelities float32 [n, k])."""
    n = norms.shape[0]
    if out is None:
        out = (torch.empty((n, k), dtype=torch.int64, device=norms.device),
               torch.empty((n, k), dtype=torch.float32, device=norms.device))
    o = _opts(k, sep, precision, rescore, cand_depth, rescore_depth, n_ranges, j_begin, j_end)
    _check(load().rope_score_topk(idx.handle, _ptr(emb_f32), _ptr(emb_bf16), _ptr(norms), n, ctypes.byref(o),
                                  _ptr(out[0]), _ptr(out[1]), _stream(stream)))
    return out


def rope_score_topk_noalloc(idx: Index, emb_f32: torch.Tensor, emb_bf16: torch.Tensor | None, norms: torch.Tensor,
                            out: tuple, k: int = 8, sep: int = 0, precision="bf16", rescore=None, cand_depth: int = 0,
                            rescore_depth: int = 0, n_ranges: int = 0, j_begin: int = 0, j_end: int = 0,
                            stream=None):
    """rope_score_topk without any device allocation inside the library: the
    caller passes the outputs (starts int64 [n, k], fidelities float32 [n, k])
    and the scratch comes from the library's fixed 16 MiB per-device array.
    Calls overlapping on one GPU race on that array."""
    n = norms.shape[0]
    o = _opts(k, sep, precision, rescore, cand_depth, rescore_depth, n_ranges, j_begin, j_end)
    _check(load().rope_score_topk_noalloc(idx.handle, _ptr(emb_f32), _ptr(emb_bf16), _ptr(norms), n,
                                          ctypes.byref(o), _ptr(out[0]), _ptr(out[1]), _stream(stream)))
    return out


def rope_score_dense(idx: Index, emb_f32: torch.Tensor, emb_bf16: torch.Tensor | None, norms: torch.Tensor,
                     j_begin: int, count: int, precision="fp32", stream=None) -> torch.Tensor:
    n = norms.shape[0]
    prec = _PREC.get(precision, precision)
    out = torch.full((n, count), float("nan"), dtype=torch.float32, device=norms.device)
    _check(load().rope_score_dense(idx.handle, _ptr(emb_f32), _ptr(emb_bf16), _ptr(norms), n, prec, j_begin, count,
                                   _ptr(out), _stream(stream)))
    return out


def rope_map(idx: Index, seqs: torch.Tensor, offsets: torch.Tensor, k: int = 8, sep: int = 0, precision="bf16",
             rescore=None, cand_depth: int = 0, rescore_depth: int = 0, n_ranges: int = 0, out=None, stream=None):
    """Whole path: encode the read heads and scan them; (starts [n, k], fidelities [n, k])."""
    n = offsets.numel() - 1
    if out is None:
        out = (torch.empty((n, k), dtype=torch.int64, device=seqs.device),
               torch.empty((n, k), dtype=torch.float32, device=seqs.device))
    o = _opts(k, sep, precision, rescore, cand_depth, rescore_depth, n_ranges, 0, 0)
    _check(load().rope_map(idx.handle, _ptr(seqs), _ptr(offsets), n, ctypes.byref(o), _ptr(out[0]), _ptr(out[1]),
                           _stream(stream)))
    return out


def rope_map_strands(idx: Index, seqs: torch.Tensor, offsets: torch.Tensor, k: int = 8, sep: int = 0,
                     precision="bf16", rescore=None, cand_depth: int = 0, rescore_depth: int = 0, n_ranges: int = 0,
                     out=None, stream=None):
    """Both strands: (starts [n, k], fidelities [n, k], strand int8 [n, k]: 0 forward, 1 reverse, -1 missing)."""
    n = offsets.numel() - 1
    if out is None:
        out = (torch.empty((n, k), dtype=torch.int64, device=seqs.device),
               torch.empty((n, k), dtype=torch.float32, device=seqs.device),
               torch.empty((n, k), dtype=torch.int8, device=seqs.device))
    o = _opts(k, sep, precision, rescore, cand_depth, rescore_depth, n_ranges, 0, 0)
    _check(load().rope_map_strands(idx.handle, _ptr(seqs), _ptr(offsets), n, ctypes.byref(o), _ptr(out[0]),
                                   _ptr(out[1]), _ptr(out[2]), _stream(stream)))
    return out


def rope_pair_fidelities(p: Params, seqs: torch.Tensor, offsets: torch.Tensor, errs: torch.Tensor, seed: int = 0,
                         stream=None) -> torch.Tensor:
    """§2.4: fidelity of each string's first N letters against its mutated copy at rate errs[i] (float32 [n])."""
    n = offsets.numel() - 1
    out = torch.empty((n,), dtype=torch.float32, device=seqs.device)
    e = errs.to(device=seqs.device, dtype=torch.float64).contiguous()
    pc = p.c()
    _check(load().rope_pair_fidelities(ctypes.byref(pc), _ptr(seqs), _ptr(offsets), n, _ptr(e), seed, _ptr(out),
                                       _stream(stream)))
    return out


def rope_refine(idx: Index, p: Params, seqs: torch.Tensor, offsets: torch.Tensor, cand_pos: torch.Tensor,
                radius: int, stream=None):
    """§3.4 refinement: per (read, candidate start) the best position within
    +-radius letters under the encoding p, and its fidelity:
    (positions int64 [n, n_cand], fidelities float32 [n, n_cand])."""
    n = offsets.numel() - 1
    cand_pos = cand_pos.reshape(n, -1).contiguous()
    nc = cand_pos.shape[1]
    out = (torch.empty((n, nc), dtype=torch.int64, device=seqs.device),
           torch.empty((n, nc), dtype=torch.float32, device=seqs.device))
    pc = p.c()
    _check(load().rope_refine(idx.handle, ctypes.byref(pc), _ptr(seqs), _ptr(offsets), n, _ptr(cand_pos), nc, radius,
                              _ptr(out[0]), _ptr(out[1]), _stream(stream)))
    return out


def rope_fragment_thresholds(idx: Index, err: float, n_samples: int = 8, seed: int = 0, j_begin: int = 0,
                             count: int | None = None, stream=None) -> torch.Tensor:
    """§3.4 per-window thresholds for mutation rate err (float32 [count])."""
    if count is None:
        count = idx.n_windows - j_begin
    out = torch.empty(count, dtype=torch.float32, device="cuda")
    _check(load().rope_fragment_thresholds(idx.handle, err, n_samples, seed & (2**64 - 1), j_begin, count, _ptr(out),
                                           _stream(stream)))
    return out


def rope_score_threshold(idx: Index, emb_bf16: torch.Tensor, thr: torch.Tensor, cap: int = 1 << 20,
                         j_begin: int = 0, j_end: int = 0, stream=None):
    """§3.5 multi-locus output: (reads int64, window numbers int64, scores
    float32, total count) of the pairs whose score reaches their window's
    threshold; only the first min(count, cap) pairs are returned."""
    n = emb_bf16.shape[0]
    r = torch.empty(max(cap, 1), dtype=torch.int64, device="cuda")
    w = torch.empty(max(cap, 1), dtype=torch.int64, device="cuda")
    s = torch.empty(max(cap, 1), dtype=torch.float32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    _check(load().rope_score_threshold(idx.handle, _ptr(emb_bf16), n, _ptr(thr.contiguous()), j_begin, j_end, cap,
                                       _ptr(r), _ptr(w), _ptr(s), _ptr(cnt), _stream(stream)))
    total = int(cnt.item())
    k = min(total, cap)
    return r[:k], w[:k], s[:k], total


def rope_profile_enable(max_calls: int):
    """Record [encode, scan, merge] CUDA-event times of the next max_calls calls."""
    _check(load().rope_profile_enable(max_calls))


def rope_profile_read(capacity: int) -> np.ndarray:
    """Milliseconds per recorded call: array [n_calls, 3] = (encode, scan, merge)."""
    ms = np.zeros(3 * capacity, dtype=np.float32)
    n = ctypes.c_int32()
    _check(load().rope_profile_read(ms.ctypes.data, capacity, ctypes.byref(n)))
    return ms[: 3 * n.value].reshape(n.value, 3).astype(np.float64)


def rope_merge_shards_host(wins: np.ndarray, scores: np.ndarray, k_out: int, sep: int = 0):
    """Merge per-shard top-k lists [n_shards, n_reads, k_in] (host arrays)."""
    wins = np.ascontiguousarray(wins, dtype=np.int64)
    scores = np.ascontiguousarray(scores, dtype=np.float32)
    n_shards, n_reads, k_in = wins.shape
    ow = np.empty((n_reads, k_out), dtype=np.int64)
    os_ = np.empty((n_reads, k_out), dtype=np.float32)
    _check(load().rope_merge_shards_host(wins.ctypes.data, scores.ctypes.data, n_shards, n_reads, k_in, k_out, sep,
                                         ow.ctypes.data, os_.ctypes.data))
    return ow, os_


# ---------------------------------------------------------------- length ladder

def rope_ladder_lengths(n_min: int = 100, n_max: int = 10000, steps_per_octave: int = 8) -> list[int]:
    """Window lengths floor(n_min * 2^(j/steps)) up to n_max, repeats dropped (host only)."""
    lib = load()
    n = lib.rope_ladder_lengths(n_min, n_max, steps_per_octave, None, 0)
    if n < 0:
        raise ValueError("bad ladder parameters")
    buf = (ctypes.c_int32 * max(n, 1))()
    lib.rope_ladder_lengths(n_min, n_max, steps_per_octave, buf, n)
    return list(buf[:n])


class Ladder:
    """Owner of a ``rope_ladder``: one index per window length over one packed reference."""

    def __init__(self, handle: int, params: Params, lengths: list[int]):
        self.handle = handle
        self.params = params
        self.lengths = lengths

    def bucket(self, j: int) -> Index:
        h = load().rope_ladder_bucket(self.handle, j)
        if not h:
            raise IndexError(j)
        return Index(h, dataclasses.replace(self.params, window_len=self.lengths[j]), owner=self)

    def graph_count(self) -> int:
        return load().rope_ladder_graph_count(self.handle)

    def free(self):
        if self.handle:
            load().rope_ladder_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def rope_ladder_create(p: Params, ref: torch.Tensor, n_min: int = 100, n_max: int = 10000, steps_per_octave: int = 8,
                       stream=None) -> Ladder:
    h = ctypes.c_void_p()
    pc = p.c()
    _check(load().rope_ladder_create(ctypes.byref(pc), _ptr(ref), ref.numel(), n_min, n_max, steps_per_octave,
                                     ctypes.byref(h), _stream(stream)))
    n = load().rope_ladder_size(h.value)
    lens = rope_ladder_lengths(n_min, min(n_max, ref.numel()), steps_per_octave)[:n]
    return Ladder(h.value, p, lens)


def rope_ladder_map(lad: Ladder, seqs: torch.Tensor, offsets: torch.Tensor, k: int = 8, sep: int = 0,
                    precision="bf16", rescore=None, cand_depth: int = 0, rescore_depth: int = 0, n_ranges: int = 0,
                    out=None, stream=None):
    """Reads of any length: (starts [n, k], fidelities [n, k], window length used [n] (-1: too short))."""
    n = offsets.numel() - 1
    if out is None:
        out = (torch.empty((n, k), dtype=torch.int64, device=seqs.device),
               torch.empty((n, k), dtype=torch.float32, device=seqs.device),
               torch.empty((n,), dtype=torch.int32, device=seqs.device))
    o = _opts(k, sep, precision, rescore, cand_depth, rescore_depth, n_ranges, 0, 0)
    _check(load().rope_ladder_map(lad.handle, _ptr(seqs), _ptr(offsets), n, ctypes.byref(o), _ptr(out[0]),
                                  _ptr(out[1]), _ptr(out[2]), _stream(stream)))
    return out


# ---------------------------------------------------------------- tuner

def rope_autotune_enable(enabled: bool):
    _check(load().rope_autotune_enable(1 if enabled else 0))


def rope_autotune_query(idx: Index, n_reads: int, k: int = 8, sep: int = 0, cand_depth: int = 0, precision="bf16"):
    """(tile variant, items per SM, sample ms) chosen for this shape class, or None."""
    o = _opts(k, sep, precision, None, cand_depth, 0, 0, 0, 0)
    v, it, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    st = load().rope_autotune_query(idx.handle, n_reads, ctypes.byref(o), ctypes.byref(v), ctypes.byref(it),
                                    ctypes.byref(ms))
    return (v.value, it.value, ms.value) if st == 0 else None


def rope_autotune_set(idx: Index, n_reads: int, variant: int, items_per_sm: int, k: int = 8, sep: int = 0,
                      cand_depth: int = 0, precision="bf16"):
    """Pin the scan configuration of this shape class."""
    o = _opts(k, sep, precision, None, cand_depth, 0, 0, 0, 0)
    _check(load().rope_autotune_set(idx.handle, n_reads, ctypes.byref(o), variant, items_per_sm))
