"""Learned candidate reranker (binding + training loop).

The scan keeps, per read, its K best candidate loci (one per bucket of width
N). A two-layer network (hidden 128, exact GELU, BF16 weight matrices, FP32
arithmetic) predicts each candidate's Levenshtein distance to the read head,
as a fraction of N, from the scan's own scores: the read's K candidate
fidelities, the candidate's fidelity, its per-band fidelities (§2.5) and its
rank. The candidates with the smallest predicted distance are kept. Labels
are exact Levenshtein distances (§1) from the library's bit-parallel DP.

Everything here marshals arguments to librotormap.so; the only host work is
building index lists (numpy) for sampling and batching.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import rotormap as rm


def n_features(K: int, m: int) -> int:
    """Feature row width: K scores, own score, m per-band fidelities, rank, 4 Hamming fidelities."""
    return K + 6 + m


class Reranker:
    """Owner of a ``rope_reranker`` (weights, AdamW state, scratch)."""

    def __init__(self, n_features: int, hidden: int = 128, seed: int = 0):
        h = ctypes.c_void_p()
        rm._check(rm.load().rope_reranker_create(n_features, hidden, seed, ctypes.byref(h)))
        self.handle = h.value
        self.F, self.H = n_features, hidden

    @property
    def n_params(self) -> int:
        return self.H * self.F + 2 * self.H + 1

    def params(self) -> tuple[np.ndarray, int]:
        """FP32 master parameters (W1 [H,F], b1 [H], w2 [H], b2) flattened, and the step count."""
        p = np.empty(self.n_params, dtype=np.float32)
        step = ctypes.c_int64()
        rm._check(rm.load().rope_reranker_get(self.handle, p.ctypes.data, ctypes.byref(step)))
        return p, step.value

    def set_params(self, p: np.ndarray, reset_optimizer: bool = True):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.n_params
        rm._check(rm.load().rope_reranker_set(self.handle, p.ctypes.data, int(reset_optimizer)))

    def grad(self, X: torch.Tensor, t: torch.Tensor, sample_idx: torch.Tensor | None = None):
        """(flat FP32 gradient [P], loss) of the batch's mean squared error."""
        B = sample_idx.numel() if sample_idx is not None else X.shape[0]
        g = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        rm._check(rm.load().rope_reranker_grad(self.handle, rm._ptr(X), rm._ptr(t), rm._ptr(sample_idx), B,
                                               rm._ptr(g), rm._ptr(loss), rm._stream()))
        return g, loss

    def train_step(self, X, t, sample_idx, lr: float = 1e-3, weight_decay: float = 0.01, loss_sum=None):
        """One AdamW step on the batch; its mean squared error is added to
        ``loss_sum`` (a device float) when given."""
        B = sample_idx.numel() if sample_idx is not None else X.shape[0]
        rm._check(rm.load().rope_reranker_train_step(self.handle, rm._ptr(X), rm._ptr(t), rm._ptr(sample_idx), B,
                                                     ctypes.c_float(lr), ctypes.c_float(weight_decay),
                                                     rm._ptr(loss_sum), rm._stream()))

    def predict(self, X: torch.Tensor) -> torch.Tensor:
        B = X.shape[0]
        y = torch.empty(B, dtype=torch.float32, device="cuda")
        rm._check(rm.load().rope_reranker_predict(self.handle, rm._ptr(X), B, rm._ptr(y), rm._stream()))
        return y

    def save(self, path: str):
        rm._check(rm.load().rope_reranker_save(self.handle, path.encode()))

    def load(self, path: str):
        rm._check(rm.load().rope_reranker_load(self.handle, path.encode()))

    def free(self):
        if self.handle:
            rm.load().rope_reranker_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def rope_levenshtein(idx: rm.Index, seqs: torch.Tensor, offsets: torch.Tensor, read_idx: torch.Tensor,
                     win_start: torch.Tensor):
    """Exact Levenshtein distance of each (read head, window) pair: (int32, float = distance / N)."""
    n = read_idx.numel()
    ld = torch.empty(n, dtype=torch.int32, device="cuda")
    frac = torch.empty(n, dtype=torch.float32, device="cuda")
    rm._check(rm.load().rope_levenshtein(idx.handle, rm._ptr(seqs), rm._ptr(offsets), rm._ptr(read_idx),
                                         rm._ptr(win_start), n, rm._ptr(ld), rm._ptr(frac), rm._stream()))
    return ld, frac


def rope_rerank_features(idx: rm.Index, seqs: torch.Tensor, offsets: torch.Tensor, emb_f32: torch.Tensor,
                         norms: torch.Tensor, cand_win: torch.Tensor, cand_score: torch.Tensor) -> torch.Tensor:
    """Feature rows [n_reads * K, K + 6 + m] of every (read, candidate)."""
    n, K = cand_win.shape
    F = n_features(K, idx.params.m)
    X = torch.empty((n * K, F), dtype=torch.float32, device="cuda")
    rm._check(rm.load().rope_rerank_features(idx.handle, rm._ptr(seqs), rm._ptr(offsets), rm._ptr(emb_f32),
                                             rm._ptr(norms), rm._ptr(cand_win), rm._ptr(cand_score), n, K,
                                             rm._ptr(X), rm._stream()))
    return X


def rope_map_rerank(idx: rm.Index, seqs: torch.Tensor, offsets: torch.Tensor, rr: Reranker | None, k: int = 16,
                    keep: int = 2, sep: int | None = None, precision="bf16"):
    """Map, then keep `keep` of the k candidates: smallest predicted distance
    (or, with rr=None, the plain score ranking). Returns (starts, fidelities,
    predicted distance / N)."""
    n = offsets.numel() - 1
    sep = idx.params.window_len if sep is None else sep
    o = rm._opts(k, sep, precision, None, 0, 0, 0, 0, 0)
    out_w = torch.empty((n, keep), dtype=torch.int64, device="cuda")
    out_s = torch.empty((n, keep), dtype=torch.float32, device="cuda")
    out_p = torch.empty((n, keep), dtype=torch.float32, device="cuda")
    rm._check(rm.load().rope_map_rerank(idx.handle, rm._ptr(seqs), rm._ptr(offsets), n, ctypes.byref(o),
                                        rr.handle if rr is not None else None, keep, rm._ptr(out_w),
                                        rm._ptr(out_s), rm._ptr(out_p), rm._stream()))
    return out_w, out_s, out_p


def training_set(idx: rm.Index, seqs: torch.Tensor, offsets: torch.Tensor, k: int = 16, precision="bf16"):
    """Candidates of every read (k per read, one per bucket of width N), their
    features, and exact distance labels. Returns (X [n*k, F], t [n*k] = LD/N,
    valid sample indices (int64, device), candidate starts [n, k])."""
    p = idx.params
    f32, bf16, norms = rm.rope_encode_reads(p, seqs, offsets)
    win, score = rm.rope_score_topk(idx, f32, bf16, norms, k=k, sep=p.window_len, precision=precision)
    X = rope_rerank_features(idx, seqs, offsets, f32, norms, win, score)
    w_h = win.reshape(-1).cpu().numpy()
    vi = np.nonzero(w_h >= 0)[0].astype(np.int64)
    read_idx = torch.from_numpy(vi // k).cuda()
    win_start = torch.from_numpy(w_h[vi]).cuda()
    _, frac = rope_levenshtein(idx, seqs, offsets, read_idx, win_start)
    t_h = np.zeros(w_h.size, dtype=np.float32)  # rows of missing candidates are never sampled
    t_h[vi] = frac.cpu().numpy()
    return X, torch.from_numpy(t_h).cuda(), torch.from_numpy(vi).cuda(), win


def train(rr: Reranker, X: torch.Tensor, t: torch.Tensor, valid: torch.Tensor, epochs: int = 5, batch: int = 4096,
          lr: float = 1e-3, weight_decay: float = 0.01, seed: int = 0) -> list[float]:
    """AdamW epochs over the valid samples in a seeded random order; returns
    the mean training loss of each epoch."""
    rng = np.random.default_rng(seed)
    v_h = valid.cpu().numpy()
    losses = []
    loss_sum = torch.empty(1, dtype=torch.float32, device="cuda")
    for _ in range(epochs):
        order = torch.from_numpy(rng.permutation(v_h)).cuda()
        loss_sum.zero_()
        n_batches = 0
        for b0 in range(0, order.numel(), batch):
            rr.train_step(X, t, order[b0:b0 + batch], lr, weight_decay, loss_sum)
            n_batches += 1
        losses.append(float(loss_sum.item()) / max(n_batches, 1))
    return losses
