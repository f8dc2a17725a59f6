"""RotorMap FP64 CPU oracle — TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously correct CPU implementation of what the GPU path
computes, written from the paper (see ``rotormap_oracle.c`` for the passage each
function follows). It shares no code with the CUDA library and neither imports
the other. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
against closed forms, invariants, values the paper prints, or brute force —
including the refinement (exact reads found, range clipping, ties, the §3.4
one-letter relation), the threshold regime (published SplitMix64 outputs,
mutation rate and split, the edit bound, identity at rate 0, agreement with
the exhaustive top-k) and the fitting curve (the paper's printed RMSE) —
except the reranker network (``mlp``), which is pinned by finite differences
only; it is marked there.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rotormap_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc + OpenMP (portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-std=c11", "-fopenmp", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64, i32, f64, p = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        sig = {
            "oracle_base": ([i32], i32),
            "oracle_pack_2bit": ([p, i64, p], i64),
            "oracle_default_bin_map": ([i32, i32, p], None),
            "oracle_mer_bins": ([p, i64, i32, p, p], i32),
            "oracle_factor": ([i32, i32, i32, p, p], None),
            "oracle_embed": ([p, i32, i32, i32, i32, i32, p, p, p], i32),
            "oracle_embed_matrix_form": ([p, i32, i32, i32, i32, i32, p, p, p], i32),
            "oracle_fidelity": ([p, p, p, p, i32], f64),
            "oracle_fidelity_per_band": ([p, p, p, p, i32, i32], f64),
            "oracle_hamming_fingerprint_fidelity": ([p, p, i32], f64),
            "oracle_n_windows": ([i64, i32, i32], i64),
            "oracle_windows_direct": ([p, i64, i32, i32, i64, i64, i32, i32, i32, i32, p, p, p], i32),
            "oracle_windows_recurrence": ([p, i64, i32, i64, i64, i32, i32, i32, i32, p, p, p], i32),
            "oracle_ip_recurrence": ([p, i64, i32, i64, i64, i32, i32, i32, i32, p, p, p, p, p], i32),
            "oracle_score_topk": ([p, i64, p, p, i64, i32, i32, i64, i64, i32, i32, i32, i32, p, i32, i32, i32, i32,
                                   p, p], i32),
            "oracle_score_pairs": ([p, i64, p, p, p, p, i64, i32, i32, i32, i32, i32, p, i32, i32, p], i32),
            "oracle_levenshtein": ([p, i32, p, i32], i32),
            "oracle_levenshtein_pairs": ([p, i64, p, p, p, p, i64, i32, i32, p], i32),
            "oracle_max_threads": ([], i32),
            "oracle_mlp_forward": ([p, p, p, f64, i32, i32, p, i64, p], None),
            "oracle_mlp_grad": ([p, p, p, f64, i32, i32, p, p, i64, p, p, p, p], f64),
            "oracle_adamw": ([p, p, p, p, i64, i64, f64, f64, f64, f64, f64], None),
            "oracle_splitmix64": ([ctypes.c_uint64, ctypes.c_uint64], ctypes.c_uint64),
            "oracle_mutate": ([p, i64, i64, i32, f64, ctypes.c_uint64, ctypes.c_uint64, p, p], i32),
            "oracle_fragment_thresholds": ([p, i64, i32, i32, i64, i64, i32, i32, i32, i32, p, i32, f64, i32,
                                            ctypes.c_uint64, i32, p], i32),
            "oracle_threshold_pairs": ([p, i64, p, p, i64, i32, i32, i64, i64, i32, i32, i32, i32, p, i32, p, i64,
                                        p, p, p], i64),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def _u8(x) -> np.ndarray:
    if isinstance(x, (bytes, bytearray)):
        return np.frombuffer(bytes(x), dtype=np.uint8).copy()
    if isinstance(x, str):
        return np.frombuffer(x.encode(), dtype=np.uint8).copy()
    return np.ascontiguousarray(x, dtype=np.uint8)


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


class Params:
    """(s, m, t, variant) of the encoding, window length N and stride."""

    def __init__(self, s=4, m=2, t=2, variant=1, N=150, stride=1, score_mode=0, bin_map=None):
        self.s, self.m, self.t, self.variant = s, m, t, variant
        self.N, self.stride, self.score_mode = N, stride, score_mode
        self.bin_map = default_bin_map(s, t) if bin_map is None else np.ascontiguousarray(bin_map, np.uint16)

    @property
    def dim(self) -> int:
        """complex dimension m * 4^t"""
        return self.m << (2 * self.t)


# ---------------------------------------------------------------- primitives

def base(c: str) -> int:
    return _load().oracle_base(ord(c))


def pack_2bit(seq) -> np.ndarray:
    seq = _u8(seq)
    out = np.zeros((len(seq) + 15) // 16, dtype=np.uint32)
    bad = _load().oracle_pack_2bit(_p(seq), len(seq), _p(out))
    if bad >= 0:
        raise ValueError(f"invalid letter at {bad}")
    return out


def default_bin_map(s: int, t: int) -> np.ndarray:
    out = np.empty(1 << (2 * s), dtype=np.uint16)
    _load().oracle_default_bin_map(s, t, _p(out))
    return out


def mer_bins(seq, s: int, bin_map: np.ndarray) -> np.ndarray:
    seq = _u8(seq)
    out = np.empty(max(len(seq) - s + 1, 0), dtype=np.int32)
    if _load().oracle_mer_bins(_p(seq), len(seq), s, _p(np.ascontiguousarray(bin_map, np.uint16)), _p(out)) != 0:
        raise ValueError("invalid letter")
    return out


def factor(m: int, variant: int, k: int) -> tuple[int, int]:
    a, q = ctypes.c_int64(), ctypes.c_int64()
    _load().oracle_factor(m, variant, k, ctypes.byref(a), ctypes.byref(q))
    return a.value, q.value


def embed(seq, p: Params, N: int | None = None, matrix_form: bool = False) -> np.ndarray:
    """Unnormalised RoPE vector of the first N letters (complex128, band-major)."""
    seq = _u8(seq)
    N = p.N if N is None else N
    if len(seq) < N:
        raise ValueError("sequence shorter than N")
    re = np.empty(p.dim)
    im = np.empty(p.dim)
    fn = _load().oracle_embed_matrix_form if matrix_form else _load().oracle_embed
    if fn(_p(seq), N, p.s, p.m, p.t, p.variant, _p(p.bin_map), _p(re), _p(im)) != 0:
        raise ValueError("invalid letter")
    return re + 1j * im


def fidelity(x: np.ndarray, y: np.ndarray) -> float:
    xr, xi = np.ascontiguousarray(x.real), np.ascontiguousarray(x.imag)
    yr, yi = np.ascontiguousarray(y.real), np.ascontiguousarray(y.imag)
    return _load().oracle_fidelity(_p(xr), _p(xi), _p(yr), _p(yi), len(x))


def fidelity_per_band(x: np.ndarray, y: np.ndarray, m: int) -> float:
    xr, xi = np.ascontiguousarray(x.real), np.ascontiguousarray(x.imag)
    yr, yi = np.ascontiguousarray(y.real), np.ascontiguousarray(y.imag)
    return _load().oracle_fidelity_per_band(_p(xr), _p(xi), _p(yr), _p(yi), m, len(x) // m)


def hamming_fingerprint_fidelity(S, T) -> float:
    S, T = _u8(S), _u8(T)
    assert len(S) == len(T)
    return _load().oracle_hamming_fingerprint_fidelity(_p(S), _p(T), len(S))


def n_windows(L: int, N: int, stride: int) -> int:
    return _load().oracle_n_windows(L, N, stride)


def windows_direct(ref, p: Params, j0: int, count: int) -> np.ndarray:
    ref = _u8(ref)
    re = np.empty((count, p.dim))
    im = np.empty((count, p.dim))
    if _load().oracle_windows_direct(_p(ref), len(ref), p.N, p.stride, j0, count, p.s, p.m, p.t, p.variant,
                                     _p(p.bin_map), _p(re), _p(im)) != 0:
        raise ValueError("window out of range or invalid letter")
    return re + 1j * im


def windows_recurrence(ref, p: Params, w0: int, count: int) -> np.ndarray:
    ref = _u8(ref)
    re = np.empty((count, p.dim))
    im = np.empty((count, p.dim))
    if _load().oracle_windows_recurrence(_p(ref), len(ref), p.N, w0, count, p.s, p.m, p.t, p.variant,
                                         _p(p.bin_map), _p(re), _p(im)) != 0:
        raise ValueError("window out of range or invalid letter")
    return re + 1j * im


def ip_recurrence(ref, p: Params, x: np.ndarray, w0: int, count: int) -> np.ndarray:
    ref = _u8(ref)
    xr, xi = np.ascontiguousarray(x.real), np.ascontiguousarray(x.imag)
    outr, outi = np.empty(count), np.empty(count)
    if _load().oracle_ip_recurrence(_p(ref), len(ref), p.N, w0, count, p.s, p.m, p.t, p.variant, _p(p.bin_map),
                                    _p(xr), _p(xi), _p(outr), _p(outi)) != 0:
        raise ValueError("window out of range or invalid letter")
    return outr + 1j * outi


def score_topk(ref, seqs, offsets, p: Params, k: int = 8, sep: int = 0, j_begin: int = 0, j_end: int | None = None,
               n_threads: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Exhaustive FP64 top-k: (window starts int64 [n,k], scores float64 [n,k])."""
    ref, seqs = _u8(ref), _u8(seqs)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    n = len(offsets) - 1
    if j_end is None:
        j_end = n_windows(len(ref), p.N, p.stride)
    out_w = np.empty((n, k), dtype=np.int64)
    out_s = np.empty((n, k), dtype=np.float64)
    rc = _load().oracle_score_topk(_p(ref), len(ref), _p(seqs), _p(offsets), n, p.N, p.stride, j_begin, j_end, p.s,
                                   p.m, p.t, p.variant, _p(p.bin_map), p.score_mode, k, sep, n_threads, _p(out_w),
                                   _p(out_s))
    if rc != 0:
        raise ValueError(f"oracle_score_topk failed ({rc})")
    return out_w, out_s


def score_pairs(ref, seqs, offsets, read_idx, win_start, p: Params, n_threads: int = 0) -> np.ndarray:
    ref, seqs = _u8(ref), _u8(seqs)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    ri = np.ascontiguousarray(read_idx, dtype=np.int64)
    ws = np.ascontiguousarray(win_start, dtype=np.int64)
    out = np.empty(len(ri))
    if _load().oracle_score_pairs(_p(ref), len(ref), _p(seqs), _p(offsets), _p(ri), _p(ws), len(ri), p.N, p.s, p.m,
                                  p.t, p.variant, _p(p.bin_map), p.score_mode, n_threads, _p(out)) != 0:
        raise ValueError("oracle_score_pairs failed")
    return out


def levenshtein(a, b) -> int:
    a, b = _u8(a), _u8(b)
    return _load().oracle_levenshtein(_p(a), len(a), _p(b), len(b))


def levenshtein_pairs(ref, seqs, offsets, read_idx, win_start, N: int, n_threads: int = 0) -> np.ndarray:
    ref, seqs = _u8(ref), _u8(seqs)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    ri = np.ascontiguousarray(read_idx, dtype=np.int64)
    ws = np.ascontiguousarray(win_start, dtype=np.int64)
    out = np.empty(len(ri), dtype=np.int32)
    if _load().oracle_levenshtein_pairs(_p(ref), len(ref), _p(seqs), _p(offsets), _p(ri), _p(ws), len(ri), N,
                                        n_threads, _p(out)) != 0:
        raise ValueError("oracle_levenshtein_pairs failed")
    return out


def max_threads() -> int:
    return _load().oracle_max_threads()


# ------------------------------------------------------------ reranker network

class MLP:
    """FP64 reference of the reranker network: y = w2 . GELU(W1 x + b1) + b2."""

    def __init__(self, W1, b1, w2, b2):
        self.W1 = np.ascontiguousarray(W1, dtype=np.float64)
        self.b1 = np.ascontiguousarray(b1, dtype=np.float64)
        self.w2 = np.ascontiguousarray(w2, dtype=np.float64)
        self.b2 = float(b2)

    @property
    def shape(self):
        return self.W1.shape  # (H, F)

    def forward(self, X) -> np.ndarray:
        X = np.ascontiguousarray(X, dtype=np.float64)
        H, F = self.shape
        y = np.empty(len(X))
        _load().oracle_mlp_forward(_p(self.W1), _p(self.b1), _p(self.w2), self.b2, F, H, _p(X), len(X), _p(y))
        return y

    def grad(self, X, t):
        """(loss, dW1, db1, dw2, db2) of the mean squared error."""
        X = np.ascontiguousarray(X, dtype=np.float64)
        t = np.ascontiguousarray(t, dtype=np.float64)
        H, F = self.shape
        gW1, gb1, gw2 = np.empty((H, F)), np.empty(H), np.empty(H)
        gb2 = ctypes.c_double()
        loss = _load().oracle_mlp_grad(_p(self.W1), _p(self.b1), _p(self.w2), self.b2, F, H, _p(X), _p(t), len(X),
                                       _p(gW1), _p(gb1), _p(gw2), ctypes.byref(gb2))
        return loss, gW1, gb1, gw2, gb2.value


def adamw(p, g, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.01):
    """In-place FP64 AdamW step on flat float64 arrays p, m, v with gradient g."""
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = np.ascontiguousarray(g, dtype=np.float64)
    _load().oracle_adamw(_p(p), _p(g), _p(m), _p(v), len(p), step, lr, beta1, beta2, eps, wd)


# ------------------------------------------------------------ reranker features

RERANK_SHIFT = 4  # largest letter shift of the shifted Hamming feature


def rerank_features(ref, seqs, offsets, cand_win, cand_score, p: Params) -> np.ndarray:
    """Feature rows [n*K, K + 6 + m] of the learned reranker for each read's K
    candidates, straight from the definitions (small inputs only):

      [0, K)      the read's K candidate scores as given (0 where missing)
      K           the candidate's own score as given
      K+1 .. K+m  the fidelity of band k alone (§2.4 restricted to band k, §2.5)
                  between the read head and the window, FP64 direct sums
      K+1+m       rank / K
      K+2+m       Hamming fingerprint fidelity ((n - d)/n)^2 (§1) of the read
                  head against the window
      K+3+m       its maximum over the windows starting -4..4 letters away
                  (letters outside the reference count as mismatches)
      K+4+m,K+5+m the same fidelity of the head's first floor(N/2) letters and
                  of the remaining letters against the window's

    Rows of missing candidates (start -1) are zero. The network these rows
    feed has no counterpart in the paper; the fidelities it is built from do.
    """
    ref = _u8(ref)
    seqs = _u8(seqs)
    cand_win = np.asarray(cand_win)
    cand_score = np.asarray(cand_score, dtype=np.float64)
    n, K = cand_win.shape
    m, N, nb = p.m, p.N, p.dim // p.m
    F = K + 6 + m
    L = len(ref)
    X = np.zeros((n * K, F))
    for r in range(n):
        head = seqs[offsets[r]:offsets[r] + N]
        x = embed(head, p)
        for c in range(K):
            w = int(cand_win[r, c])
            if w < 0:
                continue
            row = X[r * K + c]
            for f in range(K):
                row[f] = cand_score[r, f] if cand_win[r, f] >= 0 else 0.0
            row[K] = cand_score[r, c]
            y = embed(ref[w:w + N], p)
            for k in range(m):
                row[K + 1 + k] = fidelity(x[k * nb:(k + 1) * nb], y[k * nb:(k + 1) * nb])
            row[K + 1 + m] = c / K

            def window(start):
                out = np.full(N, ord("N"), dtype=np.uint8)
                lo, hi = max(start, 0), min(start + N, L)
                if hi > lo:
                    out[lo - start:hi - start] = ref[lo:hi]
                return out

            win = window(w)
            row[K + 2 + m] = hamming_fingerprint_fidelity(head, win)
            row[K + 3 + m] = max(hamming_fingerprint_fidelity(head, window(w + d))
                                 for d in range(-RERANK_SHIFT, RERANK_SHIFT + 1))
            n1 = N // 2
            row[K + 4 + m] = hamming_fingerprint_fidelity(head[:n1], win[:n1])
            row[K + 5 + m] = hamming_fingerprint_fidelity(head[n1:], win[n1:])
    return X


# ------------------------------------------------------------ both strands

_COMPLEMENT = np.arange(256, dtype=np.uint8)
for _a, _b in (("A", "T"), ("C", "G"), ("a", "t"), ("c", "g")):
    _COMPLEMENT[ord(_a)], _COMPLEMENT[ord(_b)] = ord(_b), ord(_a)


def reverse_complement(seq) -> np.ndarray:
    """The other strand of a DNA string read 5'->3': letters reversed, A<->T, C<->G."""
    return _COMPLEMENT[_u8(seq)[::-1]].copy()


def score_topk_strands(ref, seqs, offsets, p: Params, k: int = 8, sep: int = 0):
    """Top-k over both strands (§3.5 maps reads in both directions): each read
    by its head and by the head of its reverse complement, both against the
    forward reference, merged by (score descending, forward first, start
    ascending). Returns (starts, scores, strand 0/1, -1 where missing)."""
    seqs = _u8(seqs)
    offsets = np.asarray(offsets, dtype=np.int64)
    n = len(offsets) - 1
    rc = np.concatenate([reverse_complement(seqs[offsets[i]:offsets[i + 1]]) for i in range(n)]) if n else seqs
    wf, sf = score_topk(ref, seqs, offsets, p, k=k, sep=sep)
    wr, sr = score_topk(ref, rc, offsets, p, k=k, sep=sep)
    out_w = np.full((n, k), -1, dtype=np.int64)
    out_s = np.full((n, k), -np.inf)
    out_t = np.full((n, k), -1, dtype=np.int8)
    for i in range(n):
        cands = [(-sf[i, j], 0, wf[i, j]) for j in range(k) if wf[i, j] >= 0]
        cands += [(-sr[i, j], 1, wr[i, j]) for j in range(k) if wr[i, j] >= 0]
        cands.sort()
        for j, (ns, t, w) in enumerate(cands[:k]):
            out_w[i, j], out_s[i, j], out_t[i, j] = w, -ns, t
    return out_w, out_s, out_t


# ------------------------------------------------------------ refinement

def refine(ref, seqs, offsets, cand_pos, radius: int, p: Params, n_threads: int = 0):
    """§3.4, increasing the accuracy: around each candidate start c the window
    of length p.N is slid one letter at a time over [c - radius, c + radius]
    (clipped to [0, L - N]) and each position is scored against the read head
    with the encoding p, here by direct FP64 embedding of every window (the
    definition the paper's O(1) update reproduces). Per (read, candidate):
    the position of the highest fidelity (ties: the lower position) and that
    fidelity; (-1, -inf) for a candidate < 0; a candidate past the last window
    start counts as the last. Also returns every scored
    (read, position, fidelity) triple, for checks of near ties."""
    ref = _u8(ref)
    cand_pos = np.asarray(cand_pos, dtype=np.int64)
    n, nc = cand_pos.shape
    last = len(ref) - p.N
    ri, pos, owner = [], [], []
    for i in range(n):
        for c in range(nc):
            x = int(cand_pos[i, c])
            if x < 0 or last < 0:
                continue
            x = min(x, last)  # a start past the last window counts as the last
            lo, hi = max(0, x - radius), min(last, x + radius)
            for q in range(lo, hi + 1):
                ri.append(i)
                pos.append(q)
                owner.append(i * nc + c)
    out_p = np.full((n, nc), -1, dtype=np.int64)
    out_f = np.full((n, nc), -np.inf)
    if not ri:
        return out_p, out_f, (np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0))
    ri, pos, owner = np.array(ri), np.array(pos), np.array(owner)
    fid = score_pairs(ref, seqs, offsets, ri, pos, p, n_threads=n_threads)
    for o, q, f in zip(owner, pos, fid):
        i, c = divmod(int(o), nc)
        if f > out_f[i, c]:  # positions arrive in increasing order: ties keep the lower one
            out_p[i, c], out_f[i, c] = q, f
    return out_p, out_f, (owner, pos, fid)


# ------------------------------------------------------------ threshold regime

def splitmix64(seed: int, i: int) -> int:
    """The i-th output (0-based) of SplitMix64 started at state ``seed``."""
    return int(_load().oracle_splitmix64(seed & (2**64 - 1), i))


def mutate(ref, start: int, N: int, err: float, seed: int, stream: int):
    """N letters of a mutated copy of ref from ``start`` (see
    ``oracle_mutate``): (letters uint8, (walked, deletions, insertions,
    substitutions))."""
    ref = _u8(ref)
    out = np.empty(N, dtype=np.uint8)
    counts = np.zeros(4, dtype=np.int64)
    if _load().oracle_mutate(_p(ref), len(ref), start, N, err, seed & (2**64 - 1), stream, _p(out), _p(counts)) != 0:
        raise ValueError("invalid letter")
    return out, tuple(int(c) for c in counts)


def fragment_thresholds(ref, p: Params, err: float, n_samples: int, seed: int, j0: int = 0, count: int | None = None,
                        n_threads: int = 0) -> np.ndarray:
    """§3.4: per window, the mean fidelity against n_samples mutated copies
    at rate err (its cutting threshold for that mutation rate)."""
    ref = _u8(ref)
    if count is None:
        count = n_windows(len(ref), p.N, p.stride) - j0
    out = np.empty(count)
    if _load().oracle_fragment_thresholds(_p(ref), len(ref), p.N, p.stride, j0, count, p.s, p.m, p.t, p.variant,
                                          _p(p.bin_map), p.score_mode, err, n_samples, seed & (2**64 - 1),
                                          n_threads, _p(out)) != 0:
        raise ValueError("oracle_fragment_thresholds failed")
    return out


def threshold_pairs(ref, seqs, offsets, p: Params, thr: np.ndarray, j_begin: int = 0, cap: int = 1 << 20):
    """§3.5 multi-locus output: every (read, window) with fidelity >= the
    window's threshold thr[j - j_begin] over windows [j_begin, j_begin +
    len(thr)), exhaustive FP64: (reads int64, windows int64, fidelities)."""
    ref, seqs = _u8(ref), _u8(seqs)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    thr = np.ascontiguousarray(thr, dtype=np.float64)
    n = len(offsets) - 1
    r = np.empty(cap, dtype=np.int64)
    w = np.empty(cap, dtype=np.int64)
    f = np.empty(cap)
    got = _load().oracle_threshold_pairs(_p(ref), len(ref), _p(seqs), _p(offsets), n, p.N, p.stride, j_begin,
                                         j_begin + len(thr), p.s, p.m, p.t, p.variant, _p(p.bin_map), p.score_mode,
                                         _p(thr), cap, _p(r), _p(w), _p(f))
    if got < 0 or got > cap:
        raise ValueError("oracle_threshold_pairs failed or exceeded cap")
    return r[:got], w[:got], f[:got]


# ------------------------------------------------------------ fitting curve (§2.4 scoring of correlations)

def pair_fidelities(dnas, errs, p: Params, seed: int, N: int | None = None) -> np.ndarray:
    """§2.4: for each random string dnas[i] (at least N + slack letters), the
    fidelity between the encoding of its first N letters and that of its
    mutated copy at rate errs[i] (``mutate``, stream i)."""
    N = p.N if N is None else N
    out = np.empty(len(dnas))
    for i, (d, e) in enumerate(zip(dnas, errs)):
        d = _u8(d)
        mut, _ = mutate(d, 0, N, float(e), seed, i)
        x, y = embed(d, p, N), embed(mut, p, N)
        out[i] = fidelity(x, y) if p.score_mode == 0 else fidelity_per_band(x, y, p.m)
    return out


def fitting_curve(errs, fids, n_bins: int = 20, lo: float = 0.0, hi: float = 0.5):
    """§2.4 step 2: the expected fidelity at evenly spaced mutation rates (the
    mean fidelity of the samples in each of n_bins equal bins of (lo, hi)),
    connected piecewise linearly. Returns (bin centres, mean fidelities)."""
    errs, fids = np.asarray(errs, dtype=np.float64), np.asarray(fids, dtype=np.float64)
    edges = np.linspace(lo, hi, n_bins + 1)
    centres = (edges[:-1] + edges[1:]) / 2
    means = np.array([fids[(errs >= a) & (errs < b)].mean() for a, b in zip(edges[:-1], edges[1:])])
    return centres, means


def predict_err(fids, curve) -> np.ndarray:
    """The mutation rate read off the fitting curve at each observed fidelity
    (the curve is decreasing in the rate, so it is inverted by interpolation)."""
    centres, means = curve
    order = np.argsort(means)
    return np.interp(np.asarray(fids, dtype=np.float64), means[order], centres[order])


def prediction_rmse(errs, fids, curve, below: float = 1.0) -> float:
    """§2.4 step 3: root mean square of (predicted - true) mutation rate over
    the samples whose true rate is below ``below``."""
    errs = np.asarray(errs, dtype=np.float64)
    sel = errs < below
    d = predict_err(np.asarray(fids)[sel], curve) - errs[sel]
    return float(np.sqrt(np.mean(d * d)))
