"""Seeded synthetic DNA inputs (references and planted reads).

Shared by the oracle's tests and by the GPU path's tests and benchmark; holds
none of RotorMap's arithmetic. The C implementation (``synth.c``) is compiled
on first use (``build()``) into ``libsynth.so`` beside it.

Workload recipes (``WORKLOADS``) mirror the shapes of the paper's mapping tests
(§3.5: reads against a reference, top-1 locus) scaled to 150 bp reads:
uniform i.i.d. references, order-2 Markov genomes at a target GC content with
planted tandem repeats / segmental duplicates / interspersed repeat families,
and reads with substitutions and geometric-length indels.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile libsynth.so (portable flags; builds on x86_64 and aarch64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64, u64, f64, i32, p = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int32, ctypes.c_void_p
        lib.synth_uniform_ref.argtypes = [p, i64, u64]
        lib.synth_uniform_ref.restype = i64
        lib.synth_markov_ref.argtypes = [p, i64, f64, f64, f64, f64, u64]
        lib.synth_markov_ref.restype = i64
        lib.synth_reads.argtypes = [p, i64, i64, i32, f64, f64, i32, i32, f64, f64, f64, u64, p, i64, p, p, p, p, p]
        lib.synth_reads.restype = i64
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def uniform_ref(length: int, seed: int) -> np.ndarray:
    """i.i.d. uniform ACGT reference as a uint8 array of ASCII letters."""
    out = np.empty(length, dtype=np.uint8)
    _load().synth_uniform_ref(_ptr(out), length, seed)
    return out


def markov_ref(length: int, gc: float, seed: int, tandem_frac: float = 0.0, segdup_frac: float = 0.0,
               interspersed_frac: float = 0.0) -> np.ndarray:
    """Order-2 Markov genome with planted repeats, uint8 ASCII letters."""
    out = np.empty(length, dtype=np.uint8)
    _load().synth_markov_ref(_ptr(out), length, gc, tandem_frac, segdup_frac, interspersed_frac, seed)
    return out


@dataclass
class Reads:
    seqs: np.ndarray        # uint8 ASCII, concatenated
    offsets: np.ndarray     # int64 [n+1]
    true_pos: np.ndarray    # int64 [n], reference start of each read
    true_span: np.ndarray   # int32 [n], reference bases consumed
    n_edits: np.ndarray     # int32 [n], total edit length applied
    lengths: np.ndarray     # int32 [n]

    @property
    def n(self) -> int:
        return len(self.lengths)

    def read(self, i: int) -> bytes:
        return self.seqs[self.offsets[i]:self.offsets[i + 1]].tobytes()

    def subset(self, idx) -> "Reads":
        idx = np.asarray(idx, dtype=np.int64)
        parts = [self.seqs[self.offsets[i]:self.offsets[i + 1]] for i in idx]
        lens = np.array([len(p) for p in parts], dtype=np.int64)
        offs = np.zeros(len(idx) + 1, dtype=np.int64)
        offs[1:] = np.cumsum(lens)
        seqs = np.concatenate(parts) if parts else np.empty(0, np.uint8)
        return Reads(seqs, offs, self.true_pos[idx].copy(), self.true_span[idx].copy(),
                     self.n_edits[idx].copy(), self.lengths[idx].copy())


def reads(ref: np.ndarray, n: int, seed: int, length: int = 150, sub_rate: float = 0.01,
          indel_rate: float = 0.005, geom_p: float = 0.7, lognormal_sigma: float | None = None,
          len_min: int = 100, len_max: int = 10000) -> Reads:
    """Planted reads: fixed length, or lognormal (median ``length``) when
    ``lognormal_sigma`` is given, clipped to [len_min, len_max]."""
    lib = _load()
    mode = 0 if lognormal_sigma is None else 1
    cap = n * (length if mode == 0 else len_max) + 16
    seqs = np.empty(cap, dtype=np.uint8)
    offsets = np.empty(n + 1, dtype=np.int64)
    tp = np.empty(n, dtype=np.int64)
    ts = np.empty(n, dtype=np.int32)
    ne = np.empty(n, dtype=np.int32)
    ln = np.empty(n, dtype=np.int32)
    ref = np.ascontiguousarray(ref, dtype=np.uint8)
    w = lib.synth_reads(_ptr(ref), len(ref), n, mode, float(length), float(lognormal_sigma or 0.0), len_min,
                        len_max, sub_rate, indel_rate, geom_p, seed, _ptr(seqs), cap, _ptr(offsets), _ptr(tp),
                        _ptr(ts), _ptr(ne), _ptr(ln))
    if w < 0:
        raise ValueError("synth_reads failed (reference too short or capacity exceeded)")
    return Reads(seqs[:w].copy(), offsets, tp, ts, ne, ln)


def concat(parts: list[Reads]) -> Reads:
    seqs = np.concatenate([p.seqs for p in parts]) if parts else np.empty(0, np.uint8)
    offs = [0]
    for p in parts:
        offs.extend((p.offsets[1:] + offs[-1]).tolist())
    cat = lambda f, dt: np.concatenate([getattr(p, f) for p in parts]).astype(dt)
    return Reads(seqs, np.array(offs, dtype=np.int64), cat("true_pos", np.int64), cat("true_span", np.int32),
                 cat("n_edits", np.int32), cat("lengths", np.int32))


def reads_mixed_error(ref: np.ndarray, n: int, seed: int, max_rate: float = 0.15, groups: int = 10,
                      length: int = 150, sub_share: float = 2.0 / 3.0) -> Reads:
    """Reads whose error rates spread uniformly over [0, max_rate] (group g at
    rate max_rate*(g+0.5)/groups), split sub_share : 1-sub_share between
    substitutions and indel events (2:1 is the mix of 1% / 0.5%)."""
    parts = []
    for g in range(groups):
        e = max_rate * (g + 0.5) / groups
        cnt = n // groups + (1 if g < n % groups else 0)
        parts.append(reads(ref, cnt, seed=seed + 7919 * g, length=length, sub_rate=sub_share * e,
                           indel_rate=(1 - sub_share) * e))
    return concat(parts)


# Workload recipes. Sizes follow the five configurations the benchmark and the
# parity tests use; "reads" gives (count, length, sub, indel, seed).
WORKLOADS = {
    "uniform100k": dict(ref=("uniform", 100_000, 1), reads=(256, 150, 0.01, 0.005, 2)),
    "markov100M": dict(ref=("markov", 100_000_000, 3, 0.41, 0.025, 0.025, 0.0), reads=(1_000_000, 150, 0.01, 0.005, 4)),
    "markov10M_lognormal": dict(ref=("markov", 10_000_000, 5, 0.41, 0.025, 0.025, 0.0),
                                reads=(200_000, 2000, 0.032, 0.048, 6)),
    "human3G": dict(ref=("markov", 3_100_000_000, 7, 0.41, 0.0, 0.0, 0.50), reads=(100_000, 150, 0.01, 0.005, 9)),
    "maize2G": dict(ref=("markov", 2_300_000_000, 8, 0.47, 0.0, 0.0, 0.85), reads=(100_000, 150, 0.01, 0.005, 10)),
}


def make_ref(spec) -> np.ndarray:
    kind = spec[0]
    if kind == "uniform":
        _, length, seed = spec
        return uniform_ref(length, seed)
    _, length, seed, gc, tandem, segdup, inter = spec
    return markov_ref(length, gc, seed, tandem, segdup, inter)
