"""§2.4 scoring of correlations and the §3.4/§3.5 threshold regime on the
materialised (long-read) index, through the C ABI against the FP64 oracle.

* Pair fidelities: the mutated copies are fixed by the shared SplitMix64
  definition of the walk (each side implements it), so only the FP32
  arithmetic differs. Both encodings are FP32 direct sums within
  eps = 1e-5 of their norm (as the read-encoding parity tests hold), so the
  inner product of the unit vectors moves by at most 2 eps and the fidelity
  f = |ip|^2 by at most 4 eps sqrt(f) + 4 eps^2: the tolerance below.
* With the GPU's fidelities of 2000 random 20,000-letter strings at 4096
  complex dimensions and rates uniform in (0, 0.5), the fitting curve predicts
  the rate of strings mutated by less than 25% with an RMSE below 1% (the
  paper's printed claim, reproduced by the oracle's own pin).
* Per-window thresholds of the materialised index (the mean fidelity between
  a window and its mutated copies) against the oracle's, and the threshold
  pairs of its GEMM scan against the oracle's exhaustive set except pairs
  within the BF16 tolerance of their window's threshold.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from _parity import bf16_tol, dev

pytestmark = pytest.mark.gpu


def pair_tol(f):
    eps = 1e-5
    f = np.maximum(np.asarray(f, dtype=np.float64), 0)
    return 4 * eps * np.sqrt(f) + 4 * eps * eps + 1e-7


def strings(n, length, seed):
    ref = synth.uniform_ref(n * length, seed)
    offs = np.arange(n + 1, dtype=np.int64) * length
    return ref, offs


@pytest.mark.parametrize("pp", [dict(s=4, m=2, t=2, variant=1, N=150), dict(s=4, m=4, t=2, variant=1, N=150,
                                                                             score_mode=1),
                                dict(s=8, m=4, t=4, variant=1, N=2000), dict(s=6, m=1, t=6, variant=0, N=3000)])
def test_pair_fidelities_against_oracle(lib, pp):
    op = oracle.Params(**pp)
    n = 48
    seqs, offs = strings(n, op.N + 300, 201)
    errs = np.linspace(0.0, 0.5, n)
    p = lib.Params(s=op.s, m=op.m, t=op.t, variant=op.variant, score_mode=op.score_mode, window_len=op.N)
    got = lib.rope_pair_fidelities(p, dev(seqs), dev(offs), torch.from_numpy(errs), seed=77)
    lib.rope_sync_status()
    got = got.cpu().numpy().astype(np.float64)
    dnas = [seqs[offs[i]:offs[i + 1]] for i in range(n)]
    want = oracle.pair_fidelities(dnas, errs, op, 77)
    assert np.all(np.abs(got - want) <= pair_tol(want)), np.abs(got - want).max()
    assert abs(got[0] - 1.0) <= 1e-5  # rate 0: the copy is the string


def test_fitting_curve_from_gpu_fidelities(lib):
    """The paper's setting of the fitting curve: 20,000-letter random strings,
    4096 complex dimensions (s = t = 6, m = 1), rates uniform in (0, 0.5)."""
    n, N = 2000, 20000
    seqs, offs = strings(n, N + 2000, 211)
    errs = np.random.default_rng(212).uniform(0.0, 0.5, n)
    p = lib.Params(s=6, m=1, t=6, variant=0, window_len=N)
    fid = lib.rope_pair_fidelities(p, dev(seqs), dev(offs), torch.from_numpy(errs), seed=5)
    lib.rope_sync_status()
    fid = fid.cpu().numpy().astype(np.float64)
    curve = oracle.fitting_curve(errs, fid)
    assert np.all(np.diff(curve[1]) < 0)  # fidelity falls with the rate
    rmse = oracle.prediction_rmse(errs, fid, curve, below=0.25)
    assert rmse < 0.01, rmse


def _dense_index(lib, op, ref):
    p = lib.Params(s=op.s, m=op.m, t=op.t, variant=op.variant, window_len=op.N, stride=op.stride)
    return p, lib.rope_encode_reference_dense(p, dev(ref))


def thr_tol(f):
    return 1e-4 * np.abs(f) + 1e-6


@pytest.mark.parametrize("pp,err,ns", [(dict(s=8, m=4, t=4, N=2000, stride=125), 0.15, 8),
                                       (dict(s=4, m=2, t=2, N=150, stride=7), 0.1, 4),
                                       (dict(s=8, m=4, t=4, N=2000, stride=125), 0.0, 2)])
def test_dense_fragment_thresholds(lib, pp, err, ns):
    op = oracle.Params(variant=1, **pp)
    ref = synth.markov_ref(60_000, 0.41, 221, 0.05, 0.05)
    p, idx = _dense_index(lib, op, ref)
    W = idx.n_windows
    for j0, cnt in ((0, 30), (W - 20, 20)):
        got = lib.rope_fragment_thresholds(idx, err, ns, 4321, j0, cnt).cpu().numpy().astype(np.float64)
        lib.rope_sync_status()
        want = oracle.fragment_thresholds(ref, op, err, ns, 4321, j0, cnt)
        assert np.all(np.abs(got - want) <= thr_tol(want)), np.abs(got - want).max()
        if err == 0.0:
            assert np.allclose(got, 1.0, atol=1e-5)
    idx.free()


def test_dense_threshold_pairs(lib):
    """20 kbp reads (1% substitutions, 0.5% indels) against the paper's
    long-read encoding on a 1 Mbp reference: thresholds for a 15% mutation
    rate, every pair reaching its window's threshold, against the oracle's
    exhaustive set; the planted loci are among the pairs (the reads' edits and
    their offset from the nearest window start, at most 625 of 20,000 letters,
    stay well under the thresholds' 15%)."""
    op = oracle.Params(s=8, m=4, t=4, variant=1, N=20000, stride=1250)
    ref = synth.uniform_ref(1_000_000, 231)
    rd = synth.reads(ref, 40, seed=232, length=20000)
    p, idx = _dense_index(lib, op, ref)
    thr = lib.rope_fragment_thresholds(idx, 0.15, 8, 11)
    _, bf16, _ = lib.rope_encode_reads(p, dev(rd.seqs), dev(rd.offsets), want_f32=False)
    r, w, s, total = lib.rope_score_threshold(idx, bf16, thr)
    lib.rope_sync_status()
    r, w, s = r.cpu().numpy(), w.cpu().numpy(), s.cpu().numpy().astype(np.float64)
    assert total == len(r) and total > 0
    thr_h = thr.cpu().numpy().astype(np.float64)
    orr, ow, of = oracle.threshold_pairs(ref, rd.seqs, rd.offsets, op, thr_h)
    truth = oracle.score_pairs(ref, rd.seqs, rd.offsets, r, w * op.stride, op)
    assert np.all(np.abs(s - truth) <= bf16_tol(truth))
    got = set(zip(r.tolist(), w.tolist()))
    want = set(zip(orr.tolist(), ow.tolist()))
    assert len(got) == len(r)
    for (i, j) in got ^ want:
        f = oracle.score_pairs(ref, rd.seqs, rd.offsets, np.array([i]), np.array([j * op.stride]), op)[0]
        assert abs(f - thr_h[j]) <= bf16_tol(f), (i, j, f, thr_h[j])
    found = [np.any((r == i) & (np.abs(w * op.stride - rd.true_pos[i]) < op.N)) for i in range(rd.n)]
    assert np.mean(found) >= 0.9
    idx.free()
