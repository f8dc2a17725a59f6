"""Threshold regime through the C ABI against the FP64 oracle: per-window
thresholds for a mutation rate (§3.4; the mutated copies are fixed by the
shared SplitMix64 definition, so only the FP32 arithmetic differs), and the
multi-locus output of every pair reaching its window's threshold (§3.5)."""
import numpy as np
import pytest

import oracle
import synth
from _parity import bf16_tol, dev

pytestmark = pytest.mark.gpu


def thr_tol(f):
    # means of fidelities from FP32 direct sums of <= N unit phases (relative
    # error <= N * 2^-24 ~ 1e-5 per sum, a few sums per fidelity)
    return 1e-4 * np.abs(f) + 1e-6


def gparams(lib, op):
    return lib.Params(s=op.s, m=op.m, t=op.t, variant=op.variant, score_mode=op.score_mode, window_len=op.N,
                      stride=op.stride)


@pytest.mark.parametrize("pp,err,ns", [(dict(), 0.0, 4), (dict(), 0.1, 8), (dict(), 0.3, 1),
                                       (dict(m=4), 0.15, 32), (dict(stride=3, score_mode=1), 0.2, 2),
                                       (dict(s=3, m=2, t=2, variant=0, N=64), 0.25, 16)])
def test_fragment_thresholds_against_oracle(lib, pp, err, ns):
    ref = synth.markov_ref(30_000, 0.41, 161, 0.05, 0.05)
    kw = dict(s=4, m=2, t=2, variant=1, N=150, stride=1)
    kw.update(pp)
    op = oracle.Params(**kw)
    idx = lib.rope_encode_reference(gparams(lib, op), dev(ref))
    j0, cnt = 40, 300
    got = lib.rope_fragment_thresholds(idx, err, ns, 12345, j0, cnt).cpu().numpy().astype(np.float64)
    lib.rope_sync_status()
    want = oracle.fragment_thresholds(ref, op, err, ns, 12345, j0, cnt)
    assert np.all(np.abs(got - want) <= thr_tol(want)), np.abs(got - want).max()
    if err == 0.0:
        assert np.allclose(got, 1.0, atol=1e-5)
    idx.free()


def test_fragment_thresholds_last_windows(lib):
    """Copies of the last windows walk past the reference end (read as A)."""
    ref = synth.uniform_ref(5000, 171)
    op = oracle.Params(N=150)
    idx = lib.rope_encode_reference(gparams(lib, op), dev(ref))
    W = idx.n_windows
    got = lib.rope_fragment_thresholds(idx, 0.4, 8, 9, W - 50, 50).cpu().numpy().astype(np.float64)
    lib.rope_sync_status()
    want = oracle.fragment_thresholds(ref, op, 0.4, 8, 9, W - 50, 50)
    assert np.all(np.abs(got - want) <= thr_tol(want))
    idx.free()


@pytest.mark.parametrize("pp", [dict(), dict(m=4), dict(stride=8, N=400)])
def test_threshold_pairs_against_oracle(lib, pp):
    kw = dict(s=4, m=2, t=2, variant=1, N=150, stride=1)
    kw.update(pp)
    op = oracle.Params(**kw)
    ref = synth.markov_ref(30_000, 0.41, 181, 0.05, 0.05)
    rd = synth.reads(ref, 20, seed=182, length=op.N)
    p = gparams(lib, op)
    idx = lib.rope_encode_reference(p, dev(ref))
    thr = lib.rope_fragment_thresholds(idx, 0.15, 8, 7)
    _, bf16, _ = lib.rope_encode_reads(p, dev(rd.seqs), dev(rd.offsets), want_f32=False)
    r, w, s, total = lib.rope_score_threshold(idx, bf16, thr)
    lib.rope_sync_status()
    r, w, s = r.cpu().numpy(), w.cpu().numpy(), s.cpu().numpy().astype(np.float64)
    assert total == len(r) and total > 0
    thr_h = thr.cpu().numpy().astype(np.float64)
    orr, ow, of = oracle.threshold_pairs(ref, rd.seqs, rd.offsets, op, thr_h)
    # reported scores are the oracle's fidelities within the BF16 tolerance
    truth = oracle.score_pairs(ref, rd.seqs, rd.offsets, r, w * op.stride, op)
    assert np.all(np.abs(s - truth) <= bf16_tol(truth))
    # the sets agree except for pairs within the tolerance of their threshold
    got = set(zip(r.tolist(), w.tolist()))
    want = set(zip(orr.tolist(), ow.tolist()))
    assert len(got) == len(r)  # no pair twice
    for (i, j) in got ^ want:
        f = oracle.score_pairs(ref, rd.seqs, rd.offsets, np.array([i]), np.array([j * op.stride]), op)[0]
        assert abs(f - thr_h[j]) <= bf16_tol(f), (i, j, f, thr_h[j])
    # planted loci are found (reads at 1.5% error against thresholds for 15%)
    found = [np.any((r == i) & (np.abs(w * op.stride - rd.true_pos[i]) <= op.stride + 2)) for i in range(rd.n)]
    assert np.mean(found) >= 0.95
    idx.free()


def test_threshold_cap_and_range(lib):
    ref = synth.uniform_ref(20_000, 191)
    rd = synth.reads(ref, 12, seed=192)
    op = oracle.Params(N=150)
    p = gparams(lib, op)
    idx = lib.rope_encode_reference(p, dev(ref))
    W = idx.n_windows
    _, bf16, _ = lib.rope_encode_reads(p, dev(rd.seqs), dev(rd.offsets), want_f32=False)
    import torch

    low = torch.full((W,), 0.05, dtype=torch.float32, device="cuda")
    r, w, s, total = lib.rope_score_threshold(idx, bf16, low)
    rc, wc, sc, total_c = lib.rope_score_threshold(idx, bf16, low, cap=100)
    lib.rope_sync_status()
    assert total_c == total > 100 and len(rc) == 100
    assert set(zip(rc.cpu().tolist(), wc.cpu().tolist())) <= set(zip(r.cpu().tolist(), w.cpu().tolist()))
    # a window range keeps only its windows; a threshold above 1 keeps nothing
    r2, w2, _, _ = lib.rope_score_threshold(idx, bf16, low, j_begin=1000, j_end=3000)
    assert np.all((w2.cpu().numpy() >= 1000) & (w2.cpu().numpy() < 3000))
    assert set(zip(r2.cpu().tolist(), w2.cpu().tolist())) == {(a, b) for a, b in zip(r.cpu().tolist(), w.cpu().tolist())
                                                              if 1000 <= b < 3000}
    _, _, _, none = lib.rope_score_threshold(idx, bf16, torch.full((W,), 1.5, device="cuda"))
    assert none == 0
    lib.rope_sync_status()
    idx.free()
