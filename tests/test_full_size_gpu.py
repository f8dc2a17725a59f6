"""The benchmark's own workload and launch configuration — a 100 Mbp Markov
reference (10^8 windows) and one 131,072-read batch through rope_map — checked
on what the FP64 oracle can compute one by one: the fidelity of sampled
reported windows, and, for sampled reads, that no window the oracle scores
(the planted locus's neighbourhood) beats the reported best by more than the
tolerance; plus properties that hold at any size."""
import numpy as np
import pytest
import torch

import oracle
import synth
from _parity import bf16_tol, f32_tol

pytestmark = pytest.mark.gpu

L, B, K = 100_000_000, 131_072, 8


@pytest.fixture(scope="module")
def full(lib):
    ref = synth.markov_ref(L, 0.41, 3, 0.025, 0.025, 0.0)
    rd = synth.reads(ref, B, seed=4)
    p = lib.Params(s=4, m=2, t=2, variant=1, window_len=150)
    idx = lib.rope_encode_reference(p, torch.from_numpy(ref).cuda())
    seqs, offs = torch.from_numpy(rd.seqs).cuda(), torch.from_numpy(rd.offsets).cuda()
    w, s = lib.rope_map(idx, seqs, offs, k=K)
    lib.rope_sync_status()
    yield dict(ref=ref, rd=rd, w=w.cpu().numpy(), s=s.cpu().numpy().astype(np.float64), op=oracle.Params(N=150))
    idx.free()


def test_full_size_properties(full):
    w, s = full["w"], full["s"]
    assert w.shape == (B, K)
    assert np.all((w >= 0) & (w <= L - 150))
    assert np.all(np.diff(s, axis=1) <= 0)
    assert np.all((s >= 0) & (s <= 1 + 1e-5))
    srt = np.sort(w, axis=1)
    assert np.all(np.diff(srt, axis=1) > 0)  # distinct windows per read
    hit = np.abs(w[:, 0] - full["rd"].true_pos) < 150
    assert hit.mean() >= 0.98


def test_full_size_scores_match_oracle(full):
    rng = np.random.default_rng(7)
    rows = rng.choice(B, 512, replace=False)
    ri = np.repeat(rows, K)
    ws = full["w"][rows].reshape(-1)
    truth = oracle.score_pairs(full["ref"], full["rd"].seqs, full["rd"].offsets, ri, ws, full["op"])
    got = full["s"][rows].reshape(-1)
    assert np.all(np.abs(got - truth) <= f32_tol(truth)), np.abs(got - truth).max()


def test_full_size_best_not_beaten_near_truth(full):
    """For sampled reads, every window within 200 letters of the planted start
    (scored by the oracle) is at most the reported best plus the BF16
    tolerance: the scan found the best window of that neighbourhood. And over
    the windows the oracle scored for the read (that neighbourhood and the 8
    reported windows) the reported best is the oracle's best wherever the
    oracle's best beats its second by more than the FP32 tolerance (reported
    scores are re-scored in FP32): the unique planted locus is found exactly.
    (The oracle's exhaustive scan of 10^8 windows per read is out of reach
    here, so the compared set is the one the oracle can score one by one.)"""
    rng = np.random.default_rng(8)
    rows = rng.choice(B, 64, replace=False)
    rd = full["rd"]
    n_clear = 0
    for r in rows:
        lo = max(0, int(rd.true_pos[r]) - 200)
        hi = min(L - 150, int(rd.true_pos[r]) + 200)
        ws = np.arange(lo, hi + 1)
        sc = oracle.score_pairs(full["ref"], rd.seqs, rd.offsets, np.full(len(ws), r), ws, full["op"])
        best = full["s"][r, 0]
        assert sc.max() <= best + bf16_tol(sc.max()), (r, sc.max(), best)
        rep = full["w"][r]
        extra = rep[~np.isin(rep, ws)]
        sx = oracle.score_pairs(full["ref"], rd.seqs, rd.offsets, np.full(len(extra), r), extra, full["op"])
        allw, alls = np.concatenate([ws, extra]), np.concatenate([sc, sx])
        order = np.lexsort((allw, -alls))
        if alls[order[0]] - alls[order[1]] > f32_tol(alls[order[0]]):
            n_clear += 1
            assert full["w"][r, 0] == allw[order[0]], (r, full["w"][r, 0], allw[order[0]])
    assert n_clear >= 48
