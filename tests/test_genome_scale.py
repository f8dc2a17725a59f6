"""Genome scale: a maize-shaped 2.3 Gbp reference (positions past 2^31,
window numbers past 2^31), scanned in the launch configuration the benchmark
uses. Checked against the FP64 oracle on what it can compute one by one:
the fidelity of every reported window, and an exhaustive scan of the last
100,000 windows of the genome."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

L = 2_300_000_000


@pytest.fixture(scope="module")
def genome(lib):
    ref = synth.markov_ref(L, 0.47, 8, 0.0, 0.0, 0.85)
    # reads: most at uniform loci, a few planted in the last 100 kbp
    rd = synth.concat([synth.reads(ref, 448, seed=21), synth.reads(ref[L - 100_000:], 64, seed=22)])
    rd.true_pos[448:] += L - 100_000
    p = lib.Params(s=4, m=2, t=2, variant=1, window_len=150)
    idx = lib.rope_encode_reference(p, torch.from_numpy(ref).cuda())
    seqs, offs = torch.from_numpy(rd.seqs).cuda(), torch.from_numpy(rd.offsets).cuda()
    f32, bf16, norms = lib.rope_encode_reads(p, seqs, offs)
    lib.rope_sync_status()
    yield dict(ref=ref, rd=rd, idx=idx, f32=f32, bf16=bf16, norms=norms, op=oracle.Params(N=150))
    idx.free()


def test_window_count_past_2_31(genome):
    W = genome["idx"].n_windows
    assert W == L - 150 + 1 and W > 2 ** 31


@pytest.mark.parametrize("precision", ["bf16", "fp32"])
def test_reported_scores_match_oracle(lib, genome, precision):
    g = genome
    if precision == "fp32":
        sub = slice(0, 64)  # the FP32 scan is ~15x slower: a sample of reads
        f32, bf16, norms = g["f32"][sub], g["bf16"][sub], g["norms"][sub]
    else:
        f32, bf16, norms = g["f32"], g["bf16"], g["norms"]
    w, s = lib.rope_score_topk(g["idx"], f32, bf16, norms, k=4, precision=precision)
    lib.rope_sync_status()
    w, s = w.cpu().numpy(), s.cpu().numpy().astype(np.float64)
    n = w.shape[0]
    valid = w >= 0
    assert valid.all()
    ri = np.repeat(np.arange(n), 4).reshape(n, 4)
    truth = oracle.score_pairs(g["ref"], g["rd"].seqs, g["rd"].offsets, ri[valid], w[valid], g["op"])
    assert np.all(np.abs(s[valid] - truth) <= 1e-5 * truth + 1e-7)
    # planted loci are found, including past 2^31
    hit = np.abs(w[:, 0] - g["rd"].true_pos[:n]) < 150
    assert hit.mean() >= 0.95
    if precision == "bf16":
        # reads planted in the last 100 kbp (past 2^31): found there, with the
        # window numbers of those loci past 2^31 as well
        assert hit[448:].mean() >= 0.9
        assert (w[448:, 0][hit[448:]] > 2 ** 31).all()


def test_exhaustive_tail_against_oracle(lib, genome):
    g = genome
    W = g["idx"].n_windows
    jb, je = W - 100_000, W
    sel = np.r_[0:8, 448:456]
    sub = g["rd"].subset(sel)
    ow, os_ = oracle.score_topk(g["ref"], sub.seqs, sub.offsets, g["op"], k=5, j_begin=jb, j_end=je)
    idx_t = torch.from_numpy(sel).cuda()
    w, s = lib.rope_score_topk(g["idx"], g["f32"][idx_t].contiguous(), g["bf16"][idx_t].contiguous(),
                               g["norms"][idx_t].contiguous(), k=4, precision="bf16", j_begin=jb, j_end=je)
    lib.rope_sync_status()
    w, s = w.cpu().numpy(), s.cpu().numpy().astype(np.float64)
    for i in range(len(sel)):
        for j in range(4):
            if os_[i, j] - os_[i, 4] > 2e-2 * os_[i, j]:
                assert ow[i, j] in set(w[i].tolist())
        ok = w[i] >= 0
        truth = oracle.score_pairs(g["ref"], sub.seqs, sub.offsets, np.full(ok.sum(), i), w[i][ok], g["op"])
        assert np.all(np.abs(s[i][ok] - truth) <= 1e-5 * truth + 1e-7)
