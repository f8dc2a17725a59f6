"""Both strands: reads planted on either strand are mapped by their head and
by the head of their reverse complement; the merged top-k matches the FP64
oracle's, and planted loci come back with their strand."""
import numpy as np
import pytest

import oracle
import synth
from _parity import bf16_tol, dev, f32_tol

pytestmark = pytest.mark.gpu


def _planted_both_strands(ref, n, seed, length=150):
    rd = synth.reads(ref, n, seed=seed, length=length)
    flip = np.arange(n) % 2 == 1
    parts = []
    for i in range(n):
        r = rd.seqs[rd.offsets[i]:rd.offsets[i + 1]]
        parts.append(oracle.reverse_complement(r) if flip[i] else r)
    rd.seqs = np.concatenate(parts)
    return rd, flip


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_strands_against_oracle(lib, precision):
    ref = synth.markov_ref(200_000, 0.41, 41, 0.025, 0.025, 0.0)
    rd, flip = _planted_both_strands(ref, 120, 42)
    op = oracle.Params(s=4, m=2, t=2, variant=1, N=150)
    p = lib.Params(s=4, m=2, t=2, variant=1, window_len=150)
    idx = lib.rope_encode_reference(p, dev(ref))
    k = 4
    w, s, t = lib.rope_map_strands(idx, dev(rd.seqs), dev(rd.offsets), k=k, precision=precision)
    lib.rope_sync_status()
    w, s, t = w.cpu().numpy(), s.cpu().numpy().astype(np.float64), t.cpu().numpy()
    ow, os_, ot = oracle.score_topk_strands(ref, rd.seqs, rd.offsets, op, k=k + 1)
    rc = np.concatenate([oracle.reverse_complement(rd.seqs[rd.offsets[i]:rd.offsets[i + 1]]) for i in range(rd.n)])
    # every reported score is the oracle's fidelity of that window for that strand's head
    for strand, seqs in ((0, rd.seqs), (1, rc)):
        valid = (t == strand) & (w >= 0)
        ri = np.repeat(np.arange(rd.n), k).reshape(rd.n, k)[valid]
        truth = oracle.score_pairs(ref, seqs, rd.offsets, ri, w[valid], op)
        assert np.all(np.abs(s[valid] - truth) <= f32_tol(truth))
    # the merged list holds every oracle entry that beats the oracle's (k+1)-th by more than the tolerance
    tol = f32_tol if precision == "fp32" else bf16_tol
    for i in range(rd.n):
        got = set(zip(w[i].tolist(), t[i].tolist()))
        for j in range(k):
            if os_[i, j] - os_[i, k] > tol(os_[i, j]):
                assert (ow[i, j], ot[i, j]) in got
    assert np.all(np.diff(s, axis=1) <= 0)
    # planted loci come back on their strand
    hit = (np.abs(w[:, 0] - rd.true_pos) < 150) & (t[:, 0] == flip.astype(np.int8))
    assert hit.mean() >= 0.95
    idx.free()


def test_strands_forward_rows_equal_rope_map(lib):
    """Where the best hit is on the forward strand, rope_map_strands gives
    rope_map's top-1 with strand 0."""
    ref = synth.uniform_ref(100_000, 1)
    rd = synth.reads(ref, 64, seed=2)
    p = lib.Params(s=4, m=2, t=2, variant=1, window_len=150)
    idx = lib.rope_encode_reference(p, dev(ref))
    w, s, t = lib.rope_map_strands(idx, dev(rd.seqs), dev(rd.offsets), k=1)
    w1, s1 = lib.rope_map(idx, dev(rd.seqs), dev(rd.offsets), k=1)
    lib.rope_sync_status()
    fwd = t.cpu().numpy()[:, 0] == 0
    assert fwd.mean() > 0.9
    assert np.array_equal(w.cpu().numpy()[fwd], w1.cpu().numpy()[fwd])
    assert np.array_equal(s.cpu().numpy()[fwd], s1.cpu().numpy()[fwd])
    idx.free()
