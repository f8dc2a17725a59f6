"""The scan tuner: every tile variant and work split gives the oracle's
top-k, and a tuned choice is recorded per shape class."""
import numpy as np
import pytest

import oracle
import synth
from _parity import bf16_tol, check_topk, dev, f32_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case(lib):
    ref = synth.markov_ref(300_000, 0.41, 21, 0.025, 0.025, 0.0)
    rd = synth.reads(ref, 300, seed=22)
    op = oracle.Params(s=4, m=2, t=2, variant=1, N=150, stride=1)
    ow, os_ = oracle.score_topk(ref, rd.seqs, rd.offsets, op, k=9)
    p = lib.Params(s=4, m=2, t=2, variant=1, window_len=150)
    idx = lib.rope_encode_reference(p, dev(ref))
    yield dict(ref=ref, rd=rd, op=op, ow=ow, os=os_, idx=idx, seqs=dev(rd.seqs), offs=dev(rd.offsets))
    idx.free()


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("items", [1, 8, 32])
def test_each_variant_matches_oracle(lib, case, variant, items):
    c = case
    lib.rope_autotune_set(c["idx"], c["rd"].n, variant, items, k=8)
    assert lib.rope_autotune_query(c["idx"], c["rd"].n, k=8)[:2] == (variant, items)
    w, s = lib.rope_map(c["idx"], c["seqs"], c["offs"], k=8)
    lib.rope_sync_status()
    check_topk(c["ref"], c["rd"], c["op"], w.cpu().numpy(), s.cpu().numpy().astype(np.float64), c["ow"], c["os"], 8,
               bf16_tol, f32_tol)
    # raw BF16 scores (no re-scoring) are the same whatever the variant and split
    w0, s0 = lib.rope_map(c["idx"], c["seqs"], c["offs"], k=8, rescore=0)
    lib.rope_autotune_set(c["idx"], c["rd"].n, 0, 16, k=8)
    w1, s1 = lib.rope_map(c["idx"], c["seqs"], c["offs"], k=8, rescore=0)
    lib.rope_sync_status()
    assert np.array_equal(w0.cpu().numpy(), w1.cpu().numpy()) and np.array_equal(s0.cpu().numpy(), s1.cpu().numpy())


def test_tuner_records_a_choice(lib, case):
    c = case
    lib.rope_autotune_enable(False)  # forget earlier choices
    lib.rope_autotune_enable(True)
    assert lib.rope_autotune_query(c["idx"], c["rd"].n, k=8, sep=150) is None
    w, s = lib.rope_map(c["idx"], c["seqs"], c["offs"], k=8, sep=150)
    lib.rope_sync_status()
    got = lib.rope_autotune_query(c["idx"], c["rd"].n, k=8, sep=150)
    assert got is not None and got[0] in (0, 1, 2) and got[1] in (8, 16, 32) and got[2] > 0
    ow, os_ = oracle.score_topk(c["ref"], c["rd"].seqs, c["rd"].offsets, c["op"], k=9, sep=150)
    check_topk(c["ref"], c["rd"], c["op"], w.cpu().numpy(), s.cpu().numpy().astype(np.float64), ow, os_, 8,
               bf16_tol, f32_tol, sep=150)
