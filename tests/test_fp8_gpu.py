"""E4M3 tensor-core scan (the FP8 option of step a5): raw scores within the
tolerance derived from E4M3 rounding, re-scored top-k held to the FP32
tolerance, planted loci as found by the FP64 oracle, the d = 128, stride > 1
and s = 3 tile paths, and both d = 64 tile variants giving one result."""
import numpy as np
import pytest

import oracle
import synth
from _parity import check_topk, dev, f32_tol, fp8_tol

pytestmark = pytest.mark.gpu


def gparams(lib, op):
    return lib.Params(s=op.s, m=op.m, t=op.t, variant=op.variant, score_mode=op.score_mode, window_len=op.N,
                      stride=op.stride)


@pytest.fixture(scope="module")
def case(lib):
    """100 kbp uniform reference, 256 planted 150 bp reads, d = 64."""
    ref = synth.uniform_ref(100_000, 1)
    rd = synth.reads(ref, 256, seed=2)
    op = oracle.Params(s=4, m=2, t=2, variant=1, N=150, stride=1)
    ow, os_ = oracle.score_topk(ref, rd.seqs, rd.offsets, op, k=9)
    p = gparams(lib, op)
    idx = lib.rope_encode_reference(p, dev(ref))
    f32, bf16, norms = lib.rope_encode_reads(p, dev(rd.seqs), dev(rd.offsets))
    lib.rope_sync_status()
    yield dict(ref=ref, rd=rd, op=op, ow=ow, os=os_, idx=idx, f32=f32, bf16=bf16, norms=norms)
    idx.free()


@pytest.mark.parametrize("j0,cnt,nr", [(0, 2100, 256), (97_000, 2851, 37), (31, 1, 5)])
def test_dense_fp8_parity(lib, case, j0, cnt, nr):
    got = lib.rope_score_dense(case["idx"], case["f32"][:nr], case["bf16"][:nr], case["norms"][:nr], j0, cnt,
                               precision="fp8")
    lib.rope_sync_status()
    got = got.cpu().numpy().astype(np.float64)
    wins = oracle.windows_direct(case["ref"], case["op"], j0, cnt)
    want = np.empty((nr, cnt))
    for i in range(nr):
        x = oracle.embed(case["rd"].read(i), case["op"])
        for j in range(cnt):
            want[i, j] = oracle.fidelity(x, wins[j])
    assert not np.isnan(got).any()
    err = np.abs(got - want)
    assert np.all(err <= fp8_tol(want)), err.max()
    # the bound is a worst case; typical errors are an order of magnitude below it
    assert np.median(err) <= 0.01, np.median(err)
    # the planted windows (fidelity near 1) keep a fidelity near 1
    hi = want > 0.8
    assert np.all(got[hi] > 0.5)


@pytest.mark.parametrize("rescore", [1, 0])
def test_topk_fp8_config1(lib, case, rescore):
    gw, gs = lib.rope_score_topk(case["idx"], case["f32"], case["bf16"], case["norms"], k=8, precision="fp8",
                                 rescore=rescore)
    lib.rope_sync_status()
    check_topk(case["ref"], case["rd"], case["op"], gw.cpu().numpy(), gs.cpu().numpy().astype(np.float64),
               case["ow"], case["os"], 8, fp8_tol, f32_tol if rescore else fp8_tol)


def test_topk_fp8_planted_accuracy(lib, case):
    gw, _ = lib.rope_score_topk(case["idx"], case["f32"], case["bf16"], case["norms"], k=1, precision="fp8")
    hit = np.abs(gw.cpu().numpy()[:, 0] - case["rd"].true_pos) < 150
    ora = np.abs(case["ow"][:, 0] - case["rd"].true_pos) < 150
    assert hit.mean() >= 0.97
    assert abs(hit.mean() - ora.mean()) <= 1.0 / 256 + 1e-12


@pytest.mark.parametrize("pp", [dict(s=4, m=4, t=2, variant=1, N=150, stride=1),
                                dict(s=4, m=2, t=2, variant=1, N=400, stride=8),
                                dict(s=3, m=2, t=2, variant=0, N=64, stride=3)])
def test_topk_fp8_other_shapes(lib, pp):
    ref = synth.markov_ref(30_000, 0.41, 51, 0.05, 0.05)
    rd = synth.reads(ref, 45, seed=52, length=pp["N"])
    op = oracle.Params(**pp)
    ow, os_ = oracle.score_topk(ref, rd.seqs, rd.offsets, op, k=5)
    p = gparams(lib, op)
    idx = lib.rope_encode_reference(p, dev(ref))
    f32, bf16, norms = lib.rope_encode_reads(p, dev(rd.seqs), dev(rd.offsets))
    gw, gs = lib.rope_score_topk(idx, f32, bf16, norms, k=4, precision="fp8")
    lib.rope_sync_status()
    check_topk(ref, rd, op, gw.cpu().numpy(), gs.cpu().numpy().astype(np.float64), ow, os_, 4, fp8_tol, f32_tol)
    # the raw dense scores of the d = 128 / stride / s = 3 tiles
    dense = lib.rope_score_dense(idx, f32, bf16, norms, 0, 700, precision="fp8").cpu().numpy().astype(np.float64)
    wins = oracle.windows_direct(ref, op, 0, 700)
    xs = [oracle.embed(rd.read(i), op) for i in range(rd.n)]
    want = np.array([[oracle.fidelity(x, w) for w in wins] for x in xs])
    assert np.all(np.abs(dense - want) <= fp8_tol(want))
    idx.free()


def test_fp8_tile_variants_agree(lib, case):
    """All d = 64 tile variants score the same products: the same re-scored top-k."""
    out = []
    for v in (0, 1, 2):
        lib.rope_autotune_set(case["idx"], 256, v, 16, k=8, precision="fp8")
        gw, gs = lib.rope_score_topk(case["idx"], case["f32"], case["bf16"], case["norms"], k=8, precision="fp8")
        lib.rope_sync_status()
        out.append((gw.cpu().numpy(), gs.cpu().numpy()))
        assert lib.rope_autotune_query(case["idx"], 256, k=8, precision="fp8")[0] == v
    lib.rope_autotune_enable(False)
    lib.rope_autotune_enable(True)
    for o in out[1:]:
        assert np.array_equal(out[0][0], o[0])
        assert np.array_equal(out[0][1], o[1])
