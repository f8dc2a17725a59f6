"""The materialised index (§3.1's database of window encodings, the paper's
long-read configuration of §3.2/§3.5: window N = 20,000, step 1,250, the
fine-tuned compact encoding s = 8, m = 4, t = 4 = 1024 complex dimensions) and
its BF16 tcgen05 GEMM scan, against the FP64 oracle through the C ABI.

Tolerances as in the other parity tests: window encodings within
1e-5 * |c| (FP32 sums of at most N unit phases, here combined from block
sums); raw BF16 scores within max(2e-2 f, 8e-3 sqrt(f) + 2e-5); re-scored
scores within 1e-5 f + 1e-7; the top-1 window exact wherever the oracle's
best beats its second by more than the tolerance. Sizes span several 128-read
and 128-window tiles with ragged last tiles, and every way a window's block
sums are completed (whole blocks; a partial last block added; a whole last
block with its over-covered starts removed)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from _parity import bf16_tol, check_topk, dev, f32_tol

pytestmark = pytest.mark.gpu

# (s, m, t, N, stride): N - s + 1 = 19993 = 15 * 1250 + 1243 -> 16 blocks, 7
# starts removed (the paper's configuration); 147 = 21 * 7 (whole blocks);
# 147 = 14 * 10 + 7 (a whole 15th block, 3 starts removed); 147 = 7 * 20 + 7
# (7 starts of a partial block added); 1993 = 15 * 125 + 118 (the paper's
# ratio N / step = 16 at a tenth of the length)
WINDOW_CASES = [
    (8, 4, 4, 20000, 1250),
    (4, 2, 2, 150, 7),
    (4, 4, 2, 150, 10),
    (4, 2, 2, 150, 20),
    (8, 4, 4, 2000, 125),
]


def gparams(lib, s, m, t, N, stride):
    return lib.Params(s=s, m=m, t=t, variant=1, window_len=N, stride=stride)


@pytest.mark.parametrize("s,m,t,N,stride", WINDOW_CASES)
def test_dense_windows_match_oracle(lib, s, m, t, N, stride):
    ref = synth.markov_ref(400_000 if N > 2000 else 60_000, 0.41, 91, 0.05, 0.05)
    op = oracle.Params(s=s, m=m, t=t, variant=1, N=N, stride=stride)
    idx = lib.rope_encode_reference_dense(gparams(lib, s, m, t, N, stride), dev(ref))
    W = idx.n_windows
    assert W == oracle.n_windows(len(ref), N, stride)
    D = op.dim
    inv = idx.inv_norm().cpu().numpy()
    for j0, cnt in ((0, 40), (W // 2, 17), (W - 23, 23)):
        got = lib.rope_window_embeddings(idx, j0, cnt).cpu().numpy().astype(np.float64)
        want = oracle.windows_direct(ref, op, j0, cnt)
        g = got[:, :D] + 1j * got[:, D:]
        nrm = np.linalg.norm(want, axis=1, keepdims=True)
        assert np.all(np.abs(g - want) <= 1e-5 * nrm + 1e-6), np.abs(g - want).max()
        assert np.allclose(inv[j0:j0 + cnt], 1 / nrm[:, 0], rtol=1e-5)
    lib.rope_sync_status()
    idx.free()


@pytest.fixture(scope="module")
def long_reads(lib):
    """1 Mbp uniform reference (785 windows: seven 128-window tiles, the last
    ragged) and 300 planted 20 kbp reads at 15% errors (5% substitutions, 10%
    indel events): three 128-read tiles, the last ragged."""
    ref = synth.uniform_ref(1_000_000, 31)
    rd = synth.reads(ref, 300, seed=32, length=20000, sub_rate=0.05, indel_rate=0.10)
    op = oracle.Params(s=8, m=4, t=4, variant=1, N=20000, stride=1250)
    p = gparams(lib, 8, 4, 4, 20000, 1250)
    idx = lib.rope_encode_reference(p, dev(ref))  # 1024 complex dimensions: the materialised index
    seqs, offs = dev(rd.seqs), dev(rd.offsets)
    f32, bf16, norms = lib.rope_encode_reads(p, seqs, offs)
    lib.rope_sync_status()
    ow, os_ = oracle.score_topk(ref, rd.seqs, rd.offsets, op, k=9)
    yield dict(ref=ref, rd=rd, op=op, p=p, idx=idx, seqs=seqs, offs=offs, f32=f32, bf16=bf16, norms=norms, ow=ow,
               os=os_)
    idx.free()


def _oracle_dense(c, j0, cnt, nr):
    op, ref, rd = c["op"], c["ref"], c["rd"]
    wins = oracle.windows_direct(ref, op, j0, cnt)
    X = np.stack([oracle.embed(rd.read(i), op) for i in range(nr)])
    ip = X.conj() @ wins.T
    nx = np.sum(np.abs(X) ** 2, axis=1)[:, None]
    nc = np.sum(np.abs(wins) ** 2, axis=1)[None, :]
    return np.abs(ip) ** 2 / (nx * nc)


@pytest.mark.parametrize("j0,cnt,nr", [(0, 785, 300), (200, 77, 129), (700, 85, 1), (5, 1, 7)])
def test_dense_gemm_scores(lib, long_reads, j0, cnt, nr):
    c = long_reads
    got = lib.rope_score_dense(c["idx"], c["f32"][:nr], c["bf16"][:nr], c["norms"][:nr], j0, cnt, precision="bf16")
    lib.rope_sync_status()
    got = got.cpu().numpy().astype(np.float64)
    want = _oracle_dense(c, j0, cnt, nr)
    assert not np.isnan(got).any()
    err = np.abs(got - want)
    assert np.all(err <= bf16_tol(want)), (err.max(), (err / np.maximum(want, 1e-9)).max())


def test_dense_topk_rescored(lib, long_reads):
    c = long_reads
    gw, gs = lib.rope_score_topk(c["idx"], c["f32"], c["bf16"], c["norms"], k=8, precision="bf16", rescore=1)
    lib.rope_sync_status()
    gw, gs = gw.cpu().numpy(), gs.cpu().numpy().astype(np.float64)
    check_topk(c["ref"], c["rd"], c["op"], gw, gs, c["ow"], c["os"], 8, bf16_tol, f32_tol)
    clear = c["os"][:, 0] - c["os"][:, 1] > f32_tol(c["os"][:, 0])
    assert np.array_equal(gw[clear, 0], c["ow"][clear, 0])
    assert clear.mean() > 0.9
    hit = np.abs(gw[:, 0] - c["rd"].true_pos) < 20000
    assert hit.mean() >= 0.99


def test_dense_topk_raw_sep_subrange(lib, long_reads):
    c = long_reads
    k, sep = 5, 5000
    gw, gs = lib.rope_score_topk(c["idx"], c["f32"], c["bf16"], c["norms"], k=k, sep=sep, precision="bf16", rescore=0,
                                 j_begin=100, j_end=650)
    lib.rope_sync_status()
    gw, gs = gw.cpu().numpy(), gs.cpu().numpy().astype(np.float64)
    ow, os_ = oracle.score_topk(c["ref"], c["rd"].seqs, c["rd"].offsets, c["op"], k=k + 1, sep=sep, j_begin=100,
                                j_end=650)
    assert np.all((gw[gw >= 0] >= 100 * 1250) & (gw[gw >= 0] < 650 * 1250))
    check_topk(c["ref"], c["rd"], c["op"], gw, gs, ow, os_, k, bf16_tol, sep=sep)


def test_dense_map_strands(lib, long_reads):
    """Both strands (§3.5): the reverse-strand reads map to their locus on the
    reverse strand; results agree with the oracle's strand-merged top-k."""
    c = long_reads
    rd = c["rd"].subset(np.arange(40))
    # reverse-complement every other read
    parts = []
    for i in range(rd.n):
        r = np.frombuffer(rd.read(i), dtype=np.uint8)
        parts.append(oracle.reverse_complement(r) if i % 2 else r)
    seqs = np.concatenate(parts)
    offs = np.zeros(rd.n + 1, np.int64)
    offs[1:] = np.cumsum([len(x) for x in parts])
    w, s, strand = lib.rope_map_strands(c["idx"], dev(seqs), dev(offs), k=4, precision="bf16")
    lib.rope_sync_status()
    w, s, strand = w.cpu().numpy(), s.cpu().numpy().astype(np.float64), strand.cpu().numpy()
    assert np.array_equal(strand[:, 0], np.arange(rd.n) % 2)
    assert np.mean(np.abs(w[:, 0] - rd.true_pos) < 20000) >= 0.95
    ow, os_, ost = oracle.score_topk_strands(c["ref"], seqs, offs, c["op"], k=4)
    clear = os_[:, 0] - os_[:, 1] > f32_tol(os_[:, 0])
    assert np.array_equal(w[clear, 0], ow[clear, 0]) and np.array_equal(strand[clear, 0], ost[clear, 0])
    assert np.all(np.abs(s[clear, 0] - os_[clear, 0]) <= f32_tol(os_[clear, 0]))


def test_dense_small_dimension_matches_on_the_fly(lib):
    """The same GEMM at d = 64 (one 64-wide K block) against the on-the-fly
    tensor-core scan of the same encoding: re-scored top-k identical where the
    oracle's gaps are clear (both re-score in FP32), scores within FP32."""
    ref = synth.uniform_ref(100_000, 1)
    rd = synth.reads(ref, 300, seed=2)
    p = lib.Params(s=4, m=2, t=2, variant=1, window_len=150)
    a = lib.rope_encode_reference(p, dev(ref))
    b = lib.rope_encode_reference_dense(p, dev(ref))
    f32, bf16, norms = lib.rope_encode_reads(p, dev(rd.seqs), dev(rd.offsets))
    wa, sa = lib.rope_score_topk(a, f32, bf16, norms, k=4, precision="bf16")
    wb, sb = lib.rope_score_topk(b, f32, bf16, norms, k=4, precision="bf16")
    lib.rope_sync_status()
    wa, sa, wb, sb = (x.cpu().numpy() for x in (wa, sa, wb, sb))
    op = oracle.Params(s=4, m=2, t=2, variant=1, N=150)
    ow, os_ = oracle.score_topk(ref, rd.seqs, rd.offsets, op, k=5)
    check_topk(ref, rd, op, wb, sb.astype(np.float64), ow, os_, 4, bf16_tol, f32_tol)
    clear = os_[:, 0] - os_[:, 1] > f32_tol(os_[:, 0])
    assert np.array_equal(wb[clear, 0], wa[clear, 0])
    same = wa == wb
    assert np.all(np.abs(sa[same] - sb[same]) <= f32_tol(sa[same]))
    a.free()
    b.free()


def test_dense_topk_fp32_plain(lib, long_reads):
    """The plain FP32 scan of the materialised index (CUDA cores, the stored
    FP32 rows): the oracle's top-k at the FP32 tolerance, top-1 exact where
    clear."""
    c = long_reads
    gw, gs = lib.rope_score_topk(c["idx"], c["f32"], None, c["norms"], k=8, precision="fp32")
    lib.rope_sync_status()
    gw, gs = gw.cpu().numpy(), gs.cpu().numpy().astype(np.float64)
    check_topk(c["ref"], c["rd"], c["op"], gw, gs, c["ow"], c["os"], 8, f32_tol)
    clear = c["os"][:, 0] - c["os"][:, 1] > f32_tol(c["os"][:, 0])
    assert np.array_equal(gw[clear, 0], c["ow"][clear, 0])
    # a window sub-range with buckets, three read tiles of 64 (the last ragged),
    # the deepest candidate lists (32 entries: 16 KB of lists per block)
    k, sep = 4, 5000
    gw, gs = lib.rope_score_topk(c["idx"], c["f32"][:150], None, c["norms"][:150], k=k, sep=sep, precision="fp32",
                                 j_begin=50, j_end=700, cand_depth=32)
    lib.rope_sync_status()
    sub = c["rd"].subset(np.arange(150))
    ow, os_ = oracle.score_topk(c["ref"], sub.seqs, sub.offsets, c["op"], k=k + 1, sep=sep, j_begin=50, j_end=700)
    check_topk(c["ref"], sub, c["op"], gw.cpu().numpy(), gs.cpu().numpy().astype(np.float64), ow, os_, k, f32_tol,
               sep=sep)


def test_dense_refusals(lib, long_reads):
    c = long_reads
    with pytest.raises(lib.RopeError) as e:  # every score: the BF16 GEMM only
        lib.rope_score_dense(c["idx"], c["f32"], None, c["norms"], 0, 10, precision="fp32")
    assert e.value.status == 6
    out = (torch.empty((300, 4), dtype=torch.int64, device="cuda"), torch.empty((300, 4), dtype=torch.float32,
                                                                               device="cuda"))
    with pytest.raises(lib.RopeError) as e:
        lib.rope_score_topk_noalloc(c["idx"], c["f32"], c["bf16"], c["norms"], out, k=4)
    assert e.value.status == 6
    with pytest.raises(lib.RopeError) as e:  # 4^1 x 1 = 4 complex dimensions: not a multiple of 32
        lib.rope_encode_reference_dense(lib.Params(s=1, m=1, t=1, window_len=50), dev(synth.uniform_ref(1000, 1)))
    assert e.value.status == 6


@pytest.mark.parametrize("precision,tol", [("bf16", bf16_tol), ("fp32", f32_tol)])
def test_dense_topk_many_read_tiles(lib, precision, tol):
    """Enough reads that the work split runs in waves: 5000 reads (40 tiles of
    128 for the GEMM, 79 of 64 for the FP32 scan, the last ragged) against a
    materialised index of 8551 windows (67 tiles of 128); 4 window ranges per
    read, waves of 38 (GEMM) or 76 (FP32) read tiles, the second wave partial.
    At d = 64 the GEMM runs its short-K shape (resident read tile, two lists
    per read and range). Re-scored top-k against the oracle's, top-1 exact
    where clear."""
    op = oracle.Params(s=4, m=2, t=2, variant=1, N=150, stride=7)
    ref = synth.markov_ref(60_000, 0.41, 241, 0.05, 0.05)
    rd = synth.reads(ref, 5000, seed=242, length=150)
    p = gparams(lib, 4, 2, 2, 150, 7)
    idx = lib.rope_encode_reference_dense(p, dev(ref))
    f32, bf16, norms = lib.rope_encode_reads(p, dev(rd.seqs), dev(rd.offsets))
    k = 4
    gw, gs = lib.rope_score_topk(idx, f32, bf16 if precision == "bf16" else None, norms, k=k, precision=precision,
                                 rescore=1 if precision == "bf16" else None)
    lib.rope_sync_status()
    gw, gs = gw.cpu().numpy(), gs.cpu().numpy().astype(np.float64)
    ow, os_ = oracle.score_topk(ref, rd.seqs, rd.offsets, op, k=k + 1)
    # the BF16 scan proposes candidates by BF16 scores (an oracle top-k window
    # within the BF16 tolerance of the (k+1)-th may lose its place); every
    # reported score is the FP32 re-score
    check_topk(ref, rd, op, gw, gs, ow, os_, k, tol, f32_tol)
    clear = os_[:, 0] - os_[:, 1] > tol(os_[:, 0])
    assert clear.sum() > 1000
    assert np.array_equal(gw[clear, 0], ow[clear, 0])
    idx.free()


@pytest.mark.parametrize("s,m,t,N,stride", [(4, 2, 2, 150, 7), (4, 4, 2, 150, 10)])
def test_dense_short_k_shape(lib, s, m, t, N, stride):
    """The GEMM's short-K shape (2D = 64: one K block of the read tile kept in
    shared memory; 2D = 128: two) on every output mode: every score of a
    window sub-range with ragged tiles at the raw BF16 tolerance, the top-k
    with buckets against the oracle's, and the threshold pairs against the
    oracle's exhaustive set except pairs within the BF16 tolerance of their
    window's threshold."""
    op = oracle.Params(s=s, m=m, t=t, variant=1, N=N, stride=stride)
    ref = synth.markov_ref(40_000, 0.41, 251, 0.05, 0.05)
    rd = synth.reads(ref, 300, seed=252, length=N)
    p = gparams(lib, s, m, t, N, stride)
    idx = lib.rope_encode_reference_dense(p, dev(ref))
    W = idx.n_windows
    f32, bf16, norms = lib.rope_encode_reads(p, dev(rd.seqs), dev(rd.offsets))
    # dense scores over [37, 37 + 333): three window tiles, the last ragged
    j0, cnt, nr = 37, 333, 300
    got = lib.rope_score_dense(idx, f32, bf16, norms, j0, cnt, precision="bf16").cpu().numpy().astype(np.float64)
    lib.rope_sync_status()
    wins = oracle.windows_direct(ref, op, j0, cnt)
    X = np.stack([oracle.embed(rd.read(i), op) for i in range(nr)])
    want = np.abs(X.conj() @ wins.T) ** 2 / (np.sum(np.abs(X) ** 2, axis=1)[:, None] *
                                              np.sum(np.abs(wins) ** 2, axis=1)[None, :])
    assert np.all(np.abs(got - want) <= bf16_tol(want)), np.abs(got - want).max()
    # top-k with buckets of 500 letters, re-scored
    k, sep = 4, 500
    gw, gs = lib.rope_score_topk(idx, f32, bf16, norms, k=k, sep=sep, precision="bf16", rescore=1)
    lib.rope_sync_status()
    ow, os_ = oracle.score_topk(ref, rd.seqs, rd.offsets, op, k=k + 1, sep=sep)
    check_topk(ref, rd, op, gw.cpu().numpy(), gs.cpu().numpy().astype(np.float64), ow, os_, k, bf16_tol, f32_tol,
               sep=sep)
    # threshold pairs for a 10% rate
    thr = lib.rope_fragment_thresholds(idx, 0.10, 4, 5)
    r, w, sc, total = lib.rope_score_threshold(idx, bf16, thr)
    lib.rope_sync_status()
    r, w = r.cpu().numpy(), w.cpu().numpy()
    assert total == len(r) and total > 0
    thr_h = thr.cpu().numpy().astype(np.float64)
    orr, ow2, _ = oracle.threshold_pairs(ref, rd.seqs, rd.offsets, op, thr_h)
    got_set, want_set = set(zip(r.tolist(), w.tolist())), set(zip(orr.tolist(), ow2.tolist()))
    assert len(got_set) == len(r)
    for (i, j) in got_set ^ want_set:
        f = oracle.score_pairs(ref, rd.seqs, rd.offsets, np.array([i]), np.array([j * stride]), op)[0]
        assert abs(f - thr_h[j]) <= bf16_tol(f), (i, j, f, thr_h[j])
    assert W == oracle.n_windows(len(ref), N, stride)
    idx.free()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("s,m,t,N,stride", [(4, 2, 2, 150, 7), (8, 4, 4, 2000, 125)])
def test_dense_topk_subrange_and_fill(lib, precision, s, m, t, N, stride):
    """Edge cases of the materialised index's scans (short and long K): a
    range of 5 windows with k = 8 (three (-1, -inf) fills, the 5 windows in
    the oracle's order), an empty range (every slot (-1, -inf)), and no
    reads at all."""
    op = oracle.Params(s=s, m=m, t=t, variant=1, N=N, stride=stride)
    ref = synth.uniform_ref(30_000, 261)
    rd = synth.reads(ref, 9, seed=262, length=N)
    p = gparams(lib, s, m, t, N, stride)
    idx = lib.rope_encode_reference_dense(p, dev(ref))
    f32, bf16, norms = lib.rope_encode_reads(p, dev(rd.seqs), dev(rd.offsets))
    b = bf16 if precision == "bf16" else None
    gw, gs = lib.rope_score_topk(idx, f32, b, norms, k=8, precision=precision, rescore=1 if b is not None else None,
                                 j_begin=40, j_end=45)
    lib.rope_sync_status()
    gw, gs = gw.cpu().numpy(), gs.cpu().numpy().astype(np.float64)
    ow, os_ = oracle.score_topk(ref, rd.seqs, rd.offsets, op, k=8, j_begin=40, j_end=45)
    assert np.all(gw[:, 5:] == -1) and np.all(np.isneginf(gs[:, 5:]))
    assert np.array_equal(np.sort(gw[:, :5], axis=1), np.sort(ow[:, :5], axis=1))
    assert np.all(np.abs(np.sort(gs[:, :5], axis=1) - np.sort(os_[:, :5], axis=1)) <= f32_tol(np.sort(os_[:, :5], axis=1)))
    gw, gs = lib.rope_score_topk(idx, f32, b, norms, k=4, precision=precision, j_begin=10, j_end=10)
    lib.rope_sync_status()
    assert np.all(gw.cpu().numpy() == -1) and np.all(np.isneginf(gs.cpu().numpy()))
    gw, gs = lib.rope_score_topk(idx, f32[:0], b[:0] if b is not None else None, norms[:0], k=4, precision=precision)
    lib.rope_sync_status()
    assert gw.shape == (0, 4)
    idx.free()
