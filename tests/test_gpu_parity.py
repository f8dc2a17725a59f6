"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances:
  * packing, s-mer bins, window indices: bit-exact;
  * FP32 embeddings: |gpu - oracle| <= 1e-5 * ||oracle vector|| (FP32 direct
    sums of at most N unit phases);
  * FP32 scores: |gpu - oracle| <= 1e-5 * fid + 1e-7;
  * BF16 tensor-core scores before re-scoring: |gpu - oracle| <= max(2e-2 * fid, 8e-3 * sqrt(fid) + 2e-5)
    (each operand is a unit vector rounded to BF16, relative error <= 2^-9 per
    component, so |d ip| <= 2^-8 and |d fid| <= 2 * 2^-8 * sqrt(fid) + 2^-16);
  * top-k: every oracle top-k window that beats the oracle's (k+1)-th score by
    more than the tolerance is present; reported scores match the oracle's
    fidelity of the reported window; the reported best window is the oracle's
    best wherever the oracle's best beats its second by more than the
    tolerance (the planted locus is then unique).
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

from _parity import F32_ABS, F32_REL, bf16_tol, check_topk, dev, f32_tol  # noqa: F401


def gparams(op, **kw):
    from paper_2603_22245_gb300 import rotormap as rm
    d = dict(s=op.s, m=op.m, t=op.t, variant=op.variant, score_mode=op.score_mode, window_len=op.N,
             stride=op.stride, bin_map=None)
    d.update(kw)
    return rm.Params(**d)


# ---------------------------------------------------------------- fixtures

@pytest.fixture(scope="module")
def cfg1():
    """100 kbp uniform reference, 256 planted 150 bp reads (1% subs, 0.5% indels), d = 64."""
    ref = synth.uniform_ref(100_000, 1)
    rd = synth.reads(ref, 256, seed=2)
    op = oracle.Params(s=4, m=2, t=2, variant=1, N=150, stride=1)
    w9, s9 = oracle.score_topk(ref, rd.seqs, rd.offsets, op, k=9)
    return dict(ref=ref, rd=rd, op=op, ow=w9, os=s9)


@pytest.fixture(scope="module")
def cfg1_wide(lib):
    """The same reference with 640 reads: three 256-read groups of the
    tensor-core scan, the last one ragged (dense parity only)."""
    ref = synth.uniform_ref(100_000, 1)
    rd = synth.reads(ref, 640, seed=12)
    op = oracle.Params(s=4, m=2, t=2, variant=1, N=150, stride=1)
    p = gparams(op)
    idx = lib.rope_encode_reference(p, dev(ref))
    f32, bf16, norms = lib.rope_encode_reads(p, dev(rd.seqs), dev(rd.offsets))
    lib.rope_sync_status()
    yield dict(ref=ref, rd=rd, op=op), dict(idx=idx, f32=f32, bf16=bf16, norms=norms)
    idx.free()


@pytest.fixture(scope="module")
def cfg1_gpu(lib, cfg1):
    op = cfg1["op"]
    p = gparams(op)
    idx = lib.rope_encode_reference(p, dev(cfg1["ref"]))
    seqs, offs = dev(cfg1["rd"].seqs), dev(cfg1["rd"].offsets)
    f32, bf16, norms = lib.rope_encode_reads(p, seqs, offs)
    lib.rope_sync_status()
    return dict(p=p, idx=idx, seqs=seqs, offs=offs, f32=f32, bf16=bf16, norms=norms)


# ---------------------------------------------------------------- a1, a2

@pytest.mark.parametrize("n", [1, 15, 16, 17, 63, 64, 65, 129, 1000, 100_003])
def test_pack_bit_exact(lib, n):
    seq = synth.uniform_ref(n, 10 + n)
    seq[::7] = np.frombuffer(bytes(seq[::7]).lower(), dtype=np.uint8)
    got = lib.rope_pack_2bit(dev(seq)).cpu().numpy().view(np.uint32)
    lib.rope_sync_status()
    assert np.array_equal(got, oracle.pack_2bit(seq))


def test_pack_misaligned_and_invalid(lib):
    seq = synth.uniform_ref(4099, 3)
    buf = dev(np.concatenate([np.zeros(3, np.uint8), seq]))
    got = lib.rope_pack_2bit(buf[3:]).cpu().numpy().view(np.uint32)
    lib.rope_sync_status()
    assert np.array_equal(got, oracle.pack_2bit(seq))
    bad = seq.copy()
    bad[2000] = ord("N")
    lib.rope_pack_2bit(dev(bad))
    with pytest.raises(lib.RopeError) as e:
        lib.rope_sync_status()
    assert e.value.status == 2


@pytest.mark.parametrize("s,t,custom", [(1, 1, False), (4, 2, False), (4, 4, False), (6, 3, False), (8, 4, False),
                                        (5, 2, True)])
def test_mer_bins_bit_exact(lib, s, t, custom):
    seq = synth.uniform_ref(5001, 40 + s)
    bm = np.random.default_rng(s).integers(0, 4 ** t, size=4 ** s).astype(np.uint16) if custom else None
    op = oracle.Params(s=s, m=1, t=t, variant=0, N=s, bin_map=bm)
    packed = lib.rope_pack_2bit(dev(seq))
    got = lib.rope_mer_bins(gparams(op, bin_map=bm), packed, len(seq)).cpu().numpy().view(np.uint16)
    assert np.array_equal(got.astype(np.int32), oracle.mer_bins(seq, s, op.bin_map))


# ---------------------------------------------------------------- a3

ENC_PARAMS = [dict(s=4, m=2, t=2, variant=1, N=150), dict(s=4, m=4, t=2, variant=1, N=150),
              dict(s=2, m=2, t=2, variant=0, N=100), dict(s=1, m=1, t=1, variant=0, N=33),
              dict(s=8, m=4, t=4, variant=1, N=2000), dict(s=6, m=1, t=6, variant=0, N=500)]


@pytest.mark.parametrize("pp", ENC_PARAMS)
def test_encode_reads_parity(lib, pp):
    ref = synth.uniform_ref(50_000, 7)
    rd = synth.reads(ref, 37, seed=8, length=pp["N"] + 13)
    op = oracle.Params(**pp)
    f32, bf16, norms = lib.rope_encode_reads(gparams(op), dev(rd.seqs), dev(rd.offsets))
    lib.rope_sync_status()
    f32, bf16, norms = f32.cpu().numpy(), bf16.float().cpu().numpy(), norms.cpu().numpy()
    D = op.dim
    nb = 4 ** op.t
    for i in range(rd.n):
        x = oracle.embed(rd.read(i), op)
        g = f32[i, :D] + 1j * f32[i, D:]
        nx = np.linalg.norm(x)
        assert np.abs(g - x).max() <= 1e-5 * nx
        assert norms[i, 0] == pytest.approx(nx ** 2, rel=1e-5)
        for k in range(op.m):
            assert norms[i, 1 + k] == pytest.approx(np.sum(np.abs(x[k * nb:(k + 1) * nb]) ** 2), rel=1e-5, abs=1e-4)
        xn = x / nx
        gb = bf16[i, :D] + 1j * bf16[i, D:]
        assert np.abs(gb - xn).max() <= 2 ** -8 * max(np.abs(xn).max(), 1e-30)


def test_encode_reads_errors(lib):
    op = oracle.Params()
    seqs = np.frombuffer(b"ACGT" * 100, dtype=np.uint8).copy()
    lib.rope_encode_reads(gparams(op), dev(seqs), dev(np.array([0, 100, 400], np.int64)))
    with pytest.raises(lib.RopeError) as e:
        lib.rope_sync_status()
    assert e.value.status == 1  # read shorter than N
    seqs[250] = ord("X")
    lib.rope_encode_reads(gparams(op), dev(seqs), dev(np.array([0, 200, 400], np.int64)))
    with pytest.raises(lib.RopeError) as e:
        lib.rope_sync_status()
    assert e.value.status == 2
    with pytest.raises(lib.RopeError):
        lib.rope_encode_reads(gparams(op, s=9), dev(seqs), dev(np.array([0, 200], np.int64)))


# ---------------------------------------------------------------- index and a4

@pytest.mark.parametrize("pp", [dict(s=4, m=2, t=2, variant=1, N=150, stride=1),
                                dict(s=4, m=4, t=2, variant=1, N=150, stride=1),
                                dict(s=3, m=2, t=3, variant=0, N=90, stride=3),
                                dict(s=2, m=1, t=1, variant=0, N=200, stride=8),
                                dict(s=4, m=2, t=2, variant=1, N=150, stride=1, score_mode=1)])
def test_index_windows_and_norms(lib, pp):
    ref = synth.markov_ref(40_000, 0.41, 11, 0.05, 0.05)
    op = oracle.Params(**pp)
    idx = lib.rope_encode_reference(gparams(op), dev(ref))
    W = idx.n_windows
    assert W == oracle.n_windows(len(ref), op.N, op.stride)
    for j0, cnt in ((0, 700), (W - 333, 333), (1234, 1)):
        got = lib.rope_window_embeddings(idx, j0, cnt).cpu().numpy()
        want = oracle.windows_direct(ref, op, j0, cnt)
        D = op.dim
        g = got[:, :D] + 1j * got[:, D:]
        nrm = np.linalg.norm(want, axis=1, keepdims=True)
        assert np.all(np.abs(g - want) <= 1e-5 * nrm + 1e-6)
    inv = idx.inv_norm().cpu().numpy()
    sel = np.r_[0:50, W // 2:W // 2 + 50, W - 50:W]
    for j in sel:
        c = oracle.windows_direct(ref, op, int(j), 1)[0]
        n2 = np.sum(np.abs(c) ** 2)
        assert inv[j] == pytest.approx(1 / np.sqrt(n2), rel=2e-7) if n2 > 0 else inv[j] == 0
    idx.free()


# ---------------------------------------------------------------- a5: dense scores

def _dense_case(lib, cfg1, cfg1_gpu, precision, j0, cnt, nr):
    op, ref, rd = cfg1["op"], cfg1["ref"], cfg1["rd"]
    g = cfg1_gpu
    got = lib.rope_score_dense(g["idx"], g["f32"][:nr], g["bf16"][:nr], g["norms"][:nr], j0, cnt,
                               precision=precision)
    lib.rope_sync_status()
    got = got.cpu().numpy().astype(np.float64)
    wins = oracle.windows_direct(ref, op, j0, cnt)
    want = np.empty((nr, cnt))
    for i in range(nr):
        x = oracle.embed(rd.read(i), op)
        for j in range(cnt):
            want[i, j] = oracle.fidelity(x, wins[j])
    return got, want


@pytest.mark.parametrize("j0,cnt,nr", [(0, 2100, 256), (97_000, 2851, 37), (31, 1, 5)])
def test_dense_fp32_parity(lib, cfg1, cfg1_gpu, j0, cnt, nr):
    got, want = _dense_case(lib, cfg1, cfg1_gpu, "fp32", j0, cnt, nr)
    assert not np.isnan(got).any()
    assert np.all(np.abs(got - want) <= f32_tol(want)), np.abs(got - want).max()


def _bf16_error_summary(tag, got, want):
    """Observed BF16 error next to its bound: largest relative error where
    fid >= 0.16 (where the bound is the relative 2e-2) and largest absolute
    error below (where the sqrt term of the bound is the looser one)."""
    err = np.abs(got - want)
    hi = want >= 0.16
    rel_hi = (err[hi] / want[hi]).max() if hi.any() else float("nan")
    abs_lo = err[~hi].max() if (~hi).any() else float("nan")
    frac = (err / bf16_tol(want)).max()
    print(f"BF16-ERR {tag}: n={err.size} fid>=0.16: {int(hi.sum())} max rel {rel_hi:.3e}; "
          f"fid<0.16: max abs {abs_lo:.3e}; max err/bound {frac:.3f}")


@pytest.mark.parametrize("j0,cnt,nr", [(0, 2100, 256), (97_000, 2851, 37), (31, 1, 5)])
def test_dense_bf16_parity(lib, cfg1, cfg1_gpu, j0, cnt, nr):
    got, want = _dense_case(lib, cfg1, cfg1_gpu, "bf16", j0, cnt, nr)
    assert not np.isnan(got).any()
    _bf16_error_summary(f"dense j0={j0} cnt={cnt} reads={nr}", got, want)
    err = np.abs(got - want)
    assert np.all(err <= bf16_tol(want)), (err.max(), (err / np.maximum(want, 1e-9)).max())


@pytest.mark.parametrize("precision", ["bf16", "fp32"])
@pytest.mark.parametrize("j0,cnt,nr", [(1000, 17, 513), (50_000, 700, 640)])
def test_dense_parity_several_read_groups(lib, cfg1_wide, precision, j0, cnt, nr):
    """More than two 256-read groups of the tensor-core scan (the last ragged),
    each compared element by element with the oracle."""
    host, g = cfg1_wide
    got, want = _dense_case(lib, host, g, precision, j0, cnt, nr)
    assert not np.isnan(got).any()
    err = np.abs(got - want)
    if precision == "bf16":
        _bf16_error_summary(f"dense j0={j0} cnt={cnt} reads={nr}", got, want)
        assert np.all(err <= bf16_tol(want)), (err.max(), (err / np.maximum(want, 1e-9)).max())
    else:
        assert np.all(err <= f32_tol(want)), err.max()


# ---------------------------------------------------------------- a5-a7: top-k

def _check_top1(gw, ow, os_, tol_fn):
    """The reported best window is the oracle's best wherever the oracle's best
    beats its second by more than the tolerance (there it is unique); returns
    the mask of those reads."""
    clear = os_[:, 0] - os_[:, 1] > tol_fn(os_[:, 0])
    bad = np.nonzero(clear & (gw[:, 0] != ow[:, 0]))[0]
    assert bad.size == 0, (bad[:10], gw[bad[:10], 0], ow[bad[:10], 0])
    return clear


def test_topk_fp32_config1(lib, cfg1, cfg1_gpu):
    g = cfg1_gpu
    gw, gs = lib.rope_score_topk(g["idx"], g["f32"], None, g["norms"], k=8, precision="fp32")
    lib.rope_sync_status()
    gw, gs = gw.cpu().numpy(), gs.cpu().numpy().astype(np.float64)
    check_topk(cfg1["ref"], cfg1["rd"], cfg1["op"], gw, gs, cfg1["ow"], cfg1["os"], 8, f32_tol)
    assert _check_top1(gw, cfg1["ow"], cfg1["os"], f32_tol).mean() > 0.9


def test_topk_bf16_rescored_config1(lib, cfg1, cfg1_gpu):
    g = cfg1_gpu
    gw, gs = lib.rope_score_topk(g["idx"], g["f32"], g["bf16"], g["norms"], k=8, precision="bf16", rescore=1)
    lib.rope_sync_status()
    gw, gs = gw.cpu().numpy(), gs.cpu().numpy().astype(np.float64)
    check_topk(cfg1["ref"], cfg1["rd"], cfg1["op"], gw, gs, cfg1["ow"], cfg1["os"], 8, bf16_tol, f32_tol)
    # the BF16 scan only proposes candidates; once re-scored the top-1 is
    # decided in FP32, so it must be exact wherever the FP32 tolerance clears it
    assert _check_top1(gw, cfg1["ow"], cfg1["os"], f32_tol).mean() > 0.9


def test_topk_bf16_raw_config1(lib, cfg1, cfg1_gpu):
    g = cfg1_gpu
    gw, gs = lib.rope_score_topk(g["idx"], g["f32"], g["bf16"], g["norms"], k=8, precision="bf16", rescore=0)
    lib.rope_sync_status()
    gw, gs = gw.cpu().numpy(), gs.cpu().numpy().astype(np.float64)
    check_topk(cfg1["ref"], cfg1["rd"], cfg1["op"], gw, gs, cfg1["ow"], cfg1["os"], 8, bf16_tol)
    # raw BF16 scores decide the order: exact only where the gap exceeds the
    # BF16 tolerance (a minority here: a window one letter off the planted
    # start typically scores within 1% of it)
    _check_top1(gw, cfg1["ow"], cfg1["os"], bf16_tol)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_topk_planted_accuracy(lib, cfg1, cfg1_gpu, precision):
    """Planted loci: wherever the oracle's top-1 is clear of its second by the
    tolerance, the GPU finds exactly the oracle's window, so it hits the
    planted locus exactly when the oracle does; elsewhere (near ties) the two
    may pick different windows of equal score."""
    g = cfg1_gpu
    gw, _ = lib.rope_score_topk(g["idx"], g["f32"], g["bf16"], g["norms"], k=1, precision=precision)
    gw = gw.cpu().numpy()
    hit = np.abs(gw[:, 0] - cfg1["rd"].true_pos) < 150
    ora = np.abs(cfg1["ow"][:, 0] - cfg1["rd"].true_pos) < 150
    clear = _check_top1(gw, cfg1["ow"], cfg1["os"], f32_tol)  # BF16 results are re-scored in FP32
    assert np.array_equal(hit[clear], ora[clear])
    assert hit.mean() >= 0.97
    assert abs(hit.mean() - ora.mean()) <= (~clear).sum() / 256 + 1e-12


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("sep,k,nr_req", [(0, 3, 1), (150, 8, 0), (1000, 5, 5), (0, 32, 3)])
def test_topk_sep_ranges(lib, precision, sep, k, nr_req):
    ref = synth.markov_ref(60_000, 0.41, 21, 0.05, 0.05)
    rd = synth.reads(ref, 70, seed=22)
    op = oracle.Params(N=150)
    ow, os_ = oracle.score_topk(ref, rd.seqs, rd.offsets, op, k=k + 1, sep=sep)
    p = gparams(op)
    idx = lib.rope_encode_reference(p, dev(ref))
    f32, bf16, norms = lib.rope_encode_reads(p, dev(rd.seqs), dev(rd.offsets))
    gw, gs = lib.rope_score_topk(idx, f32, bf16, norms, k=k, sep=sep, precision=precision, n_ranges=nr_req,
                                 rescore=1 if precision == "bf16" else 0)
    lib.rope_sync_status()
    gw, gs = gw.cpu().numpy(), gs.cpu().numpy().astype(np.float64)
    if sep:
        for row in gw:
            b = row[row >= 0] // sep
            assert len(set(b.tolist())) == len(b)
    check_topk(ref, rd, op, gw, gs, ow, os_, k, f32_tol if precision == "fp32" else bf16_tol, f32_tol, sep=sep)
    idx.free()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_topk_subrange_and_fill(lib, precision):
    ref = synth.uniform_ref(3000, 31)
    rd = synth.reads(ref, 9, seed=32)
    op = oracle.Params(N=150)
    p = gparams(op)
    idx = lib.rope_encode_reference(p, dev(ref))
    f32, bf16, norms = lib.rope_encode_reads(p, dev(rd.seqs), dev(rd.offsets))
    # 5 windows only, k = 8: three (-1, -inf) fills
    gw, gs = lib.rope_score_topk(idx, f32, bf16, norms, k=8, precision=precision, j_begin=1000, j_end=1005)
    gw, gs = gw.cpu().numpy(), gs.cpu().numpy()
    ow, os_ = oracle.score_topk(ref, rd.seqs, rd.offsets, op, k=8, j_begin=1000, j_end=1005)
    assert np.all(gw[:, 5:] == -1) and np.all(np.isneginf(gs[:, 5:]))
    assert np.array_equal(np.sort(gw[:, :5], axis=1), np.sort(ow[:, :5], axis=1))
    tol = f32_tol(os_[:, :5])
    assert np.all(np.abs(np.sort(gs[:, :5], axis=1) - np.sort(os_[:, :5], axis=1)) <= tol)
    # empty range
    gw, gs = lib.rope_score_topk(idx, f32, bf16, norms, k=4, precision=precision, j_begin=10, j_end=10)
    assert np.all(gw.cpu().numpy() == -1)
    lib.rope_sync_status()
    idx.free()


def test_topk_per_band_fp32(lib):
    ref = synth.uniform_ref(20_000, 41)
    rd = synth.reads(ref, 40, seed=42)
    op = oracle.Params(s=4, m=4, t=2, variant=1, N=150, score_mode=1)
    ow, os_ = oracle.score_topk(ref, rd.seqs, rd.offsets, op, k=6)
    p = gparams(op)
    idx = lib.rope_encode_reference(p, dev(ref))
    f32, bf16, norms = lib.rope_encode_reads(p, dev(rd.seqs), dev(rd.offsets))
    gw, gs = lib.rope_score_topk(idx, f32, None, norms, k=5, precision="fp32")
    lib.rope_sync_status()
    check_topk(ref, rd, op, gw.cpu().numpy(), gs.cpu().numpy().astype(np.float64), ow, os_, 5, f32_tol)
    with pytest.raises(lib.RopeError):
        lib.rope_score_topk(idx, f32, bf16, norms, k=5, precision="bf16")
    idx.free()


@pytest.mark.parametrize("pp", [dict(s=4, m=4, t=2, variant=1, N=150, stride=1),
                                dict(s=4, m=2, t=2, variant=1, N=400, stride=8),
                                dict(s=3, m=2, t=2, variant=0, N=64, stride=3)])
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_topk_other_shapes(lib, pp, precision):
    ref = synth.markov_ref(30_000, 0.41, 51, 0.05, 0.05)
    rd = synth.reads(ref, 45, seed=52, length=pp["N"])
    op = oracle.Params(**pp)
    ow, os_ = oracle.score_topk(ref, rd.seqs, rd.offsets, op, k=5)
    p = gparams(op)
    idx = lib.rope_encode_reference(p, dev(ref))
    f32, bf16, norms = lib.rope_encode_reads(p, dev(rd.seqs), dev(rd.offsets))
    gw, gs = lib.rope_score_topk(idx, f32, bf16, norms, k=4, precision=precision)
    lib.rope_sync_status()
    check_topk(ref, rd, op, gw.cpu().numpy(), gs.cpu().numpy().astype(np.float64), ow, os_, 4,
               f32_tol if precision == "fp32" else bf16_tol, f32_tol)
    idx.free()


def test_zero_norm_windows(lib):
    """§3.3: all-A and periodic windows encode to zero; their fidelity is 0."""
    ref = np.frombuffer(b"A" * 400 + b"ACGT" * 100 + b"A" * 400, dtype=np.uint8).copy()
    rd = synth.reads(synth.uniform_ref(2000, 61), 4, seed=62, length=40)
    op = oracle.Params(s=1, m=1, t=1, variant=0, N=40)
    p = gparams(op)
    idx = lib.rope_encode_reference(p, dev(ref))
    f32, bf16, norms = lib.rope_encode_reads(p, dev(rd.seqs), dev(rd.offsets))
    gw, gs = lib.rope_score_topk(idx, f32, None, norms, k=3, precision="fp32")
    dense = lib.rope_score_dense(idx, f32, None, norms, 0, idx.n_windows, precision="fp32").cpu().numpy()
    lib.rope_sync_status()
    assert np.all(dense[:, 0] == 0) and np.all(dense[:, 400] == 0)
    ow, os_ = oracle.score_topk(ref, rd.seqs, rd.offsets, op, k=4)
    check_topk(ref, rd, op, gw.cpu().numpy(), gs.cpu().numpy().astype(np.float64), ow, os_, 3, f32_tol)
    idx.free()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_map_equals_encode_and_score(lib, cfg1, cfg1_gpu, precision):
    g = cfg1_gpu
    w1, s1 = lib.rope_map(g["idx"], g["seqs"], g["offs"], k=8, precision=precision)
    w2, s2 = lib.rope_score_topk(g["idx"], g["f32"], g["bf16"], g["norms"], k=8, precision=precision)
    lib.rope_sync_status()
    assert torch.equal(w1, w2) and torch.equal(s1, s2)


def test_invalid_arguments(lib, cfg1_gpu):
    g = cfg1_gpu
    with pytest.raises(lib.RopeError):
        lib.rope_score_topk(g["idx"], g["f32"], g["bf16"], g["norms"], k=0)
    with pytest.raises(lib.RopeError):
        lib.rope_score_topk(g["idx"], g["f32"], g["bf16"], g["norms"], k=33)
    with pytest.raises(lib.RopeError):
        lib.rope_score_topk(g["idx"], g["f32"], None, g["norms"], k=8, precision="bf16")
    with pytest.raises(lib.RopeError):
        lib.rope_encode_reference(lib.Params(window_len=5000), dev(synth.uniform_ref(1000, 1)))
