"""Length ladder (reads of many lengths, §3.5 head mapping per read): bucket
choice bit-exact, every bucket's top-k against the FP64 oracle at that
bucket's window length, and the same results as rope_map on the bucket's own
index."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from _parity import bf16_tol, check_topk, dev, f32_tol

pytestmark = pytest.mark.gpu

STRIDE = 8


def expected_len(n, n_min=100, n_max=3000, spo=8):
    """Largest floor(n_min * 2^(j/spo)) <= min(n, n_max), or -1."""
    best, j = -1, 0
    while True:
        v = math.floor(n_min * 2 ** (j / spo))
        if v > n_max:
            return best
        if v <= n:
            best = v
        j += 1


@pytest.fixture(scope="module", params=[(2, 240), (4, 80)], ids=["d64", "d128"])
def ladder_case(request, lib):
    m, n_reads = request.param
    ref = synth.markov_ref(400_000, 0.41, 5, 0.025, 0.025, 0.0)
    # lognormal lengths (median 600, sigma 0.7), 8% errors split 40% substitutions / 60% indels
    rd = synth.reads(ref, n_reads, seed=6 + m, length=600, sub_rate=0.032, indel_rate=0.048, lognormal_sigma=0.7,
                     len_min=60, len_max=3000)
    p = lib.Params(s=4, m=m, t=2, variant=1, window_len=100, stride=STRIDE)
    lad = lib.rope_ladder_create(p, dev(ref), 100, 3000, 8)
    yield dict(ref=ref, rd=rd, p=p, lad=lad, m=m, seqs=dev(rd.seqs), offs=dev(rd.offsets))
    lad.free()


def test_ladder_lengths(lib, ladder_case):
    lad = ladder_case["lad"]
    want = sorted({math.floor(100 * 2 ** (j / 8)) for j in range(64) if math.floor(100 * 2 ** (j / 8)) <= 3000})
    assert lad.lengths == want
    for j in (0, len(want) - 1):
        assert lad.bucket(j).n_windows == (len(ladder_case["ref"]) - want[j]) // STRIDE + 1


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_ladder_against_oracle(lib, ladder_case, precision):
    c = ladder_case
    rd, ref = c["rd"], c["ref"]
    k = 4
    w, s, used = lib.rope_ladder_map(c["lad"], c["seqs"], c["offs"], k=k, precision=precision)
    lib.rope_sync_status()
    w, s, used = w.cpu().numpy(), s.cpu().numpy().astype(np.float64), used.cpu().numpy()
    want = np.array([expected_len(int(n)) for n in rd.lengths])
    assert np.array_equal(used, want)
    short = want < 0
    assert (~short).any()
    assert (w[short] == -1).all() and np.isneginf(s[short]).all()
    hits, longs = 0, 0
    for N in np.unique(want[~short]):
        sel = np.nonzero(want == N)[0]
        sub = rd.subset(sel)
        op = oracle.Params(s=4, m=c["m"], t=2, variant=1, N=int(N), stride=STRIDE)
        ow, os_ = oracle.score_topk(ref, sub.seqs, sub.offsets, op, k=k + 1)
        score_tol = f32_tol
        tol = f32_tol if precision == "fp32" else bf16_tol
        check_topk(ref, sub, op, w[sel], s[sel], ow, os_, k, tol, score_tol)
        if N >= 500:
            longs += len(sel)
            hits += int((np.abs(w[sel, 0] - sub.true_pos) < N).sum())
    print(f"top-1 at the planted locus, heads >= 500 bp: {hits}/{longs}")
    assert longs == 0 or hits >= 0.5 * longs


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_ladder_equals_bucket_map(lib, ladder_case, precision):
    c = ladder_case
    rd = c["rd"]
    w, s, used = lib.rope_ladder_map(c["lad"], c["seqs"], c["offs"], k=4, precision=precision)
    used = used.cpu().numpy()
    lens = c["lad"].lengths
    # the two most populated buckets
    vals, cnt = np.unique(used[used > 0], return_counts=True)
    for N in vals[np.argsort(-cnt)[:2]]:
        sel = np.nonzero(used == N)[0]
        sub = rd.subset(sel)
        idx = c["lad"].bucket(lens.index(int(N)))
        bw, bs = lib.rope_map(idx, dev(sub.seqs), dev(sub.offsets), k=4, precision=precision)
        lib.rope_sync_status()
        assert torch.equal(bw.cpu(), w[torch.from_numpy(sel).cuda()].cpu())
        assert torch.equal(bs.cpu(), s[torch.from_numpy(sel).cuda()].cpu())


def test_ladder_empty_and_all_short(lib, ladder_case):
    c = ladder_case
    offs = torch.zeros(1, dtype=torch.int64, device="cuda")
    w, s, used = lib.rope_ladder_map(c["lad"], c["seqs"], offs, k=3)
    assert w.shape == (0, 3)
    short = synth.reads(c["ref"], 5, seed=99, length=50)
    w, s, used = lib.rope_ladder_map(c["lad"], dev(short.seqs), dev(short.offsets), k=3)
    lib.rope_sync_status()
    assert (w.cpu() == -1).all() and torch.isneginf(s.cpu()).all() and (used.cpu() == -1).all()


def test_ladder_graph_replay(lib, ladder_case):
    """The second call with the same bucket sizes, buffers and options captures
    the buckets' work in a CUDA graph and later calls replay it: every call
    gives the first (eager) call's results, also after the reads change."""
    c = ladder_case
    n = c["rd"].n
    out = (torch.empty((n, 4), dtype=torch.int64, device="cuda"), torch.empty((n, 4), dtype=torch.float32,
                                                                              device="cuda"),
           torch.empty((n,), dtype=torch.int32, device="cuda"))
    runs = []
    for _ in range(4):
        lib.rope_ladder_map(c["lad"], c["seqs"], c["offs"], k=4, out=out)
        lib.rope_sync_status()
        runs.append(tuple(t.cpu().clone() for t in out))
    for r in runs[1:]:
        assert all(torch.equal(a, b) for a, b in zip(runs[0], r))
    assert c["lad"].graph_count() >= 1  # the buckets' work was captured
    # same lengths (so the same bucket sizes), other letters: the replay sees the new reads
    other = synth.reads(c["ref"], n, seed=77, length=600, sub_rate=0.032, indel_rate=0.048, lognormal_sigma=0.7,
                        len_min=60, len_max=3000)
    seqs2 = c["seqs"].clone()
    for i in range(n):
        a, b = int(c["rd"].offsets[i]), int(c["rd"].offsets[i + 1])
        o = int(other.offsets[i])
        m = min(b - a, int(other.offsets[i + 1]) - o)
        seqs2[a:a + m] = torch.from_numpy(other.seqs[o:o + m]).cuda()
    c["seqs"].copy_(seqs2)  # in place: the captured pointers stay valid
    lib.rope_ladder_map(c["lad"], c["seqs"], c["offs"], k=4, out=out)
    lib.rope_sync_status()
    replay = tuple(t.cpu().clone() for t in out)
    fresh = lib.rope_ladder_map(c["lad"], c["seqs"], c["offs"], k=4)  # new output buffers: eager
    lib.rope_sync_status()
    assert all(torch.equal(a, b.cpu()) for a, b in zip(replay, fresh))
    assert not torch.equal(replay[0], runs[0][0])
