"""Window-range sharding on the CUDA path: the window ranges of
shard.window_shards are scanned one after another by rope_score_topk on this
GPU (what each rank of a window-sharded run does), their per-shard top-k lists
are merged by rope_merge_shards_host. With sep > 0 the shards are aligned to the
bucket width, as the sharded layout requires.

* FP32 scan, and BF16 scan without re-scoring: the merged result equals the
  unsharded scan exactly (windows and scores): the union of per-shard top-k
  lists holds the overall top-k, and a window's score does not depend on the
  range it was scanned in.
* BF16 scan with FP32 re-scoring: each shard re-scores its own best raw
  candidates, a superset of the unsharded call's candidates (which are the
  best raw candidates overall), so the merged list is the FP32 top-k of a
  superset: score by score it is at least the unsharded one, and equal
  wherever both report the same window.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case(lib):
    ref = synth.markov_ref(300_000, 0.41, 71, 0.05, 0.05)
    rd = synth.reads(ref, 700, seed=72)
    p = lib.Params(s=4, m=2, t=2, variant=1, window_len=150)
    idx = lib.rope_encode_reference(p, torch.from_numpy(ref).cuda())
    enc = lib.rope_encode_reads(p, torch.from_numpy(rd.seqs).cuda(), torch.from_numpy(rd.offsets).cuda())
    lib.rope_sync_status()
    yield idx, enc
    idx.free()


@pytest.mark.parametrize("precision,rescore", [("fp32", 0), ("bf16", 0), ("bf16", 1)])
@pytest.mark.parametrize("world,sep,k", [(2, 0, 8), (3, 0, 5), (4, 1000, 8)])
def test_sharded_scan_matches_unsharded(lib, case, precision, rescore, world, sep, k):
    from paper_2603_22245_gb300 import shard

    idx, (f32, bf16, norms) = case
    W = idx.n_windows
    fw, fs = lib.rope_score_topk(idx, f32, bf16, norms, k=k, sep=sep, precision=precision, rescore=rescore)
    fw, fs = fw.cpu().numpy(), fs.cpu().numpy()
    ws, ss = [], []
    for b, e in shard.window_shards(W, world, align=max(sep, 1)):
        w, s = lib.rope_score_topk(idx, f32, bf16, norms, k=k, sep=sep, precision=precision, rescore=rescore,
                                   j_begin=b, j_end=e)
        ws.append(w.cpu().numpy())
        ss.append(s.cpu().numpy())
    lib.rope_sync_status()
    mw, ms = lib.rope_merge_shards_host(np.stack(ws), np.stack(ss), k, sep)
    if not rescore:
        assert np.array_equal(mw, fw)
        assert np.array_equal(ms, fs)
    else:
        assert np.all(ms >= fs)
        same = mw == fw
        assert np.array_equal(ms[same], fs[same])
