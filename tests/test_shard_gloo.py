"""Window-range sharding across two ranks (gloo, CPU): the gathered and merged
per-shard top-k equals the unsharded scan. Shard results come from the oracle
here (the merge is host code; the GPU scan of a range is checked elsewhere)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, sep, k, q):
    import torch
    import torch.distributed as dist

    import oracle
    import synth
    from paper_2603_22245_gb300 import shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ref = synth.markov_ref(30_000, 0.41, 5, 0.05, 0.05)
        rd = synth.reads(ref, 12, seed=6)
        op = oracle.Params(N=150)
        W = oracle.n_windows(len(ref), 150, 1)
        b, e = shard.window_shards(W, world, align=max(sep, 1))[rank]
        w, s = oracle.score_topk(ref, rd.seqs, rd.offsets, op, k=k, sep=sep, j_begin=b, j_end=e)
        mw, ms = shard.gather_merge(torch.from_numpy(w), torch.from_numpy(s.astype(np.float32)), k, sep)
        if rank == 0:
            fw, fs = oracle.score_topk(ref, rd.seqs, rd.offsets, op, k=k, sep=sep)
            q.put((np.array_equal(mw, fw), float(np.abs(ms - fs.astype(np.float32)).max())))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("sep,k", [(0, 6), (150, 5)])
def test_window_sharding_merge_equals_single_scan(sep, k):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, sep, k, q), nprocs=2, join=True, start_method="spawn")
    same, err = q.get(timeout=60)
    assert same and err == 0.0


def test_window_shards_cover():
    from paper_2603_22245_gb300 import shard

    for W, world, align in ((10, 3, 1), (99_851, 4, 150), (5, 8, 1)):
        rs = shard.window_shards(W, world, align)
        assert rs[0][0] == 0 and rs[-1][1] == W
        for (a, b), (c, d) in zip(rs, rs[1:]):
            assert b == c and (b % align == 0 or b == W)


def test_merge_host_ties_and_fill():
    from paper_2603_22245_gb300 import rotormap as rm

    W = np.array([[[5, 9, -1]], [[2, 7, 11]]], dtype=np.int64)
    S = np.array([[[0.5, 0.4, -np.inf]], [[0.5, 0.45, 0.1]]], dtype=np.float32)
    ow, os_ = rm.rope_merge_shards_host(W, S, 4)
    assert ow.tolist() == [[2, 5, 7, 9]]
    ow, os_ = rm.rope_merge_shards_host(W, S, 6, sep=4)  # buckets: 2->0, 5->1, 7->1, 9->2, 11->2
    assert ow.tolist() == [[2, 5, 9, -1, -1, -1]] and np.isneginf(os_[0, 3:]).all()
