"""Multi-GPU sharding of the scan (§2.8: segments are processed independently
and recombined).

Two layouts:
  * reads sharded, index replicated: every rank maps its own reads; no data
    exchange (what bench.py --gpus N does).
  * windows sharded: rank r scans the window range ``window_shards(...)[r]``
    for all reads; the per-rank top-k lists are gathered to every rank and
    merged on the host by ``rope_merge_shards_host`` (same order and bucket
    rule as a single scan).
"""
from __future__ import annotations

import numpy as np
import torch

from . import rotormap as rm


def window_shards(n_windows: int, world: int, align: int = 1) -> list[tuple[int, int]]:
    """Split [0, n_windows) into `world` contiguous ranges whose boundaries are
    multiples of `align` windows (e.g. the bucket width in windows)."""
    per = -(-n_windows // world)
    per = -(-per // align) * align
    out = []
    for r in range(world):
        b = min(r * per, n_windows)
        out.append((b, min(b + per, n_windows)))
    return out


def gather_merge(win: torch.Tensor, score: torch.Tensor, k_out: int, sep: int = 0, group=None):
    """All-gather each rank's [n_reads, k] top-k (any device) and merge on the
    host. Returns numpy (starts [n, k_out], scores [n, k_out]) on every rank."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    backend = dist.get_backend(group)
    dev = win.device if backend == "nccl" else torch.device("cpu")
    w = win.to(dev).contiguous()
    s = score.to(dev).contiguous()
    ws = [torch.empty_like(w) for _ in range(world)]
    ss = [torch.empty_like(s) for _ in range(world)]
    dist.all_gather(ws, w, group=group)
    dist.all_gather(ss, s, group=group)
    W = np.stack([x.cpu().numpy() for x in ws])
    S = np.stack([x.cpu().numpy() for x in ss])
    return rm.rope_merge_shards_host(W, S, k_out, sep)
