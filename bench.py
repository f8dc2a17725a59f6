#!/usr/bin/env python
"""RotorMap hot-path benchmark: prints one JSON line.

Workload (default "markov100M"): a 100 Mbp order-2 Markov reference (GC 41%,
planted tandem repeats and segmental duplicates) and 1,000,000 planted 150 bp
reads (1% substitutions, 0.5% indels of geometric length), encoded with the
fine-tuned compact RoPE s=4, m=2, t=2 (d = 64 reals), every window of length
150 at stride 1 scored exhaustively, top-8 per read. A step maps one batch of
reads (default 131,072; 8 steps = the whole read set) through rope_map: read
encoding, the on-chip window recurrence fused with the BF16 tensor-core scan
and top-k, and FP32 re-scoring. The reference index is built once before the
timed region (the paper's "preloaded data").

  value       BF16 tensor-core read x window scores/s over all ranks
  fp32_plain  the FP32 CUDA-core scan on a read subset (same metric)
  fp8_option  the same steps with the E4M3 tensor-core scan (rate, top-1
              accuracy, scan roofline against twice the BF16 peak)
  refine      §3.4 refinement of the top-2 candidates of one batch (+-8
              letters, 2 x 4^8-bin encoding): rate and exact-start fraction
  top1_acc    fraction of planted reads whose top-1 window overlaps the truth
  e2e         the same metric through host buffers (H2D of the reads, D2H of
              the top-k) around every step
  roofline    the scan kernel (CUDA events around its launch) against the
              measured sustained BF16 tensor peak
  cpu_baseline the FP64 oracle on a bounded sample, on this host's cores

--impl reference times the FP64 oracle (the only reference implementation
of this path) on the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "read×window scores/s and reads/s, BF16-TC vs FP32 plain, at equal top-1 acc"
UNIT = "scores/s"

WORKLOADS = {
    "markov100M": dict(
        desc="100 Mbp order-2 Markov reference (GC 41%, 2.5% tandem repeats, 2.5% segmental duplicates), "
             "1M x 150 bp planted reads (1% sub, 0.5% indel geom p=0.7), fine-tuned compact RoPE s=4 m=2 t=2 "
             "(d=64), N=150, stride 1, exhaustive, top-8",
        L=100_000_000, gc=0.41, tandem=0.025, segdup=0.025, inter=0.0, ref_seed=3,
        n_reads=1_000_000, read_len=150, sub=0.01, indel=0.005, read_seed=4,
        s=4, m=2, t=2, variant=1, N=150, stride=1, k=8),
    "markov10M_lognormal": dict(
        desc="10 Mbp order-2 Markov reference (GC 41%, 2.5% tandem repeats, 2.5% segmental duplicates), 200k "
             "planted reads of lognormal length (median 2 kbp, sigma 0.7, clipped to 100-10000), 8% errors (3.2% "
             "sub, 4.8% indel geom p=0.7), d=64 (s=4 m=2 t=2 fine-tuned), stride 8, length ladder "
             "floor(100*2^(j/8)) <= 10 kbp (54 window lengths; each read mapped by its longest fitting head), top-8",
        L=10_000_000, gc=0.41, tandem=0.025, segdup=0.025, inter=0.0, ref_seed=5,
        n_reads=200_000, read_len=2000, sigma=0.7, len_min=100, len_max=10000, sub=0.032, indel=0.048,
        read_seed=6, s=4, m=2, t=2, variant=1, N=100, stride=8, k=8, ladder=(100, 10000, 8)),
    "markov10M_lognormal_d128": dict(
        desc="as markov10M_lognormal with d=128 (s=4 m=4 t=2 fine-tuned)",
        L=10_000_000, gc=0.41, tandem=0.025, segdup=0.025, inter=0.0, ref_seed=5,
        n_reads=200_000, read_len=2000, sigma=0.7, len_min=100, len_max=10000, sub=0.032, indel=0.048,
        read_seed=6, s=4, m=4, t=2, variant=1, N=100, stride=8, k=8, ladder=(100, 10000, 8)),
    "markov20M": dict(
        desc="20 Mbp order-2 Markov reference (GC 41%, 2.5% tandem repeats, 2.5% segmental duplicates), "
             "32768 x 150 bp planted reads (1% sub, 0.5% indel geom p=0.7), d=64, N=150, stride 1, top-8 "
             "(a one-batch case small enough for a full ncu capture of the scan)",
        L=20_000_000, gc=0.41, tandem=0.025, segdup=0.025, inter=0.0, ref_seed=3,
        n_reads=32768, read_len=150, sub=0.01, indel=0.005, read_seed=4,
        s=4, m=2, t=2, variant=1, N=150, stride=1, k=8),
    "human3G": dict(
        desc="3.1 Gbp human-shaped order-2 Markov genome (GC 41%, 50% interspersed repeats), 100k x 150 bp planted "
             "reads (1% sub, 0.5% indel geom p=0.7), d=64 (s=4 m=2 t=2 fine-tuned), N=150, stride 1, exhaustive, top-8",
        L=3_100_000_000, gc=0.41, tandem=0.0, segdup=0.0, inter=0.50, ref_seed=7,
        n_reads=100_000, read_len=150, sub=0.01, indel=0.005, read_seed=8,
        s=4, m=2, t=2, variant=1, N=150, stride=1, k=8, batch=16_384, fp32_reads=128),
    "maize2300M": dict(
        desc="2.3 Gbp maize-shaped order-2 Markov genome (GC 47%, 85% interspersed repeats), 100k x 150 bp planted "
             "reads (1% sub, 0.5% indel geom p=0.7), d=64 (s=4 m=2 t=2 fine-tuned), N=150, stride 1, exhaustive, top-8",
        L=2_300_000_000, gc=0.47, tandem=0.0, segdup=0.0, inter=0.85, ref_seed=8,
        n_reads=100_000, read_len=150, sub=0.01, indel=0.005, read_seed=9,
        s=4, m=2, t=2, variant=1, N=150, stride=1, k=8, batch=16_384, fp32_reads=128),
    "human3G_20k": dict(
        desc="3.1 Gbp human-shaped order-2 Markov genome (GC 41%, 50% interspersed repeats), 96k planted 20 kbp reads "
             "at 15% errors (5% substitutions, 10% indel events of geometric length p=0.7), every other read "
             "reverse-complemented, mapped on both strands; fine-tuned compact RoPE s=8 m=4 t=4 (1024 complex "
             "dimensions, d=2048), window N=20000, step 1250 (the paper's long-read configuration), materialised "
             "index scored by the BF16 tcgen05 GEMM, FP32 re-scoring, top-8",
        L=3_100_000_000, gc=0.41, tandem=0.0, segdup=0.0, inter=0.50, ref_seed=7,
        n_reads=96_000, read_len=20000, sub=0.05, indel=0.10, read_seed=10,
        s=8, m=4, t=4, variant=1, N=20000, stride=1250, k=8, strands=True, batch=24_000, cpu_reads=16,
        cpu_windows=3000, fp32_reads=512),
    "markov300M_20k": dict(
        desc="300 Mbp order-2 Markov reference (GC 41%, 2.5% tandem repeats, 2.5% segmental duplicates), 8192 planted "
             "20 kbp reads at 15% errors, both strands, s=8 m=4 t=4 (d=2048), N=20000, step 1250, top-8 (a one-batch "
             "case of the long-read configuration small enough for ncu captures)",
        L=300_000_000, gc=0.41, tandem=0.025, segdup=0.025, inter=0.0, ref_seed=3,
        n_reads=8192, read_len=20000, sub=0.05, indel=0.10, read_seed=11,
        s=8, m=4, t=4, variant=1, N=20000, stride=1250, k=8, strands=True, batch=8192, cpu_reads=16,
        cpu_windows=3000, fp32_reads=512),
    "human30M_20k_thr": dict(
        desc="threshold regime (multi-locus output) on a 30 Mbp human-shaped order-2 Markov genome (GC 41%, 50% "
             "interspersed repeats), 2000 planted 20 kbp reads at 15% per-letter edits split evenly between "
             "substitutions, insertions and deletions (the thresholds' own mutation model), s=8 m=4 t=4 (d=2048), "
             "N=20000, step 1250; per-window thresholds from 8 mutated copies for rates 0.15, 0.20, 0.25; every "
             "(read, window) pair reaching its window's threshold",
        L=30_000_000, gc=0.41, tandem=0.0, segdup=0.0, inter=0.50, ref_seed=12,
        n_reads=2000, read_len=20000, sub=0.05, indel=0.10, geom_p=1.0, read_seed=13,
        s=8, m=4, t=4, variant=1, N=20000, stride=1250, k=8, threshold=dict(errs=[0.15, 0.20, 0.25], n_samples=8)),
    "markov10M_d128_thr": dict(
        desc="threshold regime on a 10 Mbp order-2 Markov reference (GC 41%, 2.5% tandem repeats, 2.5% segmental "
             "duplicates), 2000 planted 150 bp reads at 15% per-letter edits split evenly (substitutions, insertions, "
             "deletions), s=4 m=4 t=2 (d=128), N=150, stride 1; thresholds from 8 copies for rates 0.15, 0.20, 0.25",
        L=10_000_000, gc=0.41, tandem=0.025, segdup=0.025, inter=0.0, ref_seed=5,
        n_reads=2000, read_len=150, sub=0.05, indel=0.10, geom_p=1.0, read_seed=14,
        s=4, m=4, t=2, variant=1, N=150, stride=1, k=8, threshold=dict(errs=[0.15, 0.20, 0.25], n_samples=8)),
    "uniform100k": dict(
        desc="100 kbp uniform reference, 256 x 150 bp planted reads (1% sub, 0.5% indel), d=64, stride 1, top-8",
        L=100_000, gc=None, ref_seed=1, n_reads=256, read_len=150, sub=0.01, indel=0.005, read_seed=2,
        s=4, m=2, t=2, variant=1, N=150, stride=1, k=8),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="markov100M", choices=sorted(WORKLOADS))
    ap.add_argument("--batch", type=int, default=0, help="reads per step (0: the workload's default)")
    ap.add_argument("--fp32-reads", type=int, default=4096)
    ap.add_argument("--fp8-steps", type=int, default=2)
    ap.add_argument("--refine-radius", type=int, default=8)
    ap.add_argument("--scan-variant", type=int, default=-1,
                    help="pin the scan's tile variant (and 16 items per SM) instead of the library's choice")
    ap.add_argument("--e2e-steps", type=int, default=-1, help="end-to-end steps (-1: as many as --steps)")
    ap.add_argument("--cpu-reads", type=int, default=32)
    ap.add_argument("--cpu-windows", type=int, default=1_000_000)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--rerank-train-reads", type=int, default=65536)
    ap.add_argument("--rerank-eval-reads", type=int, default=32768)
    return ap.parse_args()


def make_inputs(wl, rank):
    import synth

    if wl.get("gc") is None:
        ref = synth.uniform_ref(wl["L"], wl["ref_seed"])
    else:
        ref = synth.markov_ref(wl["L"], wl["gc"], wl["ref_seed"], wl["tandem"], wl["segdup"], wl["inter"])
    rd = synth.reads(ref, wl["n_reads"], seed=wl["read_seed"] + 1000 * rank, length=wl["read_len"],
                     sub_rate=wl["sub"], indel_rate=wl["indel"], geom_p=wl.get("geom_p", 0.7),
                     lognormal_sigma=wl.get("sigma"), len_min=wl.get("len_min", 100),
                     len_max=wl.get("len_max", 10000))
    if wl.get("strands"):
        rd = reverse_every_other(rd)
    return ref, rd


_COMPLEMENT = np.zeros(256, dtype=np.uint8)
for _a, _b in zip(b"ACGTacgt", b"TGCAtgca"):
    _COMPLEMENT[_a] = _b


def reverse_every_other(rd):
    """Reads of both strands: every odd read is replaced by its reverse
    complement (the locus it came from is unchanged; its strand is 1)."""
    seqs = rd.seqs.copy()
    for i in range(1, rd.n, 2):
        a, b = rd.offsets[i], rd.offsets[i + 1]
        seqs[a:b] = _COMPLEMENT[rd.seqs[a:b][::-1]]
    rd.seqs = seqs
    return rd


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


TRAFFIC_RECORDS = {  # workload -> (ncu traffic record, kernel source it was taken on, batch it is scaled to)
    "markov100M": ("scan_tc_traffic.json", "rope_scan_tc.cu", 131072),
    "human3G_20k": ("gemm_tc_traffic.json", "rope_dense.cu", 24000),
}


def traffic_record(workload, batch):
    """DRAM bytes per scan launch from the committed ncu summary, if it was
    taken on the current kernel source and scaled to this launch (else None)."""
    if workload not in TRAFFIC_RECORDS:
        return None
    name, kernel, b = TRAFFIC_RECORDS[workload]
    path = os.path.join(ROOT, "profiles", name)
    src = os.path.join(ROOT, "paper_2603_22245_gb300", "csrc", kernel)
    if batch != b or not os.path.exists(path):
        return None
    rec = json.load(open(path))
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return rec if rec.get("kernel_sha") == h else None


class Clocks:
    """nvidia-smi samples (200 ms) during the timed region."""

    def __init__(self, device_index: int):
        self.proc = None
        self.path = None
        self.dev = device_index

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline(ref, rd, wl, n_reads, n_windows):
    """The FP64 oracle, as it stands, on a bounded sample of the workload."""
    import oracle

    op = oracle.Params(s=wl["s"], m=wl["m"], t=wl["t"], variant=wl["variant"], N=wl["N"], stride=wl["stride"])
    W = oracle.n_windows(len(ref), wl["N"], wl["stride"])
    n_windows = min(n_windows, W)
    cores = oracle.max_threads()
    sub = rd.subset(np.arange(min(n_reads, rd.n)))
    t0 = time.perf_counter()
    oracle.score_topk(ref, sub.seqs, sub.offsets, op, k=wl["k"], j_begin=0, j_end=n_windows, n_threads=cores)
    dt = time.perf_counter() - t0
    # the oracle's full-DP Levenshtein distance (reranker labels) on all cores,
    # about 2e9 DP cells
    n_ld = max(16, int(2.25e9 // (wl["N"] * wl["N"])))
    rng = np.random.default_rng(0)
    ri = rng.integers(0, rd.n, n_ld)
    ws = rng.integers(0, len(ref) - wl["N"], n_ld)
    t0 = time.perf_counter()
    oracle.levenshtein_pairs(ref, rd.seqs, rd.offsets, ri, ws, wl["N"], n_threads=cores)
    dt_ld = time.perf_counter() - t0
    # the same scoring on one core, on an eighth of the sample (last: it sets
    # the oracle's thread count to 1)
    one = rd.subset(np.arange(max(1, sub.n // 8)))
    t0 = time.perf_counter()
    oracle.score_topk(ref, one.seqs, one.offsets, op, k=wl["k"], j_begin=0, j_end=n_windows, n_threads=1)
    dt1 = time.perf_counter() - t0
    return {"value": sub.n * n_windows / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{sub.n} reads x the first {n_windows} windows, exhaustive FP64 scoring + full sort",
            "seconds": dt,
            "single_thread": {"value": one.n * n_windows / dt1, "unit": UNIT, "cores": 1, "seconds": dt1,
                              "sample": f"{one.n} reads x the first {n_windows} windows"},
            "levenshtein": {"pairs_per_s": n_ld / dt_ld, "cores": cores, "seconds": dt_ld,
                            "sample": f"{n_ld} (read head, window) pairs of {wl['N']} letters, full DP"}}


def rerank_leg(rm, idx, ref, wl, args):
    """Learned reranker (outside the timed region): candidates k=16 (one per
    bucket of width N) of reads at 0-15% error, exact Levenshtein labels, 5
    AdamW epochs on the GPU, then on new reads: keep 2 of 16 by predicted
    distance vs by score, against the plain top-8."""
    import torch

    import synth
    from paper_2603_22245_gb300 import rerank

    K, N = 16, wl["N"]
    tr = synth.reads_mixed_error(ref, args.rerank_train_reads, seed=wl["read_seed"] + 500)
    te = synth.reads_mixed_error(ref, args.rerank_eval_reads, seed=wl["read_seed"] + 900)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X, t, valid, _ = rerank.training_set(idx, torch.from_numpy(tr.seqs).cuda(), torch.from_numpy(tr.offsets).cuda(),
                                         k=K)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    rr = rerank.Reranker(rerank.n_features(K, wl["m"]), 128, seed=11)
    losses = rerank.train(rr, X, t, valid, epochs=5, batch=4096, lr=1e-3, weight_decay=0.01)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    sd, od = torch.from_numpy(te.seqs).cuda(), torch.from_numpy(te.offsets).cuda()
    rerank.rope_map_rerank(idx, sd, od, rr, k=K, keep=2)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    w_rr, _, _ = rerank.rope_map_rerank(idx, sd, od, rr, k=K, keep=2)
    torch.cuda.synchronize()
    t4 = time.perf_counter()
    w_sc, _, _ = rerank.rope_map_rerank(idx, sd, od, None, k=K, keep=2)
    w8, _ = rm.rope_map(idx, sd, od, k=8, sep=N)
    rm.rope_sync_status()
    hit = lambda w: float((np.abs(w.cpu().numpy() - te.true_pos[:, None]) < N).any(axis=1).mean())
    n_pairs = int(valid.numel())
    rr.free()
    return {"train_pairs": n_pairs, "label_s": t1 - t0, "train_s": t2 - t1, "epochs": 5,
            "train_pairs_per_s": 5 * n_pairs / (t2 - t1), "epoch_loss": [round(x, 6) for x in losses],
            "eval_reads": te.n, "map_rerank_reads_per_s": te.n / (t4 - t3),
            "recall_top2_reranked": hit(w_rr), "recall_top2_score": hit(w_sc), "recall_top8_score": hit(w8),
            "errors": "0-15% per read (2:1 substitutions : indel events)"}


def encode_roofline(rm, p, dref, ref, rd, n_reads):
    """HBM roofline of the encode pass: the reference's 2-bit packing (1 B in +
    0.25 B out per letter) and the read encoding (N letters in, FP32 + BF16
    encodings and 1+m norms out per read), CUDA events around 10 launches.
    The packing is timed on the reference repeated to >= 10^9 letters and the
    encoding on every read of the workload, so that each launch moves enough
    bytes for its time not to be the host's call overhead."""
    import torch

    peaks, src = measured_peaks()
    peak = peaks["hbm_gbs"]

    def timed(fn, reps=10):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps / 1000.0

    big = dref.repeat(max(1, -(-1_000_000_000 // dref.numel())))
    L = big.numel()
    t_pack = timed(lambda: rm.rope_pack_2bit(big))
    b_pack = L * 1.25
    seqs = torch.from_numpy(rd.seqs).cuda()
    n_reads = rd.n
    offs = torch.from_numpy(rd.offsets).cuda()
    t_enc = timed(lambda: rm.rope_encode_reads(p, seqs, offs))
    D = p.dim
    b_enc = n_reads * (p.window_len + 2 * D * 4 + 2 * D * 2 + (1 + p.m) * 4) + (n_reads + 1) * 8
    rm.rope_sync_status()
    del big
    return {"bound": "hbm", "peak": peak, "unit": "GB/s", "peak_source": f"{src} hbm_gbs",
            "pack": {"bytes": b_pack, "ms": t_pack * 1e3, "achieved": b_pack / t_pack / 1e9,
                     "frac": b_pack / t_pack / 1e9 / peak, "letters": L},
            "encode_reads": {"bytes": b_enc, "ms": t_enc * 1e3, "achieved": b_enc / t_enc / 1e9,
                             "frac": b_enc / t_enc / 1e9 / peak, "reads": n_reads,
                             "reads_timed": 10 * n_reads, "s_per_million_reads": t_enc / n_reads * 1e6}}


def run_reference(args, wl):
    """--impl reference: the FP64 oracle on this host's cores, K steps of a bounded sample."""
    ws, rank, _ = dist_setup(args)
    if rank != 0:
        return
    import oracle

    ref, rd = make_inputs(dict(wl, n_reads=min(wl["n_reads"], 4096)), 0)
    op = oracle.Params(s=wl["s"], m=wl["m"], t=wl["t"], variant=wl["variant"], N=wl["N"], stride=wl["stride"])
    W = oracle.n_windows(len(ref), wl["N"], wl["stride"])
    nw = min(W, 200_000)
    # the oracle's OpenMP loop runs over reads: one read per host core per step
    per_step = max(8, oracle.max_threads())
    times = []
    for i in range(args.warmup + args.steps):
        sub = rd.subset(np.arange(i * per_step, (i + 1) * per_step) % rd.n)
        t0 = time.perf_counter()
        oracle.score_topk(ref, sub.seqs, sub.offsets, op, k=wl["k"], j_begin=0, j_end=nw)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    total = sum(times)
    value = args.steps * per_step * nw / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload + ": " + wl["desc"],
                       "sample_per_step": f"{per_step} reads x the first {nw} windows"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": f"{per_step} reads x {nw} windows per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ladder(args, wl):
    """Reads of many lengths through the length ladder: a step maps the whole
    read set (every read against every window of its bucket's index)."""
    import torch

    ws, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_2603_22245_gb300 import rotormap as rm

    rm.load()
    ref, rd = make_inputs(wl, rank)
    p = rm.Params(s=wl["s"], m=wl["m"], t=wl["t"], variant=wl["variant"], window_len=wl["N"], stride=wl["stride"])
    dref = torch.from_numpy(ref).cuda()
    t0 = time.perf_counter()
    lad = rm.rope_ladder_create(p, dref, *wl["ladder"])
    torch.cuda.synchronize()
    index_s = time.perf_counter() - t0
    del dref
    seqs = torch.from_numpy(rd.seqs).cuda()
    offs = torch.from_numpy(rd.offsets).cuda()
    n, k = rd.n, wl["k"]
    outs = [(torch.empty((n, k), dtype=torch.int64, device="cuda"), torch.empty((n, k), dtype=torch.float32,
                                                                              device="cuda"),
             torch.empty((n,), dtype=torch.int32, device="cuda")) for _ in range(2)]
    for i in range(args.warmup):
        rm.rope_ladder_map(lad, seqs, offs, k=k, out=outs[i % 2])
    rm.rope_sync_status()
    used = outs[0][2].cpu().numpy()
    lens = np.array(lad.lengths)
    W_of = {N: (len(ref) - N) // wl["stride"] + 1 for N in lad.lengths}
    scores_step = int(sum(W_of[int(N)] for N in used[used > 0]))
    rm.rope_profile_enable(args.steps)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for i in range(args.steps):
        rm.rope_ladder_map(lad, seqs, offs, k=k, out=outs[i % 2])
    ev1.record()
    torch.cuda.synchronize()
    clocks = clk.stop()
    elapsed = ev0.elapsed_time(ev1) / 1000.0
    if dist:
        t = torch.tensor([elapsed], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())
        dist.barrier()
    rm.rope_sync_status()
    stage_ms = rm.rope_profile_read(args.steps)
    rm.rope_profile_enable(0)
    w = outs[(args.steps - 1) % 2][0][:, 0].cpu().numpy()
    ok = used > 0
    acc = float(np.mean(np.abs(w[ok] - rd.true_pos[ok]) < used[ok]))
    value = ws * args.steps * scores_step / elapsed
    work_ms = float(np.mean(stage_ms[:, 1]))  # encode + scan + merge of every bucket (streams joined)
    flops = scores_step * 8 * p.dim
    peaks, peak_src = measured_peaks()
    peak = peaks["bf16_tflops_sustained"]
    achieved = flops / (work_ms / 1000.0) / 1e12
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "scan_tc_kernel over all buckets (encode and merge included: the "
                "buckets overlap on 4 streams)", "peak_source": f"{peak_src} bf16_tflops_sustained",
                "flops_per_step": flops,
                "stage_ms": {"bucket_sort_and_sync": float(np.mean(stage_ms[:, 0])), "buckets": work_ms,
                             "free": float(np.mean(stage_ms[:, 2]))}}
    hist = {int(N): int(c) for N, c in zip(*np.unique(used[ok], return_counts=True))}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * elapsed / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": args.workload + ": " + wl["desc"], "reads_per_step_per_gpu": n,
                   "scores_per_step_per_gpu": scores_step, "ladder_lengths": len(lens), "reads_per_length": hist,
                   "reads_too_short": int((~ok).sum()), "index_build_s": index_s,
                   "l2": "inputs larger than L2 (54 bucket indexes, 0.5 GB)"},
        "reads_per_s": ws * args.steps * n / elapsed, "top1_acc": acc, "roofline": roofline,
        "gpu_launches": None, "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    lad.free()
    if dist:
        dist.destroy_process_group()


def locus_stats(reads, wins, true_pos, n_reads, stride, N):
    """§3.5 multi-locus output per read: loci = runs of output windows whose
    starts lie within N of the previous one (overlapping windows of one
    locus); unique = exactly one locus; missed = no output window within N of
    the planted start."""
    order = np.lexsort((wins, reads))
    r, w = reads[order], wins[order] * stride
    loci = np.zeros(n_reads, dtype=np.int64)
    hit = np.zeros(n_reads, dtype=bool)
    if len(r):
        new = np.ones(len(r), dtype=bool)
        new[1:] = (r[1:] != r[:-1]) | (w[1:] - w[:-1] > N)
        np.add.at(loci, r[new], 1)
        near = np.abs(w - true_pos[r]) < N
        hit[np.unique(r[near])] = True
    return {"loci_per_read": float(loci.mean()), "unique_fraction": float(np.mean(loci == 1)),
            "missed_fraction": float(np.mean(~hit)), "pairs_per_read": len(reads) / n_reads,
            "reads_without_output": float(np.mean(loci == 0))}


def run_threshold(args, wl):
    """Threshold regime: thresholds for every window, then every pair reaching
    its window's threshold; the paper's §3.5 quantities per read."""
    import torch

    from paper_2603_22245_gb300 import rotormap as rm

    rm.load()
    ref, rd = make_inputs(wl, 0)
    p = rm.Params(s=wl["s"], m=wl["m"], t=wl["t"], variant=wl["variant"], window_len=wl["N"], stride=wl["stride"])
    idx = rm.rope_encode_reference(p, torch.from_numpy(ref).cuda())
    W = idx.n_windows
    th = wl["threshold"]
    _, bf16, _ = rm.rope_encode_reads(p, torch.from_numpy(rd.seqs).cuda(), torch.from_numpy(rd.offsets).cuda(),
                                      want_f32=False)
    cap = 1 << 26
    sweep = []
    ms = None
    for err in th["errs"]:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        thr = rm.rope_fragment_thresholds(idx, err, th["n_samples"], 12345)
        torch.cuda.synchronize()
        t_thr = time.perf_counter() - t0
        rm.rope_score_threshold(idx, bf16, thr, cap=cap)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            r, w, s, total = rm.rope_score_threshold(idx, bf16, thr, cap=cap)
        e1.record()
        torch.cuda.synchronize()
        rm.rope_sync_status()
        ms = e0.elapsed_time(e1) / args.steps if ms is None else ms
        stats = locus_stats(r.cpu().numpy(), w.cpu().numpy(), rd.true_pos, rd.n, wl["stride"], wl["N"])
        thr_h = thr.cpu().numpy()
        sweep.append(dict(stats, err=err, n_samples=th["n_samples"], pairs=int(total),
                          pairs_dropped=int(max(0, total - cap)), threshold_s=t_thr,
                          threshold_windows_per_s=W / t_thr, threshold_mean=float(thr_h.mean()),
                          threshold_p10_p90=[float(np.percentile(thr_h, 10)), float(np.percentile(thr_h, 90))]))
    line = {"metric": METRIC, "value": rd.n * W / (ms / 1000.0), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": 1, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16", "data": "synthetic",
            "config": {"workload": args.workload + ": " + wl["desc"], "reads": rd.n, "n_windows": W},
            "threshold_regime": sweep, "gpu_launches": 2 * args.steps * len(sweep)}
    print(json.dumps(line), flush=True)
    idx.free()


def main():
    args = parse()
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl)
        return
    if "ladder" in wl:
        run_ladder(args, wl)
        return
    if "threshold" in wl:
        run_threshold(args, wl)
        return

    import torch

    ws, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_2603_22245_gb300 import rotormap as rm

    rm.load()
    ref, rd = make_inputs(wl, rank)
    p = rm.Params(s=wl["s"], m=wl["m"], t=wl["t"], variant=wl["variant"], window_len=wl["N"], stride=wl["stride"])
    dref = torch.from_numpy(ref).cuda()
    t0 = time.perf_counter()
    idx = rm.rope_encode_reference(p, dref)
    torch.cuda.synchronize()
    index_s = time.perf_counter() - t0
    encode_pass = encode_roofline(rm, p, dref, ref, rd, min(args.batch, rd.n))
    del dref
    W = idx.n_windows
    seqs = torch.from_numpy(rd.seqs).cuda()
    offs = torch.from_numpy(rd.offsets).cuda()
    B = min(args.batch if args.batch > 0 else wl.get("batch", 131072), rd.n)
    n_batches = max(1, rd.n // B)
    k = wl["k"]
    strands = bool(wl.get("strands"))
    dense_index = p.dim > 128  # materialised index: the BF16 GEMM scan only
    rows = 2 if strands else 1  # query rows per read (both strands)

    def new_out():
        o = (torch.empty((B, k), dtype=torch.int64, device="cuda"), torch.empty((B, k), dtype=torch.float32,
                                                                               device="cuda"))
        return o + (torch.empty((B, k), dtype=torch.int8, device="cuda"),) if strands else o

    # read batches as views: seqs is shared, offsets are absolute into it
    outs = new_out()
    true_pos = rd.true_pos
    true_strand = (np.arange(rd.n) % 2) if strands else np.zeros(rd.n, dtype=np.int64)

    def step(bi, precision="bf16", o=None):
        b = bi % n_batches
        ob = offs[b * B:(b + 1) * B + 1]
        if strands:
            return rm.rope_map_strands(idx, seqs, ob, k=k, precision=precision, out=o or outs)
        return rm.rope_map(idx, seqs, ob, k=k, precision=precision, out=o or outs)

    def hits_of(res, b):
        top = res[0][:, 0].cpu().numpy()
        h = np.abs(top - true_pos[b * B:(b + 1) * B]) < wl["N"]
        if strands:
            h &= res[2][:, 0].cpu().numpy() == true_strand[b * B:(b + 1) * B]
        return h

    if args.scan_variant >= 0 and not dense_index:
        rm.rope_autotune_set(idx, B, args.scan_variant, 16, k=k)
    for i in range(args.warmup):
        step(i)
    rm.rope_sync_status()
    tuned = None if dense_index else rm.rope_autotune_query(idx, B, k=k)  # chosen during the first warm-up step
    rm.rope_profile_enable(args.steps)
    step_outs = [new_out() for _ in range(args.steps)]
    hits = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for i in range(args.steps):
        step(i, o=step_outs[i])
    ev1.record()
    torch.cuda.synchronize()
    clocks = clk.stop()
    elapsed = ev0.elapsed_time(ev1) / 1000.0
    if dist:
        t = torch.tensor([elapsed], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())
        dist.barrier()
    rm.rope_sync_status()
    top2_step0 = step_outs[0][0][:, :2].clone()  # the refinement leg's candidates (batch 0)
    stage_ms = rm.rope_profile_read(args.steps)
    rm.rope_profile_enable(0)
    for i in range(args.steps):
        hits.append(hits_of(step_outs[i], i % n_batches))
    acc_bf16 = float(np.concatenate(hits).mean())
    scores_step = rows * B * W
    value = ws * args.steps * scores_step / elapsed
    reads_s = ws * args.steps * B / elapsed

    # roofline of the scan kernel (CUDA events around its launch, same stream)
    scan_s = float(np.mean(stage_ms[:, 1])) / 1000.0
    flops = scores_step * 8 * p.dim
    peaks, peak_src = measured_peaks()
    peak = peaks["bf16_tflops_sustained"]
    achieved = flops / scan_s / 1e12
    trec = traffic_record(args.workload, B)
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": (trec["dram_bytes_per_launch_scaled"] * 1.0) if trec else None,
                "kernel": "gemm_tc_kernel (BF16 tcgen05 GEMM over the materialised index, A operand build included)"
                if dense_index else "scan_tc_kernel (BF16 tcgen05)", "peak_source": f"{peak_src} bf16_tflops_sustained",
                "flops_per_launch": flops, "ms_per_launch": scan_s * 1000.0,
                "ms_per_launch_median": float(np.median(stage_ms[:, 1])),
                "stage_ms": {"encode": float(np.mean(stage_ms[:, 0])), "scan": float(np.mean(stage_ms[:, 1])),
                             "merge_rescore": float(np.mean(stage_ms[:, 2]))}}

    # FP32 plain path and BF16 on the same read subset (equal-accuracy check)
    fp32 = None
    F = min(wl.get("fp32_reads", args.fp32_reads), B)
    if F > 0:
        osub = offs[:F + 1]

        def map_sub(precision):
            if strands:
                return rm.rope_map_strands(idx, seqs, osub, k=k, precision=precision)
            return rm.rope_map(idx, seqs, osub, k=k, precision=precision)

        def hits_sub(res):
            h = np.abs(res[0][:, 0].cpu().numpy() - true_pos[:F]) < wl["N"]
            return h & (res[2][:, 0].cpu().numpy() == true_strand[:F]) if strands else h

        map_sub("fp32")
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        n32 = 2
        for _ in range(n32):
            fo = map_sub("fp32")
        e1.record()
        torch.cuda.synchronize()
        t32 = e0.elapsed_time(e1) / 1000.0 / n32
        acc32 = float(np.mean(hits_sub(fo)))
        bo = map_sub("bf16")
        acc16_sub = float(np.mean(hits_sub(bo)))
        agree = float(torch.mean((bo[0][:, 0] == fo[0][:, 0]).float()).item())
        rm.rope_sync_status()
        fp32 = {"value": rows * F * W / t32, "unit": UNIT, "reads_per_s": F / t32, "reads": F, "top1_acc": acc32,
                "bf16_top1_acc_same_reads": acc16_sub, "top1_window_agreement": agree,
                "path": "FP32 CUDA-core scan over the stored FP32 rows" if dense_index else
                "FP32 CUDA-core scan with on-chip windows"}

    # E4M3 option: the same steps with the FP8 tensor-core scan (same batches,
    # same rescoring), its top-1 accuracy on the same planted reads
    fp8 = None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.fp8_steps > 0 and not dense_index:
        step(0, precision="fp8")
        rm.rope_sync_status()
        rm.rope_profile_enable(args.fp8_steps)
        e0.record()
        for i in range(args.fp8_steps):
            step(i, precision="fp8", o=step_outs[i])
        e1.record()
        torch.cuda.synchronize()
        t8 = e0.elapsed_time(e1) / 1000.0
        st8 = rm.rope_profile_read(args.fp8_steps)
        rm.rope_profile_enable(0)
        rm.rope_sync_status()
        h8 = [hits_of(step_outs[i], i % n_batches) for i in range(args.fp8_steps)]
        h16 = np.concatenate(hits[:args.fp8_steps])
        scan8 = float(np.mean(st8[:, 1])) / 1000.0
        peak8 = peak * 2.0  # E4M3 dense rate = 2x BF16 (nominal 4.5 vs 2.25 PFLOP/s)
        fp8 = {"value": ws * args.fp8_steps * scores_step / t8, "unit": UNIT, "steps": args.fp8_steps,
               "top1_acc": float(np.concatenate(h8).mean()), "bf16_top1_acc_same_reads": float(h16.mean()),
               "scan_ms": scan8 * 1000.0,
               "roofline": {"bound": "tensor", "achieved": flops / scan8 / 1e12, "peak": peak8, "unit": "TFLOP/s",
                            "frac": flops / scan8 / 1e12 / peak8,
                            "peak_source": f"{peak_src} bf16_tflops_sustained x 2 (nominal E4M3/BF16 ratio)"}}

    # refinement (§3.4): the first step's top-2 candidates of each read slid
    # +-radius letters under a 2 x 4^8-bin encoding (s = t = 8, m = 2
    # fine-tuned: two bands of different frequency, so that a shifted window
    # changes the bands' relative phase)
    refine = None
    if args.refine_radius > 0 and not dense_index:
        try:
            fine = rm.Params(s=8, m=2, t=8, variant=1, window_len=wl["N"])
            cand = top2_step0
            ob = offs[:B + 1]
            rm.rope_refine(idx, fine, seqs, ob, cand, args.refine_radius)
            torch.cuda.synchronize()
            e0.record()
            n_rf = 3
            for _ in range(n_rf):
                rp, rf = rm.rope_refine(idx, fine, seqs, ob, cand, args.refine_radius)
            e1.record()
            torch.cuda.synchronize()
            rm.rope_sync_status()
            t_rf = e0.elapsed_time(e1) / 1000.0 / n_rf
            tp0 = true_pos[:B]
            best = rp.gather(1, rf.argmax(dim=1, keepdim=True))[:, 0].cpu().numpy()
            refine = {"candidates_per_s": 2 * B / t_rf, "positions_per_s": 2 * B * (2 * args.refine_radius + 1) / t_rf,
                      "ms": t_rf * 1e3, "reads": B, "radius": args.refine_radius, "encoding": "s=8 m=2 t=8 fine-tuned (2 x 4^8 bins)",
                      "exact_start_before": float(np.mean(top2_step0[:, 0].cpu().numpy() == tp0)),
                      "exact_start_after": float(np.mean(best == tp0))}
        except Exception as exc:  # a failure here must not cost the bench line
            refine = {"error": str(exc)}

    # end to end through host buffers, every step a different batch: H2D of
    # the batch's reads from pinned host memory, rope_map, D2H of the top-k
    e2e = None
    n_e2e = args.e2e_steps if args.e2e_steps >= 0 else args.steps
    if n_e2e > 0:
        lim = rd.offsets[min(n_batches, n_e2e + 1) * B]  # letters of the batches used
        seq_pin = torch.from_numpy(np.ascontiguousarray(rd.seqs[:lim])).pin_memory()
        nb_e2e = min(n_batches, n_e2e + 1)
        # per batch, its offsets relative to its first letter (host side, pinned)
        off_pin = torch.from_numpy(np.stack([rd.offsets[b * B:(b + 1) * B + 1] - rd.offsets[b * B]
                                             for b in range(nb_e2e)])).pin_memory()
        w_pin = torch.empty((B, k), dtype=torch.int64).pin_memory()
        s_pin = torch.empty((B, k), dtype=torch.float32).pin_memory()
        t_pin = torch.empty((B, k), dtype=torch.int8).pin_memory()
        max_letters = int(max(rd.offsets[(b + 1) * B] - rd.offsets[b * B] for b in range(min(n_batches, n_e2e + 1))))
        dseq = torch.empty((max_letters,), dtype=torch.uint8, device="cuda")
        doff = torch.empty((B + 1,), dtype=torch.int64, device="cuda")
        h2d = d2h = 0
        for it in range(1 + n_e2e):
            if it == 1:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                h2d = d2h = 0
            b = it % min(n_batches, n_e2e + 1)
            a0, a1 = int(rd.offsets[b * B]), int(rd.offsets[(b + 1) * B])
            dseq[:a1 - a0].copy_(seq_pin[a0:a1], non_blocking=True)
            doff.copy_(off_pin[b], non_blocking=True)
            if strands:
                w_, s_, t_ = rm.rope_map_strands(idx, dseq, doff, k=k, precision="bf16", out=outs)
                t_pin.copy_(t_, non_blocking=True)
            else:
                w_, s_ = rm.rope_map(idx, dseq, doff, k=k, precision="bf16", out=outs)
            w_pin.copy_(w_, non_blocking=True)
            s_pin.copy_(s_, non_blocking=True)
            torch.cuda.synchronize()
            h2d += (a1 - a0) + (B + 1) * 8
            d2h += w_pin.numel() * 8 + s_pin.numel() * 4 + (t_pin.numel() if strands else 0)
        te = (time.perf_counter() - t0) / n_e2e
        if dist:
            t = torch.tensor([te], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            te = float(t.item())
        e2e = {"value": ws * scores_step / te, "unit": UNIT, "reads_per_s": ws * B / te, "steps": n_e2e,
               "batches": f"{min(n_batches, n_e2e + 1)} distinct batches of {B} reads, one per step",
               "h2d_bytes_per_step": int(h2d // n_e2e), "d2h_bytes_per_step": int(d2h // n_e2e)}

    reranker = None
    if args.rerank_train_reads > 0 and not dense_index:
        reranker = rerank_leg(rm, idx, ref, wl, args)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(ref, rd, wl, wl.get("cpu_reads", args.cpu_reads), wl.get("cpu_windows", args.cpu_windows))

    # bytes one scan pass streams: the packed reference and 8 B of anchors and
    # norms per window, or the materialised index's two BF16 window matrices
    # ([W, 2D] each)
    index_gb = (2 * W * 2 * p.dim * 2 if dense_index else wl['L'] / 4 + 8 * W) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * elapsed / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": args.workload + ": " + wl["desc"], "reads_per_step_per_gpu": B, "n_windows": W,
                   "scores_per_step_per_gpu": scores_step, "l2": f"inputs larger than L2 ({index_gb:.1f} GB index "
                   f"streamed per scan pass; reads {B * wl['read_len'] / 1e6:.0f} MB/step)", "index_build_s": index_s, "parallelism": f"replicated index, "
                   f"reads sharded over {ws} GPU(s)",
                   "scan_tiles": None if tuned is None else {"variant": tuned[0], "items_per_sm": tuned[1],
                                                              "tuned_scan_ms": tuned[2]}},
        "reads_per_s": reads_s, "top1_acc": acc_bf16, "fp32_plain": fp32, "fp8_option": fp8, "refine": refine,
        "encode_pass": encode_pass,
        "speedup_vs_fp32_plain": value / ws / fp32["value"] if fp32 else None,
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "reranker": reranker,
        # per step: encode, scan, merge; with both strands two encodes and the
        # strand merge; on a materialised index also the A-operand build
        "gpu_launches": (3 + (2 if strands else 0) + (1 if dense_index else 0)) * args.steps, "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    idx.free()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
