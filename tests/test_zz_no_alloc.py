"""The allocation-free scan entry point against the ordinary one.

Some callers cannot let a library allocate device memory in the middle of a
call: a process that hands nearly all device memory to its own arena at
start-up (an allocation later can fail or fragment that arena), or a
latency-critical loop that cannot take the device-wide synchronisation
cudaMalloc/cudaFree imply. rope_score_topk_noalloc serves them by running the
same scan, merge and re-scoring kernels as rope_score_topk on a fixed 16 MiB
scratch array inside the library, with the caller passing inputs and outputs.

Checked here, through the C ABI: its output equals rope_score_topk's on the
same inputs (windows exactly, fidelities within the FP32 tolerance the other
tests use), on two calls in a row (the array keeps the previous call's
contents), in both precisions, also when the second call is smaller than the
first and when the entry point picks its own split of the windows; a request
larger than the array is refused with a clear error; a warm call changes the
device's free memory by nothing (checked in a fresh process, where the
library's memory pool has never served a call); and a bounded wait that runs
out (a wait limit of nanoseconds) gives (-1, -inf) for every read, not the
previous call's candidates, with the timeout reported by
rope_noalloc_sync_status. This file is collected last so that a failure here
leaves every other test already run.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
import torch

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def _inputs(lib, n_reads, ref_len=100_000):
    ref = synth.uniform_ref(ref_len, 1)
    rd = synth.reads(ref, n_reads, seed=2)
    p = lib.Params(s=4, m=2, t=2, variant=1, window_len=150)
    idx = lib.rope_encode_reference(p, torch.from_numpy(ref).cuda())
    f32, bf16, norms = lib.rope_encode_reads(p, torch.from_numpy(rd.seqs).cuda(), torch.from_numpy(rd.offsets).cuda())
    lib.rope_sync_status()
    return idx, f32, bf16, norms


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_noalloc_matches_score_topk_twice(lib, precision):
    n, k = 300, 8
    idx, f32, bf16, norms = _inputs(lib, n)
    want_w, want_s = lib.rope_score_topk(idx, f32, bf16, norms, k=k, precision=precision, n_ranges=6)
    lib.rope_sync_status()
    want_w, want_s = want_w.cpu().numpy(), want_s.cpu().numpy().astype(np.float64)
    for _ in range(2):
        out = (torch.full((n, k), -7, dtype=torch.int64, device="cuda"),
               torch.full((n, k), float("nan"), dtype=torch.float32, device="cuda"))
        lib.rope_score_topk_noalloc(idx, f32, bf16, norms, out, k=k, precision=precision, n_ranges=6)
        lib.rope_sync_status()
        got_w, got_s = out[0].cpu().numpy(), out[1].cpu().numpy().astype(np.float64)
        assert np.array_equal(got_w, want_w)
        assert np.all(np.abs(got_s - want_s) <= 1e-5 * np.abs(want_s) + 1e-7)
    idx.free()


def test_noalloc_automatic_split_and_oversize(lib):
    n, k = 300, 8
    idx, f32, bf16, norms = _inputs(lib, n)
    # FP32 without re-scoring is exact whatever the window split, so the
    # automatic split the entry point picks must give the ordinary result
    want = lib.rope_score_topk(idx, f32, None, norms, k=k, precision="fp32")
    out = (torch.empty((n, k), dtype=torch.int64, device="cuda"), torch.empty((n, k), dtype=torch.float32,
                                                                              device="cuda"))
    lib.rope_score_topk_noalloc(idx, f32, None, norms, out, k=k, precision="fp32")
    lib.rope_sync_status()
    assert torch.equal(out[0], want[0])
    # more candidates than the 16 MiB array holds: refused before any launch
    big = 131_073
    f = torch.empty((big, 64), dtype=torch.float32, device="cuda")
    nm = torch.ones((big, 3), dtype=torch.float32, device="cuda")
    o = (torch.empty((big, k), dtype=torch.int64, device="cuda"), torch.empty((big, k), dtype=torch.float32,
                                                                              device="cuda"))
    with pytest.raises(lib.RopeError) as e:
        lib.rope_score_topk_noalloc(idx, f, None, nm, o, k=k, precision="fp32", cand_depth=16)
    assert e.value.status == 1 and "allocation-free scratch" in str(e.value)
    idx.free()


def _out(n, k):
    return (torch.full((n, k), -7, dtype=torch.int64, device="cuda"),
            torch.full((n, k), float("nan"), dtype=torch.float32, device="cuda"))


def test_noalloc_smaller_second_call(lib):
    """A call that needs less of the array than the one before it (fewer reads,
    a shorter reference) must not see that call's leftover candidates."""
    k = 8
    big = _inputs(lib, 300)
    lib.rope_score_topk_noalloc(*big, _out(300, k), k=k, precision="bf16", n_ranges=6)
    small = _inputs(lib, 50, ref_len=20_000)
    for precision in ("bf16", "fp32"):
        want = lib.rope_score_topk(*small, k=k, precision=precision, n_ranges=2)
        got = _out(50, k)
        lib.rope_score_topk_noalloc(*small, got, k=k, precision=precision, n_ranges=2)
        lib.rope_sync_status()
        lib.rope_noalloc_sync_status()
        assert torch.equal(got[0], want[0])
        assert torch.all((got[1] - want[1]).abs() <= 1e-5 * want[1].abs() + 1e-7)
    big[0].free()
    small[0].free()


def test_noalloc_bf16_automatic_split(lib):
    """4096 reads over a 1 Mbp reference: the default split does not fit the
    array, so the entry point re-plans with fewer window ranges; with BF16
    scores and FP32 re-scoring the result is still rope_score_topk's."""
    n, k = 4096, 8
    idx, f32, bf16, norms = _inputs(lib, n, ref_len=1_000_000)
    want = lib.rope_score_topk(idx, f32, bf16, norms, k=k, precision="bf16", rescore=1, cand_depth=16)
    got = _out(n, k)
    lib.rope_score_topk_noalloc(idx, f32, bf16, norms, got, k=k, precision="bf16", rescore=1, cand_depth=16)
    lib.rope_sync_status()
    lib.rope_noalloc_sync_status()
    assert torch.equal(got[0], want[0])
    assert torch.equal(got[1], want[1])
    idx.free()


def test_noalloc_timeout_gives_empty_rows(lib):
    """A wait limit of nanoseconds makes the scan's first unsatisfied wait run
    out: the call then reports (-1, -inf) for every read even though the
    previous call left full candidate lists in the array, and the status
    query says ROPE_ERR_TIMEOUT; at the ordinary limit the next call is exact."""
    n, k = 300, 8
    idx, f32, bf16, norms = _inputs(lib, n)
    want = _out(n, k)
    lib.rope_score_topk_noalloc(idx, f32, bf16, norms, want, k=k, precision="bf16", n_ranges=6)
    lib.rope_noalloc_sync_status()
    assert torch.all(want[0] >= 0)
    got = _out(n, k)
    lib.rope_set_wait_limit(1e-9)
    try:
        lib.rope_score_topk_noalloc(idx, f32, bf16, norms, got, k=k, precision="bf16", n_ranges=6)
        with pytest.raises(lib.RopeError) as e:
            lib.rope_noalloc_sync_status()
        assert e.value.status == 5
    finally:
        lib.rope_set_wait_limit(0)
    assert torch.all(got[0] == -1) and torch.all(torch.isneginf(got[1]))
    lib.rope_noalloc_sync_status()  # read and cleared
    again = _out(n, k)
    lib.rope_score_topk_noalloc(idx, f32, bf16, norms, again, k=k, precision="bf16", n_ranges=6)
    lib.rope_noalloc_sync_status()
    assert torch.equal(again[0], want[0]) and torch.equal(again[1], want[1])
    idx.free()


_FRESH = textwrap.dedent("""
    import sys, torch
    sys.path.insert(0, {root!r})
    import synth
    from paper_2603_22245_gb300 import rotormap as lib
    ref = synth.uniform_ref(100_000, 1)
    p = lib.Params(s=4, m=2, t=2, variant=1, window_len=150)
    idx = lib.rope_encode_reference(p, torch.from_numpy(ref).cuda())
    outs = []
    for n in (300, 120):
        rd = synth.reads(ref, n, seed=2)
        enc = lib.rope_encode_reads(p, torch.from_numpy(rd.seqs).cuda(), torch.from_numpy(rd.offsets).cuda())
        outs.append((enc, (torch.empty((n, 8), dtype=torch.int64, device="cuda"),
                           torch.empty((n, 8), dtype=torch.float32, device="cuda"))))
    lib.rope_sync_status()
    def calls():
        for (enc, out) in outs:
            for precision in ("bf16", "fp32"):
                lib.rope_score_topk_noalloc(idx, *enc, out, k=8, precision=precision, n_ranges=6)
        lib.rope_noalloc_sync_status()
        torch.cuda.synchronize()
    calls()  # warm: the first call's set-up, and every kernel's first (lazy) load
    before = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    calls()
    calls()
    after = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    print("FREE", before[0], after[0], before[1], after[1])
    assert before == after, (before, after)
""")


def test_noalloc_allocates_nothing():
    """In a fresh process (the library's pool has never served a call there,
    so an allocation from it would have to take new device memory) warm calls
    of several sizes and both precisions leave the device's free memory and
    torch's allocated memory unchanged."""
    r = subprocess.run([sys.executable, "-c", _FRESH.format(root=ROOT)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
