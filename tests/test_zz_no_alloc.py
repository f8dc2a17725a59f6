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
contents), in both precisions; and a request larger than the array is refused
with a clear error. This file is collected last so that a failure here leaves
every other test already run.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _inputs(lib, n_reads):
    ref = synth.uniform_ref(100_000, 1)
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
