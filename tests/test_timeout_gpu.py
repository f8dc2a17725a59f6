"""Failure detection on the GPU without a fault: every wait inside the
tensor-core scan is bounded, and a wait that runs out sets the timeout bit,
after which the kernel waits for its own copies and tensor-core operations in
flight, frees its tensor memory and returns. A wait limit of nanoseconds
(rope_set_wait_limit) makes the scan's first unsatisfied wait run out, so
this path runs on an ordinary small scan: rope_sync_status reports
ROPE_ERR_TIMEOUT, and the next call at the ordinary limit is exact again (the
context stays usable)."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small(lib):
    ref = synth.uniform_ref(100_000, 1)
    rd = synth.reads(ref, 256, seed=2)
    p = lib.Params(s=4, m=2, t=2, variant=1, window_len=150)
    idx = lib.rope_encode_reference(p, torch.from_numpy(ref).cuda())
    enc = lib.rope_encode_reads(p, torch.from_numpy(rd.seqs).cuda(), torch.from_numpy(rd.offsets).cuda())
    lib.rope_sync_status()
    yield idx, enc
    idx.free()


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_scan_timeout_reported_and_recovered(lib, small, precision):
    idx, (f32, bf16, norms) = small
    want = lib.rope_score_topk(idx, f32, bf16, norms, k=8, precision=precision, n_ranges=4)
    lib.rope_sync_status()
    lib.rope_set_wait_limit(1e-9)
    try:
        lib.rope_score_topk(idx, f32, bf16, norms, k=8, precision=precision, n_ranges=4)
        with pytest.raises(lib.RopeError) as e:
            lib.rope_sync_status()
        assert e.value.status == 5
        # the dense mode of the same kernel takes the same path
        lib.rope_score_dense(idx, f32, bf16, norms, 0, 5000, precision=precision)
        with pytest.raises(lib.RopeError) as e:
            lib.rope_sync_status()
        assert e.value.status == 5
    finally:
        lib.rope_set_wait_limit(0)
    got = lib.rope_score_topk(idx, f32, bf16, norms, k=8, precision=precision, n_ranges=4)
    lib.rope_sync_status()
    assert torch.equal(got[0], want[0]) and torch.equal(got[1], want[1])


def test_wait_limit_bounds(lib):
    with pytest.raises(lib.RopeError):
        lib.rope_set_wait_limit(-1.0)
    with pytest.raises(lib.RopeError):
        lib.rope_set_wait_limit(1e3)
    lib.rope_set_wait_limit(0.5)
    lib.rope_set_wait_limit(0)
