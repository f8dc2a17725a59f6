"""Helpers shared by the GPU parity tests: tolerances and the top-k check
against the FP64 oracle."""
import numpy as np
import torch

import oracle

F32_REL, F32_ABS = 1e-5, 1e-7


def bf16_tol(f):
    f = np.asarray(f, dtype=np.float64)
    return np.maximum(2e-2 * f, 8e-3 * np.sqrt(np.maximum(f, 0)) + 2e-5)


# E4M3 scan: per operand entry the relative rounding error is at most 2^-4
# (3 mantissa bits, round to nearest), after the BF16 rounding (2^-8) of the
# read's encoding; the window's FP32 entries carry ~1e-5. So every product
# x_i c_i is off by at most (2^-4 + 2^-8 + 2^-12) + 2^-4 + (their product)
# < 0.134 of |x_i c_i|, and Re/Im of the inner product of two unit vectors by
# eps <= 0.134 * sum|x_i c_i| + (subnormal floor) <= 0.136. The fidelity
# Re^2 + Im^2 then moves by at most 2 eps (|Re| + |Im|) + 2 eps^2
# <= 2 eps sqrt(2 f) + 2 eps^2.
FP8_EPS = 0.136


def fp8_tol(f):
    f = np.maximum(np.asarray(f, dtype=np.float64), 0)
    return 2 * FP8_EPS * np.sqrt(2 * f) + 2 * FP8_EPS ** 2


def f32_tol(f):
    return F32_REL * np.abs(np.asarray(f, dtype=np.float64)) + F32_ABS


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.cuda() if dtype is None else t.to(dtype).cuda()


def check_topk(ref, rd, op, gw, gs, ow, os_, k, tol_fn, score_tol_fn=None, sep=0):
    """gw/gs: GPU top-k; ow/os_: oracle top-(k+1).

    Every reported score must equal the oracle's fidelity of the reported
    window; every oracle top-k entry that beats the oracle's (k+1)-th score by
    more than the tolerance must be reported. With sep > 0 the unique object is
    the bucket floor(start/sep): the GPU must report that bucket, with a window
    whose oracle score is within the tolerance of the bucket's best.
    """
    n = gw.shape[0]
    score_tol_fn = score_tol_fn or tol_fn
    valid = gw >= 0
    ri = np.repeat(np.arange(n), k).reshape(n, k)[valid]
    ws = gw[valid]
    assert np.all(ws % op.stride == 0)
    truth = np.full(gw.shape, -np.inf)
    truth[valid] = oracle.score_pairs(ref, rd.seqs, rd.offsets, ri, ws, op)
    assert np.all(np.abs(gs[valid] - truth[valid]) <= score_tol_fn(truth[valid])), \
        np.abs(gs[valid] - truth[valid]).max()
    assert np.all(np.diff(gs, axis=1) <= 0)
    missing = 0
    for i in range(n):
        kth1 = os_[i, k]
        for j in range(k):
            if not os_[i, j] - kth1 > tol_fn(os_[i, j]):
                continue
            if sep == 0:
                missing += ow[i, j] not in set(gw[i].tolist())
            else:
                hit = [c for c in range(k) if gw[i, c] >= 0 and gw[i, c] // sep == ow[i, j] // sep]
                missing += not hit or truth[i, hit[0]] < os_[i, j] - tol_fn(os_[i, j])
    assert missing == 0, f"{missing} oracle top-k windows missing"
