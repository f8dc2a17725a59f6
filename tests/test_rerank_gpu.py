"""Learned reranker: exact Levenshtein labels, forward/backward/AdamW parity
with the FP64 oracle network, checkpointing, and what the trained network
gains over the plain score ranking."""
import os
import tempfile

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rr_mod(lib):
    from paper_2603_22245_gb300 import rerank

    return rerank


def bf16_round(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy()


# ---------------------------------------------------------------- Levenshtein labels

@pytest.mark.parametrize("N", [40, 64, 65, 150, 200, 256])
def test_levenshtein_bit_exact(lib, rr_mod, N):
    ref = synth.markov_ref(50_000, 0.41, 3, 0.05, 0.05)
    rd = synth.reads(ref, 300, seed=4, length=N, sub_rate=0.05, indel_rate=0.05)
    p = lib.Params(s=4, m=2, t=2, variant=1, window_len=N)
    idx = lib.rope_encode_reference(p, torch.from_numpy(ref).cuda())
    rng = np.random.default_rng(N)
    ri = np.concatenate([np.arange(rd.n), rng.integers(0, rd.n, 500)])
    ws = np.concatenate([rd.true_pos, rng.integers(0, len(ref) - N, 500)])
    ld, frac = rr_mod.rope_levenshtein(idx, torch.from_numpy(rd.seqs).cuda(), torch.from_numpy(rd.offsets).cuda(),
                                       torch.from_numpy(ri).cuda(), torch.from_numpy(ws).cuda())
    lib.rope_sync_status()
    want = oracle.levenshtein_pairs(ref, rd.seqs, rd.offsets, ri, ws, N)
    assert np.array_equal(ld.cpu().numpy(), want)
    assert np.allclose(frac.cpu().numpy(), want / N, rtol=0, atol=1e-7)
    idx.free()


# ---------------------------------------------------------------- feature rows

@pytest.mark.parametrize("m", [2, 4])
def test_features_match_oracle(lib, rr_mod, m):
    """Feature rows against the FP64 oracle on seeded candidates (planted
    loci, loci a few letters off, random loci, reference ends, missing)."""
    ref = synth.markov_ref(60_000, 0.41, 7, 0.05, 0.05)
    rd = synth.reads(ref, 40, seed=8, sub_rate=0.03, indel_rate=0.02)
    p = lib.Params(s=4, m=m, t=2, variant=1, window_len=150)
    op = oracle.Params(s=4, m=m, t=2, variant=1, N=150)
    idx = lib.rope_encode_reference(p, torch.from_numpy(ref).cuda())
    rng = np.random.default_rng(9)
    K = 6
    W = len(ref) - 150 + 1
    cw = np.stack([rd.true_pos, rd.true_pos + rng.integers(-3, 4, rd.n), rng.integers(0, W, rd.n),
                   np.zeros(rd.n, np.int64), np.full(rd.n, W - 1), np.full(rd.n, -1)], axis=1)
    cw[:, 1] = np.clip(cw[:, 1], 0, W - 1)
    cs = np.sort(rng.uniform(0, 1, (rd.n, K)), axis=1)[:, ::-1].copy()
    cs[:, -1] = -np.inf
    sd, od = torch.from_numpy(rd.seqs).cuda(), torch.from_numpy(rd.offsets).cuda()
    f32, _, norms = lib.rope_encode_reads(p, sd, od, want_bf16=False)
    X = rr_mod.rope_rerank_features(idx, sd, od, f32, norms, torch.from_numpy(cw).cuda(),
                                    torch.from_numpy(cs.astype(np.float32)).cuda())
    lib.rope_sync_status()
    got = X.cpu().numpy().astype(np.float64)
    want = oracle.rerank_features(ref, rd.seqs, rd.offsets, cw, cs.astype(np.float32), op)
    assert got.shape == want.shape == (rd.n * K, K + 6 + m)
    bands = slice(K + 1, K + 1 + m)
    assert np.allclose(got[:, bands], want[:, bands], rtol=1e-5, atol=1e-6)
    rest = np.ones(got.shape[1], bool)
    rest[bands] = False
    assert np.allclose(got[:, rest], want[:, rest], rtol=0, atol=1e-6)
    idx.free()


# ---------------------------------------------------------------- network parity

def _random_net(rr_mod, F=20, H=128, seed=0):
    rr = rr_mod.Reranker(F, H, seed=seed)
    rng = np.random.default_rng(seed)
    W1 = rng.normal(size=(H, F)) * 0.3
    b1 = rng.normal(size=H) * 0.1
    w2 = rng.normal(size=H) * 0.2
    b2 = 0.05
    rr.set_params(np.concatenate([W1.ravel(), b1, w2, [b2]]).astype(np.float32))
    # the device holds W1 and w2 in BF16: the FP64 reference uses the same values
    net = oracle.MLP(bf16_round(W1), np.float32(b1), bf16_round(w2), np.float32(b2))
    return rr, net


def test_forward_and_gradient_match_fp64_oracle(rr_mod):
    F, H, B = 20, 128, 3000
    rr, net = _random_net(rr_mod, F, H)
    rng = np.random.default_rng(5)
    X = rng.normal(size=(B + 17, F)).astype(np.float32)
    t = rng.uniform(0, 0.3, size=B + 17).astype(np.float32)
    sel = rng.permutation(B + 17)[:B].astype(np.int64)
    Xd, td, sd = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda(), torch.from_numpy(sel).cuda()
    y = rr.predict(Xd).cpu().numpy().astype(np.float64)
    assert np.allclose(y, net.forward(X.astype(np.float64)), rtol=1e-5, atol=1e-5)
    g, loss = rr.grad(Xd, td, sd)
    g = g.cpu().numpy().astype(np.float64)
    l64, gW1, gb1, gw2, gb2 = net.grad(X[sel].astype(np.float64), t[sel].astype(np.float64))
    want = np.concatenate([gW1.ravel(), gb1, gw2, [gb2]])
    assert float(loss.item()) == pytest.approx(l64, rel=1e-4)
    scale = np.abs(want).max()
    assert np.abs(g - want).max() <= 1e-4 * scale, np.abs(g - want).max() / scale
    rr.free()


def test_adamw_step_matches_fp64_oracle(rr_mod):
    F, H, B = 20, 128, 2048
    rr, net = _random_net(rr_mod, F, H, seed=2)
    rng = np.random.default_rng(6)
    X = rng.normal(size=(B, F)).astype(np.float32)
    t = rng.uniform(0, 0.3, size=B).astype(np.float32)
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    p0, step0 = rr.params()
    g, _ = rr.grad(Xd, td)
    rr.train_step(Xd, td, None, lr=1e-3, weight_decay=0.01)
    p1, step1 = rr.params()
    assert step1 == step0 + 1
    p = p0.astype(np.float64).copy()
    m, v = np.zeros_like(p), np.zeros_like(p)
    oracle.adamw(p, g.cpu().numpy().astype(np.float64), m, v, 1, lr=1e-3, wd=0.01)
    assert np.allclose(p1, p, rtol=0, atol=2e-6)
    rr.free()


def test_checkpoint_round_trip(rr_mod):
    rr, _ = _random_net(rr_mod, 20, 128, seed=3)
    X = torch.randn(64, 20, device="cuda")
    t = torch.rand(64, device="cuda")
    for _ in range(3):
        rr.train_step(X, t, None)
    y0 = rr.predict(X)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "rr.bin")
        rr.save(path)
        rr2 = rr_mod.Reranker(20, 128, seed=99)
        rr2.load(path)
        assert torch.equal(rr2.predict(X), y0)
        assert rr2.params()[1] == rr.params()[1]
        assert np.array_equal(rr2.params()[0], rr.params()[0])
        # training resumes identically from the checkpoint
        rr.train_step(X, t, None)
        rr2.train_step(X, t, None)
        assert torch.equal(rr2.predict(X), rr.predict(X))
        rr2.free()
    rr.free()


# ---------------------------------------------------------------- gain over the score ranking

def _reads_mixed_error(ref, n, seed, max_rate=0.15):
    rd = synth.reads_mixed_error(ref, n, seed, max_rate)
    return rd.seqs, rd.offsets, rd.true_pos


def test_reranker_trains_and_prunes(lib, rr_mod):
    ref = synth.markov_ref(3_000_000, 0.41, 31, 0.025, 0.025, 0.0)
    p = lib.Params(s=4, m=2, t=2, variant=1, window_len=150)
    idx = lib.rope_encode_reference(p, torch.from_numpy(ref).cuda())
    K = 16
    s_tr, o_tr, _ = _reads_mixed_error(ref, 6000, 100)
    X, t, valid, _ = rr_mod.training_set(idx, torch.from_numpy(s_tr).cuda(), torch.from_numpy(o_tr).cuda(), k=K)
    rr = rr_mod.Reranker(rr_mod.n_features(K, p.m), 128, seed=7)
    losses = rr_mod.train(rr, X, t, valid, epochs=5, batch=4096, lr=1e-3)
    assert losses[-1] < losses[0]
    # held-out reads: keep 2 of 16 by predicted distance vs by score
    s_te, o_te, tp = _reads_mixed_error(ref, 4000, 500)
    sd, od = torch.from_numpy(s_te).cuda(), torch.from_numpy(o_te).cuda()
    w_rr, _, pred = rr_mod.rope_map_rerank(idx, sd, od, rr, k=K, keep=2)
    w_sc, _, _ = rr_mod.rope_map_rerank(idx, sd, od, None, k=K, keep=2)
    w8 = lib.rope_map(idx, sd, od, k=8, sep=150)[0]
    lib.rope_sync_status()
    hit = lambda w: (np.abs(w.cpu().numpy() - tp[:, None]) < 150).any(axis=1).mean()
    r_rr, r_sc, r8 = hit(w_rr), hit(w_sc), hit(w8)
    print(f"true-locus recall: reranked top-2 {r_rr:.4f}, score top-2 {r_sc:.4f}, score top-8 {r8:.4f}")
    # the network, given the Hamming fingerprint fidelities next to the RoPE
    # fidelities, keeps the true locus more often than the score ranking
    assert r_rr > r_sc + 0.005
    assert r8 >= r_sc
    rr.free()
    idx.free()
