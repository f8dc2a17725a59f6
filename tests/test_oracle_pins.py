"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it checks. These run on CPU only.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")
LETTERS = b"ACGT"


def rand_seq(n, seed):
    return synth.uniform_ref(n, seed)


def de_bruijn(k, n):
    """de Bruijn sequence B(k, n) (every length-n word over k letters exactly
    once, cyclically), by the Lyndon-word construction; linearised by
    appending its first n-1 letters."""
    a = [0] * k * n
    seq = []

    def db(t, p):
        if t > n:
            if n % p == 0:
                seq.extend(a[1:p + 1])
        else:
            a[t] = a[t - p]
            db(t + 1, p)
            for j in range(a[t - p] + 1, k):
                a[t] = j
                db(t + 1, t)

    db(1, 1)
    seq = seq + seq[: n - 1]
    return bytes(LETTERS[i] for i in seq)


PARAMS = [
    dict(s=4, m=2, t=2, variant=1),   # d=64 reading
    dict(s=4, m=4, t=2, variant=1),   # d=128 reading
    dict(s=2, m=2, t=2, variant=0),   # paper-pure default, no compaction
    dict(s=3, m=1, t=3, variant=0),
    dict(s=5, m=3, t=3, variant=1),
]


# ------------------------------------------------------------------ §1

def test_hamming_fingerprint_golden():
    facts = json.load(open(GOLDEN))["hamming_fingerprint"]
    for f in facts:
        assert oracle.hamming_fingerprint_fidelity(f["S"], f["T"]) == pytest.approx(f["fidelity"], abs=1e-15)


def test_hamming_fingerprint_formula_random():
    rng = np.random.default_rng(0)
    for n in (1, 7, 64, 300):
        S = rand_seq(n, 11 + n)
        for d in sorted(set([0, 1, n // 3, n])):
            T = S.copy()
            for i in rng.choice(n, size=d, replace=False):
                T[i] = LETTERS[(LETTERS.index(S[i]) + 1 + rng.integers(3)) % 4]
            assert oracle.hamming_fingerprint_fidelity(S, T) == pytest.approx(((n - d) / n) ** 2, abs=1e-14)


# ------------------------------------------------------------------ §2.1–2.3, §3.3 golden dimensions

def test_dimensions_golden():
    facts = json.load(open(GOLDEN))
    for f in facts["dimensions"]:
        p = oracle.Params(s=f["s"], m=f["m"], t=f["t"], variant=0, N=4 ** f["s"] + 8)
        assert p.dim == f["complex_dim"]
        assert 2 * f["t"] + int(math.log2(f["m"])) == f["qubits"]
        if f["complex_dim"] <= 1024:
            x = oracle.embed(rand_seq(p.N, 5), p)
            assert x.shape == (f["complex_dim"],)
    fr = facts["fine_tuned_factor_range"]
    fs = [a / q for a, q in (oracle.factor(fr["m"], 1, k) for k in range(1, fr["m"] + 1))]
    assert min(fs) == fr["min"] and max(fs) == fr["max"]
    assert all(b > a for a, b in zip(fs, fs[1:]))
    assert [a / q for a, q in (oracle.factor(4, 0, k) for k in range(1, 5))] == [1, 2, 3, 4]
    assert oracle.factor(1, 1, 1) == (1, 1)
    wc = facts["window_count"]
    assert oracle.n_windows(wc["L"], wc["N"], wc["step"]) == pytest.approx(wc["approx_windows"], rel=wc["rel_tol"])
    so = facts["scan_ops"]
    assert 4 * so["windows"] * so["complex_dim"] == pytest.approx(so["approx_ops_per_read"], rel=so["rel_tol"])


# ------------------------------------------------------------------ §2.1 letters, packing, s-mers

def test_pack_bit_layout():
    seq = rand_seq(1000, 3)
    packed = oracle.pack_2bit(seq)
    assert packed.shape == ((1000 + 15) // 16,)
    for i in range(1000):
        assert (int(packed[i // 16]) >> (2 * (i % 16))) & 3 == LETTERS.index(seq[i])
    assert int(packed[-1]) >> (2 * (1000 % 16)) == 0
    assert np.array_equal(oracle.pack_2bit(bytes(seq).lower()), packed)
    with pytest.raises(ValueError):
        oracle.pack_2bit(b"ACGTN")


def test_mer_bins_brute_force():
    seq = rand_seq(200, 4)
    for s, t in ((1, 1), (3, 3), (4, 2), (6, 3)):
        bm = oracle.default_bin_map(s, t)
        bins = oracle.mer_bins(seq, s, bm)
        for p in range(len(seq) - s + 1):
            code = 0
            for i in range(s):
                code = code * 4 + LETTERS.index(seq[p + i])
            assert bins[p] == bm[code]


def test_default_bin_map_properties():
    for s in range(1, 8):
        assert np.array_equal(oracle.default_bin_map(s, s), np.arange(4 ** s))
    for s, t in ((4, 2), (6, 3), (8, 4)):
        bm = oracle.default_bin_map(s, t)
        counts = np.bincount(bm, minlength=4 ** t)
        assert len(counts) == 4 ** t and counts.min() > 0
        assert counts.max() - counts.min() <= max(2, 4 ** (s - t) // 4)


# ------------------------------------------------------------------ §2.1–2.3 embedding

@pytest.mark.parametrize("pp", PARAMS)
def test_matrix_form_equals_direct_sum(pp):
    p = oracle.Params(N=180, **pp)
    for seed in range(3):
        seq = rand_seq(180, 20 + seed)
        x = oracle.embed(seq, p)
        y = oracle.embed(seq, p, matrix_form=True)
        assert np.abs(x - y).max() < 1e-12 * max(1.0, np.abs(x).max())


@pytest.mark.parametrize("pp", PARAMS)
def test_band_sum_closed_form(pp):
    """Summing a band over all bins gives sum_{l=0}^{N-s} w^{f l}: a geometric
    series, independent of the letters."""
    N = 151
    p = oracle.Params(N=N, **pp)
    nb = 4 ** p.t
    x = oracle.embed(rand_seq(N, 7), p)
    for k in range(1, p.m + 1):
        a, q = oracle.factor(p.m, p.variant, k)
        z = np.exp(2j * np.pi * a / (q * N))
        closed = (1 - z ** (N - p.s + 1)) / (1 - z)
        assert abs(x[(k - 1) * nb:k * nb].sum() - closed) < 1e-11


@pytest.mark.parametrize("s", [1, 2, 3])
def test_norm_of_distinct_smers(s):
    """With every s-mer at most once and t = s, each bin holds one unit phase,
    so ||c^(k)||^2 = N - s + 1 for every band."""
    seq = de_bruijn(4, s)
    N = len(seq)
    for m, variant in ((1, 0), (3, 0), (4, 1)):
        p = oracle.Params(s=s, m=m, t=s, variant=variant, N=N)
        x = oracle.embed(seq, p)
        nb = 4 ** s
        for k in range(m):
            band = x[k * nb:(k + 1) * nb]
            assert np.sum(np.abs(band) ** 2) == pytest.approx(N - s + 1, abs=1e-10)
            assert np.allclose(np.abs(band), 1.0, atol=1e-12)


def test_all_A_and_periodic_give_zero_vector():
    """§3.3: evenly spaced unit phases sum to zero; an all-A string, or a
    periodic one whose period divides N, gives the zero vector (s = 1, default
    factors)."""
    N = 120
    for m in (1, 2, 4):
        p = oracle.Params(s=1, m=m, t=1, variant=0, N=N)
        assert np.abs(oracle.embed(b"A" * N, p)).max() < 1e-12
        assert np.abs(oracle.embed(b"ACGT" * (N // 4), p)).max() < 1e-12
        assert np.abs(oracle.embed(b"GATTAC" * (N // 6), p)).max() < 1e-12
    # the fine-tuned factors (§3.3) break the cancellation for k > 1
    p = oracle.Params(s=1, m=4, t=1, variant=1, N=N)
    x = oracle.embed(b"A" * N, p)
    assert np.abs(x[:4]).max() < 1e-12
    assert np.abs(x[4:]).max() > 0.1


def test_random_walk_modulus():
    """§3.3: the sum of n random unit phases has Rayleigh modulus, mean
    sqrt(n pi)/2."""
    facts = json.load(open(GOLDEN))["random_walk_modulus"]
    N, s = 20000, 2
    p = oracle.Params(s=s, m=1, t=s, variant=0, N=N)
    ratios = []
    for seed in range(12):
        seq = rand_seq(N, 100 + seed)
        x = oracle.embed(seq, p)
        counts = np.bincount(oracle.mer_bins(seq, s, p.bin_map), minlength=16)
        ratios.extend(np.abs(x) / np.sqrt(counts))
    assert np.mean(ratios) == pytest.approx(facts["mean_factor"], rel=0.06)


# ------------------------------------------------------------------ fidelity

def test_fidelity_identity_bounds_phase():
    for pp in PARAMS:
        p = oracle.Params(N=150, **pp)
        x = oracle.embed(rand_seq(150, 1), p)
        y = oracle.embed(rand_seq(150, 2), p)
        assert oracle.fidelity(x, x) == pytest.approx(1.0, abs=1e-14)
        f = oracle.fidelity(x, y)
        assert 0.0 <= f <= 1.0
        assert oracle.fidelity(x, y * np.exp(0.7j)) == pytest.approx(f, abs=1e-14)
        assert oracle.fidelity(3.5 * x, y) == pytest.approx(f, abs=1e-14)
        assert oracle.fidelity(x, np.zeros_like(x)) == 0.0
        # definition written out with numpy's complex inner product
        assert f == pytest.approx(abs(np.vdot(x, y)) ** 2 / (np.vdot(x, x).real * np.vdot(y, y).real), rel=1e-12)


def test_complex_real_identity():
    """§4: |<z1|z2>|^2 = (<x1|x2> + <y1|y2>)^2 + (<x1|y2> - <y1|x2>)^2, the real
    contraction the tensor cores evaluate."""
    p = oracle.Params(N=150)
    for seed in range(5):
        z1 = oracle.embed(rand_seq(150, 30 + seed), p)
        z2 = oracle.embed(rand_seq(150, 40 + seed), p)
        x1, y1, x2, y2 = z1.real, z1.imag, z2.real, z2.imag
        lhs = oracle.fidelity(z1, z2) * np.sum(np.abs(z1) ** 2) * np.sum(np.abs(z2) ** 2)
        rhs = (x1 @ x2 + y1 @ y2) ** 2 + (x1 @ y2 - y1 @ x2) ** 2
        assert lhs == pytest.approx(rhs, rel=1e-12)


def test_fidelity_tracks_mutation():
    """§1/§2.4: more edits, lower fidelity (monotone in expectation)."""
    p = oracle.Params(s=4, m=4, t=4, variant=0, N=1000)
    ref = rand_seq(5000, 77)
    fids = []
    for rate in (0.0, 0.02, 0.1, 0.3):
        rd = synth.reads(ref, 40, seed=5, length=1000, sub_rate=rate / 2, indel_rate=rate / 2)
        f = [oracle.fidelity(oracle.embed(rd.read(i), p), oracle.embed(ref[rd.true_pos[i]:rd.true_pos[i] + 1000], p))
             for i in range(rd.n)]
        fids.append(np.mean(f))
    assert fids[0] == pytest.approx(1.0, abs=1e-12)
    assert fids[0] > fids[1] > fids[2] > fids[3]


def test_per_band_mean_and_shift_invariance():
    """§2.5: for m = 1 a cyclic shift changes c only by a global phase (up to
    the wrapped s-mers), so the fidelity stays near 1; for m > 1 the bands
    rotate by different phases and the concatenated fidelity drops, while the
    per-band mean stays near 1."""
    N, l = 2000, 150
    seq = rand_seq(N, 9)
    shifted = np.concatenate([seq[-l:], seq[:-l]])
    p1 = oracle.Params(s=4, m=1, t=4, variant=0, N=N)
    assert oracle.fidelity(oracle.embed(seq, p1), oracle.embed(shifted, p1)) > 0.97
    p4 = oracle.Params(s=4, m=4, t=4, variant=0, N=N)
    x, y = oracle.embed(seq, p4), oracle.embed(shifted, p4)
    assert oracle.fidelity(x, y) < 0.8
    assert oracle.fidelity_per_band(x, y, 4) > 0.97
    # per-band mean written out band by band
    nb = 4 ** 4
    manual = np.mean([oracle.fidelity(x[k * nb:(k + 1) * nb], y[k * nb:(k + 1) * nb]) for k in range(4)])
    assert oracle.fidelity_per_band(x, y, 4) == pytest.approx(manual, abs=1e-15)


def test_bin_permutation_invariance():
    """With s = t a relabelling of the bins permutes both vectors alike and
    leaves fidelities unchanged."""
    rng = np.random.default_rng(3)
    a, b = rand_seq(150, 50), rand_seq(150, 51)
    p = oracle.Params(s=3, m=2, t=3, variant=1, N=150)
    q = oracle.Params(s=3, m=2, t=3, variant=1, N=150, bin_map=rng.permutation(64).astype(np.uint16))
    assert oracle.fidelity(oracle.embed(a, p), oracle.embed(b, p)) == pytest.approx(
        oracle.fidelity(oracle.embed(a, q), oracle.embed(b, q)), abs=1e-14)


# ------------------------------------------------------------------ §3.4 recurrences

@pytest.mark.parametrize("pp", PARAMS)
def test_window_recurrence_equals_direct(pp):
    ref = rand_seq(3000, 60)
    p = oracle.Params(N=150, **pp)
    rec = oracle.windows_recurrence(ref, p, 17, 2000)
    dirct = oracle.windows_direct(ref, p, 17, 2000)
    assert np.abs(rec - dirct).max() < 1e-11


def test_window_recurrence_on_repeats():
    """The coinciding-exception case (same s-mer leaves and enters) occurs
    constantly on a tandem repeat."""
    ref = np.frombuffer(b"ACGTTGCA" * 100, dtype=np.uint8)
    p = oracle.Params(s=4, m=2, t=2, variant=1, N=64)
    assert np.abs(oracle.windows_recurrence(ref, p, 0, 700) - oracle.windows_direct(ref, p, 0, 700)).max() < 1e-11


@pytest.mark.parametrize("pp", PARAMS[:3])
def test_ip_recurrence_equals_direct(pp):
    ref = rand_seq(2000, 61)
    p = oracle.Params(N=150, **pp)
    x = oracle.embed(rand_seq(150, 62), p)
    ip = oracle.ip_recurrence(ref, p, x, 5, 1500)
    direct = oracle.windows_direct(ref, p, 5, 1500) @ np.conj(x)
    assert np.abs(ip - direct).max() < 1e-10


# ------------------------------------------------------------------ §3.1 / §3.5 exhaustive top-k

def brute_topk(ref, heads, p, k, sep):
    W = oracle.n_windows(len(ref), p.N, p.stride)
    wins = oracle.windows_direct(ref, p, 0, W)
    out_w, out_s = [], []
    for h in heads:
        x = oracle.embed(h, p)
        sc = [(oracle.fidelity(x, wins[j]) if p.score_mode == 0 else oracle.fidelity_per_band(x, wins[j], p.m),
               j * p.stride) for j in range(W)]
        sc.sort(key=lambda t: (-t[0], t[1]))
        got, taken = [], set()
        for s_, w in sc:
            if sep > 0:
                if w // sep in taken:
                    continue
                taken.add(w // sep)
            got.append((w, s_))
            if len(got) == k:
                break
        got += [(-1, -np.inf)] * (k - len(got))
        out_w.append([g[0] for g in got])
        out_s.append([g[1] for g in got])
    return np.array(out_w), np.array(out_s)


@pytest.mark.parametrize("stride,sep,k,mode", [(1, 0, 5, 0), (3, 0, 4, 0), (1, 20, 4, 0), (2, 0, 300, 0),
                                               (1, 0, 6, 1)])
def test_score_topk_brute_force(stride, sep, k, mode):
    ref = rand_seq(400, 70)
    # tandem-repeat patch: exact score ties between distinct windows
    ref[100:180] = np.frombuffer(b"ACGTA" * 16, dtype=np.uint8)
    rd = synth.reads(ref, 6, seed=71, length=40)
    p = oracle.Params(s=3, m=2, t=2, variant=1, N=40, stride=stride, score_mode=mode)
    heads = [rd.read(i)[:40] for i in range(rd.n)]
    bw, bs = brute_topk(ref, heads, p, k, sep)
    ow, os_ = oracle.score_topk(ref, rd.seqs, rd.offsets, p, k=k, sep=sep)
    assert np.array_equal(ow, bw)
    assert np.allclose(os_, bs, rtol=1e-14, atol=0)


def test_score_topk_finds_planted_reads():
    ref = rand_seq(30000, 80)
    rd = synth.reads(ref, 24, seed=81)
    p = oracle.Params(N=150)
    w, s = oracle.score_topk(ref, rd.seqs, rd.offsets, p, k=3)
    hit = np.abs(w[:, 0] - rd.true_pos) <= 150
    assert hit.mean() >= 0.9
    assert np.all(s[:, 0] >= s[:, 1])


def test_score_pairs_matches_topk():
    ref = rand_seq(5000, 90)
    rd = synth.reads(ref, 5, seed=91)
    p = oracle.Params(N=150)
    w, s = oracle.score_topk(ref, rd.seqs, rd.offsets, p, k=4)
    ri = np.repeat(np.arange(5), 4)
    sp = oracle.score_pairs(ref, rd.seqs, rd.offsets, ri, w.ravel(), p)
    assert np.array_equal(sp, s.ravel())


# ------------------------------------------------------------------ Levenshtein (§1)

def brute_levenshtein(a, b):
    """breadth-first search over single edits (tiny strings, alphabet of a+b)"""
    alphabet = sorted(set(a + b)) or ["A"]
    if a == b:
        return 0
    seen = {a}
    frontier = [a]
    d = 0
    limit = len(a) + len(b) + 1
    while frontier and d < limit:
        d += 1
        nxt = []
        for u in frontier:
            cands = set()
            for i in range(len(u) + 1):
                for c in alphabet:
                    cands.add(u[:i] + c + u[i:])
                if i < len(u):
                    cands.add(u[:i] + u[i + 1:])
                    for c in alphabet:
                        cands.add(u[:i] + c + u[i + 1:])
            for v in cands:
                if len(v) > max(len(a), len(b)) + 1 or v in seen:
                    continue
                if v == b:
                    return d
                seen.add(v)
                nxt.append(v)
        frontier = nxt
    raise AssertionError("unreachable")


def test_levenshtein_brute_force():
    words = ["".join(w) for n in range(0, 5) for w in itertools.product("AC", repeat=n)]
    rng = np.random.default_rng(5)
    for a in words:
        for b in rng.choice(words, size=6):
            assert oracle.levenshtein(a, b) == brute_levenshtein(a, str(b))


def test_levenshtein_properties():
    assert oracle.levenshtein("kitten", "sitting") == 3
    rng = np.random.default_rng(6)
    for _ in range(50):
        a, b, c = (bytes(rng.choice(list(LETTERS), size=rng.integers(0, 30))) for _ in range(3))
        dab = oracle.levenshtein(a, b)
        assert dab == oracle.levenshtein(b, a)
        assert oracle.levenshtein(a, a) == 0
        assert oracle.levenshtein(a, b"") == len(a)
        assert dab <= oracle.levenshtein(a, c) + oracle.levenshtein(c, b)
        assert dab >= abs(len(a) - len(b))
        if len(a) == len(b):
            assert dab <= sum(x != y for x, y in zip(a, b))


def test_levenshtein_of_planted_reads_bounded_by_edits():
    ref = rand_seq(20000, 95)
    rd = synth.reads(ref, 50, seed=96, sub_rate=0.03, indel_rate=0.03)
    for i in range(rd.n):
        span = ref[rd.true_pos[i]:rd.true_pos[i] + rd.true_span[i]].tobytes()
        assert oracle.levenshtein(rd.read(i), span) <= rd.n_edits[i]


# ------------------------------------------------------------------ reranker network reference

def _mlp(F=7, H=5, seed=0):
    rng = np.random.default_rng(seed)
    return oracle.MLP(rng.normal(size=(H, F)) * 0.5, rng.normal(size=H) * 0.1, rng.normal(size=H) * 0.5, 0.3)


def test_mlp_forward_gelu_closed_form():
    """GELU(z) = z * Phi(z): with one hidden unit, W1 = e_f, b1 = 0, w2 = 1, b2 = 0
    the network returns z * Phi(z) of the chosen input."""
    from scipy.stats import norm

    net = oracle.MLP(np.array([[0.0, 1.0, 0.0]]), np.zeros(1), np.ones(1), 0.0)
    z = np.array([-3.0, -1.0, -0.2, 0.0, 0.5, 1.0, 2.5])
    X = np.stack([np.full_like(z, 7.0), z, np.full_like(z, -4.0)], axis=1)
    assert np.allclose(net.forward(X), z * norm.cdf(z), rtol=1e-14, atol=1e-16)


def test_mlp_grad_finite_differences():
    net = _mlp()
    rng = np.random.default_rng(1)
    X, t = rng.normal(size=(11, 7)), rng.normal(size=11)
    loss, gW1, gb1, gw2, gb2 = net.grad(X, t)
    assert loss == pytest.approx(np.mean((net.forward(X) - t) ** 2), rel=1e-13)
    h = 1e-6
    for name, arr, g in (("W1", net.W1, gW1), ("b1", net.b1, gb1), ("w2", net.w2, gw2)):
        flat, gflat = arr.reshape(-1), g.reshape(-1)
        for i in range(flat.size):
            old = flat[i]
            flat[i] = old + h
            lp = np.mean((net.forward(X) - t) ** 2)
            flat[i] = old - h
            lm = np.mean((net.forward(X) - t) ** 2)
            flat[i] = old
            assert gflat[i] == pytest.approx((lp - lm) / (2 * h), rel=1e-6, abs=1e-9), (name, i)
    b = net.b2
    net.b2 = b + h
    lp = np.mean((net.forward(X) - t) ** 2)
    net.b2 = b - h
    lm = np.mean((net.forward(X) - t) ** 2)
    net.b2 = b
    assert gb2 == pytest.approx((lp - lm) / (2 * h), rel=1e-6)


def test_adamw_first_step_closed_form():
    """At step 1 the bias-corrected update is -lr * sign(g) (|g| >> eps), plus
    the decoupled decay p * lr * wd."""
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -0.7, 2.0])
    m, v = np.zeros(3), np.zeros(3)
    p0 = p.copy()
    oracle.adamw(p, g, m, v, 1, lr=1e-2, wd=0.1)
    assert np.allclose(p, p0 * (1 - 1e-3) - 1e-2 * np.sign(g), rtol=0, atol=1e-9)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


# ---------------------------------------------------------------- reranker features (oracle)

def test_rerank_features_pins():
    """Feature rows: the Hamming fingerprint fidelities of §1 are 1 for an exact
    copy, find a copy shifted by up to 4 letters, split into halves at N/2; the
    band fidelities average to the per-band score of §2.5; missing rows are 0."""
    ref = synth.uniform_ref(4000, 11)
    p = oracle.Params(s=4, m=2, t=2, variant=1, N=150)
    w = 1000
    head_exact = ref[w:w + 150]
    head_shift = ref[w + 3:w + 153]  # the window 3 letters further on
    mut = head_exact.copy()
    mut[10] = ord("A") if mut[10] != ord("A") else ord("C")  # one substitution in the first half
    seqs = np.concatenate([head_exact, head_shift, mut])
    offs = np.array([0, 150, 300, 450])
    cw = np.array([[w, -1], [w, 200], [w, 3000]])
    cs = np.array([[0.8, -np.inf], [0.7, 0.2], [0.6, 0.5]])
    X = oracle.rerank_features(ref, seqs, offs, cw, cs, p)
    K, m = 2, 2
    assert X.shape == (6, K + 6 + m)
    r0 = X[0]
    one = pytest.approx(1.0, abs=1e-12)
    assert r0[K + 2 + m] == one and r0[K + 3 + m] == one and r0[K + 4 + m] == one and r0[K + 5 + m] == one
    assert np.all(r0[K + 1:K + 1 + m] == pytest.approx(1.0))
    assert np.all(X[1] == 0)                                  # missing candidate
    assert X[0, 1] == 0 and X[0, 0] == 0.8 and X[0, K] == 0.8  # scores, missing = 0
    assert X[3, K + 1 + m] == 0.5                              # rank / K
    r2 = X[2]
    assert r2[K + 3 + m] == one and r2[K + 2 + m] < 0.7       # the shifted copy is found at d = +3
    r4 = X[4]
    assert r4[K + 2 + m] == pytest.approx((149 / 150) ** 2)
    assert r4[K + 4 + m] == pytest.approx((74 / 75) ** 2) and r4[K + 5 + m] == one
    # band fidelities average to the per-band score of the C oracle
    x = oracle.embed(mut, p)
    y = oracle.embed(ref[3000:3150], p)
    assert X[5, K + 1:K + 1 + m].mean() == pytest.approx(oracle.fidelity_per_band(x, y, m), rel=1e-12)


def test_hamming_fingerprint_other_letters():
    """§1 fingerprint over {A, C, G, T, other}: a letter outside ACGT is one
    more alphabet letter, so it mismatches every base."""
    assert oracle.hamming_fingerprint_fidelity(b"ACGT", b"ACGN") == pytest.approx((3 / 4) ** 2)
    assert oracle.hamming_fingerprint_fidelity(b"NNAC", b"GTAC") == pytest.approx((2 / 4) ** 2)
    assert oracle.hamming_fingerprint_fidelity(b"ACGTACGT", b"TGCATGCA") == pytest.approx(0.0, abs=1e-15)


def test_reverse_complement_and_strands():
    """The other strand: reversal with A<->T, C<->G, an involution; a read that
    is the reverse complement of a window is found there on strand 1 with
    fidelity 1, and a forward copy on strand 0."""
    assert bytes(oracle.reverse_complement(b"ACGTTG")) == b"CAACGT"
    s = synth.uniform_ref(500, 3)
    assert np.array_equal(oracle.reverse_complement(oracle.reverse_complement(s)), s)
    ref = synth.uniform_ref(3000, 4)
    p = oracle.Params(s=4, m=2, t=2, variant=1, N=150)
    fwd = ref[700:850]
    rev = oracle.reverse_complement(ref[1900:2050])
    seqs = np.concatenate([fwd, rev])
    w, sc, t = oracle.score_topk_strands(ref, seqs, np.array([0, 150, 300]), p, k=3)
    assert w[0, 0] == 700 and t[0, 0] == 0 and sc[0, 0] == pytest.approx(1.0, abs=1e-9)
    assert w[1, 0] == 1900 and t[1, 0] == 1 and sc[1, 0] == pytest.approx(1.0, abs=1e-9)
    assert np.all(np.diff(sc, axis=1) <= 0)


# ---------------------------------------------------------------- refinement (§3.4, increasing the accuracy)

@pytest.mark.parametrize("pp", [dict(s=4, m=2, t=2, variant=1), dict(s=8, m=1, t=8, variant=0),
                                dict(s=5, m=3, t=3, variant=1, score_mode=1)])
def test_refine_finds_exact_reads(pp):
    """An error-free read is its own window: fidelity 1 (identity) at the true
    start, which the refinement finds from any candidate within the radius;
    a random reference has no other window at fidelity 1."""
    ref = synth.uniform_ref(6000, 71)
    rd = synth.reads(ref, 12, seed=72, sub_rate=0.0, indel_rate=0.0)
    op = oracle.Params(N=150, **pp)
    rng = np.random.default_rng(73)
    cand = rd.true_pos[:, None] + rng.integers(-9, 10, size=(12, 3))
    pos, fid, _ = oracle.refine(ref, rd.seqs, rd.offsets, cand, 9, op)
    ok = (cand >= 0) & (cand <= len(ref) - 150)
    assert np.all(pos[ok] == np.broadcast_to(rd.true_pos[:, None], pos.shape)[ok])
    assert np.allclose(fid[ok], 1.0, atol=1e-12)


def test_refine_range_clipping_and_missing():
    ref = synth.uniform_ref(2000, 81)
    rd = synth.reads(ref, 3, seed=82)
    op = oracle.Params(N=150)
    last = len(ref) - 150
    cand = np.array([[3, -1], [last - 2, 0], [last + 40, 1000]], dtype=np.int64)
    pos, fid, (owner, scored, _) = oracle.refine(ref, rd.seqs, rd.offsets, cand, 5, op)
    assert pos[0, 1] == -1 and np.isneginf(fid[0, 1])
    # each candidate's scored positions are exactly its clipped range
    want = {0: range(0, 9), 2: range(last - 7, last + 1), 3: range(0, 6), 4: range(last - 5, last + 1),
            5: range(995, 1006)}
    for o, rng_ in want.items():
        assert scored[owner == o].tolist() == list(rng_)
    assert np.all((pos[pos >= 0] >= 0) & (pos[pos >= 0] <= last))
    # radius 0 returns the candidate itself
    p0, f0, _ = oracle.refine(ref, rd.seqs, rd.offsets, np.array([[500], [17], [1200]]), 0, op)
    assert p0[:, 0].tolist() == [500, 17, 1200]


def test_refine_ties_take_the_lower_position():
    """A reference of period 8 repeats every window 8 letters on: a read equal
    to one window scores fidelity 1 at every start of the same phase, and the
    lowest of them in the range is returned."""
    unit = np.frombuffer(b"ACGGTCAT", dtype=np.uint8)
    ref = np.tile(unit, 200).copy()
    read = ref[100:250].copy()
    offs = np.array([0, 150], dtype=np.int64)
    op = oracle.Params(N=150)
    pos, fid, _ = oracle.refine(ref, read, offs, np.array([[300]]), 20, op)
    assert pos[0, 0] == 284 and fid[0, 0] == pytest.approx(1.0, abs=1e-12)  # 284 = 100 (mod 8), >= 280


# ---------------------------------------------------------------- threshold regime (§3.4 thresholds, §3.5 output)

def test_splitmix64_published_vector():
    """SplitMix64 started at state 0: the published first three outputs."""
    assert [oracle.splitmix64(0, i) for i in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                          0x06C45D188009454F]


def test_mutate_rate_split_and_edit_bound():
    """Mutations occur at the given rate per reference letter, split evenly
    between deletions, insertions and substitutions; a copy with no mutation
    is the reference itself; and the copy is within (number of applied
    mutations) edits of the reference letters it walked."""
    ref = synth.uniform_ref(50_000, 131)
    c, cnt = oracle.mutate(ref, 1000, 150, 0.0, 5, 0)
    assert bytes(c) == bytes(ref[1000:1150]).upper() and cnt == (150, 0, 0, 0)
    tot = np.zeros(4)
    for k in range(600):
        c, cnt = oracle.mutate(ref, 37 * k, 150, 0.3, 11, k)
        walked, nd, ni, ns = cnt
        ld = oracle.levenshtein(c, ref[37 * k:37 * k + walked])
        assert ld <= nd + ni + ns
        tot += cnt
    n_mut = tot[1:].sum()
    assert abs(n_mut / tot[0] - 0.3) < 4 * math.sqrt(0.3 * 0.7 / tot[0])
    for share in tot[1:] / n_mut:
        assert abs(share - 1 / 3) < 4 * math.sqrt(2 / 9 / n_mut)


def test_fragment_thresholds_identity_and_monotone():
    """At rate 0 every copy is the fragment: threshold 1 (identity); the mean
    threshold falls as the mutation rate grows and stays in [0, 1]."""
    ref = synth.uniform_ref(8000, 141)
    op = oracle.Params(N=150)
    assert np.allclose(oracle.fragment_thresholds(ref, op, 0.0, 3, 1, 0, 200), 1.0, atol=1e-12)
    means = [oracle.fragment_thresholds(ref, op, e, 8, 2, 0, 300).mean() for e in (0.02, 0.1, 0.3)]
    assert 1.0 > means[0] > means[1] > means[2] > 0.0


def test_threshold_pairs_against_topk():
    """Exhaustive threshold output agrees with the exhaustive top-k: with a
    threshold of 0 every pair is reported; with a constant threshold t, each
    read's pairs are exactly its windows of the top-k list scoring >= t."""
    ref = synth.uniform_ref(3000, 151)
    rd = synth.reads(ref, 6, seed=152)
    op = oracle.Params(N=150)
    W = oracle.n_windows(len(ref), 150, 1)
    r, w, f = oracle.threshold_pairs(ref, rd.seqs, rd.offsets, op, np.zeros(W))
    assert len(r) == 6 * W
    ow, os_ = oracle.score_topk(ref, rd.seqs, rd.offsets, op, k=200)
    t = 0.3
    r, w, f = oracle.threshold_pairs(ref, rd.seqs, rd.offsets, op, np.full(W, t))
    for i in range(6):
        want = set(ow[i][os_[i] >= t].tolist())
        assert len(want) < 200  # the top-200 list reaches below t
        assert set(w[r == i].tolist()) == want


def test_refine_scores_follow_the_ip_recurrence():
    """The fidelities the refinement oracle scores along a candidate's range
    equal |ip|^2 / (X C) with ip from the paper's one-letter slide relation
    (§3.4) and C from the direct window encodings."""
    ref = synth.uniform_ref(4000, 161)
    rd = synth.reads(ref, 1, seed=162)
    p = oracle.Params(s=4, m=2, t=2, variant=1, N=150)
    c0 = int(rd.true_pos[0])
    _, _, (owner, pos, fid) = oracle.refine(ref, rd.seqs, rd.offsets, np.array([[c0]]), 12, p)
    x = oracle.embed(rd.seqs[:150], p)
    lo = int(pos[0])
    ip = oracle.ip_recurrence(ref, p, x, lo, len(pos))
    C = np.sum(np.abs(oracle.windows_direct(ref, p, lo, len(pos))) ** 2, axis=1)
    X = np.sum(np.abs(x) ** 2)
    assert np.allclose(fid, np.abs(ip) ** 2 / (X * C), rtol=1e-10, atol=1e-14)


# ---------------------------------------------------------------- fitting curve (§2.4 scoring of correlations)

def test_fitting_curve_rate_zero_and_monotone():
    p = oracle.Params(s=4, m=2, t=2, variant=1, N=1000)
    dnas = [synth.uniform_ref(1400, 200 + i) for i in range(160)]
    assert np.allclose(oracle.pair_fidelities(dnas[:10], np.zeros(10), p, 3), 1.0, atol=1e-12)
    errs = np.random.default_rng(4).uniform(0, 0.5, 160)
    fids = oracle.pair_fidelities(dnas, errs, p, 3)
    c, m = oracle.fitting_curve(errs, fids, n_bins=8)
    assert np.all(np.diff(m) < 0) and m[0] < 1.0 and m[-1] > 0.0


def test_fitting_curve_rmse_as_printed():
    """The paper's random-pair experiment (20,000-letter random strings,
    4096 complex dimensions, mutation rates uniform in (0, 0.5) split evenly
    between deletions, insertions and substitutions) predicts the rate from
    the fidelity with an RMSE under 1% where the rate is below 25%; here with
    s = t = 6, m = 1 (4^6 = 4096 bins)."""
    N = 20_000
    p = oracle.Params(s=6, m=1, t=6, variant=0, N=N)
    n = 400
    dnas = [synth.uniform_ref(N + 4000, 300 + i) for i in range(n)]
    errs = np.random.default_rng(5).uniform(0, 0.5, n)
    fids = oracle.pair_fidelities(dnas, errs, p, 6)
    curve = oracle.fitting_curve(errs, fids, n_bins=10)
    assert oracle.prediction_rmse(errs, fids, curve, below=0.25) < 0.01
