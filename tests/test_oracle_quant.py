"""Pins for the q-bit input forms of the oracle (Sec. IV-C): unpacking of
floor(32/q) q-bit soft values per 32-bit word, the branch metric with
mu = +-Q (Q = 2^(q-1) - 1; hard decisions for q = 1), and the block form on
such values."""
import os

import numpy as np
import pytest

import oracle
from paper_1608_00066_gb300 import synth

K3 = (0o7, 0o5)
K7 = (0o171, 0o133)


def _rows(golden_dir):
    with open(os.path.join(golden_dir, "packed_soft_example.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                q, vals, word = line.split(":")
                yield int(q), [int(x) for x in vals.split()], int(word)


def test_unpack_hand_packed_words(golden_dir):
    for q, vals, word in _rows(golden_dir):
        got = oracle.unpack_soft(q, [word], len(vals))
        want = [(1 if v > 0 else -1) if q == 1 else v for v in vals]
        assert got.tolist() == want, q
        assert synth.pack_q(np.array(vals), q).tolist() == [word], q


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5, 8])
def test_pack_unpack_round_trip(q):
    rng = np.random.default_rng(q)
    Q = oracle.q_max(q)
    lo = -1 if q == 1 else -(1 << (q - 1))
    vals = rng.integers(lo, Q + 1, size=1001)
    if q == 1:
        vals = np.where(vals < 0, -1, 1)
    words = synth.pack_q(vals, q)
    assert len(words) == (1001 + 32 // q - 1) // (32 // q)
    assert oracle.unpack_soft(q, words, 1001).tolist() == vals.tolist()


def test_branch_metric_q_closed_forms():
    for q in (1, 3, 4, 8):
        Q = oracle.q_max(q)
        for R in (2, 3):
            for c in range(1 << R):
                for rx in range(1 << R):
                    lam = [Q - 2 * Q * ((rx >> (R - 1 - r)) & 1) for r in range(R)]
                    # hard values: 2Q per differing code bit
                    assert oracle.branch_metric_q(lam, c, Q) == 2 * Q * bin(c ^ rx).count("1")
                if q > 1:
                    assert oracle.branch_metric_q([0] * R, c, Q) == Q * R
                    assert oracle.branch_metric_q([-Q - 1] * R, c, Q) == oracle.branch_metric_q([-Q] * R, c, Q)
    rng = np.random.default_rng(1)
    for _ in range(50):
        lam = rng.integers(-127, 128, size=2)
        for c in range(4):
            assert oracle.branch_metric_q(lam, c, 127) == oracle.branch_metric(lam, c)


def test_block_q_with_q127_is_the_block_form():
    rng = np.random.default_rng(2)
    llr = rng.integers(-127, 128, size=(3000, 2)).astype(np.int8)
    for D, L in ((64, 42), (512, 0), (8, 20)):
        assert np.array_equal(oracle.viterbi_block_q(7, K7, llr, D, L, 127), oracle.viterbi_block(7, K7, llr, D, L))


def _search_q(K, gens, rows, Q, known_start):
    """Exhaustive search over a window's paths with the q-bit metric, ending in
    S_0: (smallest metric, count, first minimiser's input bits)."""
    R = len(gens)
    v = K - 1
    N = 1 << v
    m = len(rows)
    table = oracle.output_table(K, gens)
    starts = np.array([0] if known_start else list(range(N)), dtype=np.int64)
    xs = np.arange(1 << m, dtype=np.int64)
    d = np.repeat(starts, 1 << m)
    x_all = np.tile(xs, len(starts))
    metric = np.zeros(d.shape, dtype=np.int64)
    for t in range(m):
        x = (x_all >> t) & 1
        lam = [max(int(l), -Q) for l in rows[t]]
        bm = np.array([sum(abs(lam[r] - (-Q if (c >> (R - 1 - r)) & 1 else Q)) for r in range(R))
                       for c in range(1 << R)], dtype=np.int64)
        metric += bm[table[d, x]]
        d = (d >> 1) | (x << (v - 1))
    ok = d == 0
    best = metric[ok].min()
    hits = np.flatnonzero(ok & (metric == best))
    first = int(x_all[hits[0]])
    return int(best), len(hits), [(first >> t) & 1 for t in range(m)]


@pytest.mark.parametrize("q", [1, 2, 3, 4])
@pytest.mark.parametrize("K,gens,n,D,L", [(3, K3, 21, 8, 3), (5, (0o23, 0o35), 26, 8, 3), (7, K7, 22, 8, 2)])
def test_block_q_equals_exhaustive_search(q, K, gens, n, D, L):
    Q = oracle.q_max(q)
    spec = synth.CodeSpec("t", K, tuple(gens))
    unique = 0
    for seed in range(4):
        f = synth.make_packed_frame(spec, n - (K - 1), -1.0 + seed, q, seed=40 + seed)
        vals = oracle.unpack_soft(q, f.words, n * spec.R).reshape(n, spec.R)
        bits = oracle.viterbi_block_q(K, gens, vals, D, L, Q)
        for b in range((n + D - 1) // D):
            f0, f1 = max(0, b * D - L), min(n, (b + 1) * D + L) - 1
            o0, o1 = b * D, min((b + 1) * D, n)
            best, count, path = _search_q(K, gens, [vals[s] for s in range(f0, f1 + 1)], Q, f0 == 0)
            if count == 1:
                unique += 1
                assert bits[o0:o1].tolist() == path[o0 - f0:o1 - f0], (q, K, b)
    assert unique > 0


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_scaled_int8_values_decode_the_same(q):
    """Multiplying q-bit values by s = floor(127 / Q) maps the q-bit metric to
    s * BM_q + (127 - s Q) R per stage (|s lambda| < 127), a positive-affine
    change of every branch metric of the stage, so the decisions, ties
    included, and hence the bits are those of the q-bit metric."""
    Q = oracle.q_max(q)
    s = 127 // Q
    for K, gens, D, L in ((7, K7, 64, 42), (3, K3, 8, 6), (9, (0o557, 0o663, 0o711), 128, 64)):
        spec = synth.CodeSpec("t", K, tuple(gens))
        f = synth.make_packed_frame(spec, 4000, 1.0, q, seed=q * K)
        vals = oracle.unpack_soft(q, f.words, f.n_stages * spec.R).reshape(-1, spec.R)
        want = oracle.viterbi_block_q(K, gens, vals, D, L, Q)
        scaled = (np.maximum(vals.astype(np.int16), -Q) * s).astype(np.int8)
        assert np.array_equal(oracle.viterbi_block(K, gens, scaled, D, L), want), (q, K)


@pytest.mark.parametrize("q", [1, 2, 3, 4])
@pytest.mark.parametrize("K, gens", [(7, K7), (5, (0o23, 0o35)), (7, (0o171, 0o165, 0o133))])
def test_metric_spread_bound(q, K, gens):
    """The bound that 8-bit path metrics rest on, read off the oracle's own
    metrics: with the q-bit branch metric (in [0, 2QR]) every state is reached
    from the best state of v = K - 1 stages earlier, so from stage v - 1 on
    (known start, every state reachable) max - min <= v * 2QR, and the
    smallest metric grows by at most 2QR per stage.  The oracle's full-frame
    form runs on the scaled int8 values (s * BM_q plus the same offset on
    every branch of a stage), so metric differences are s times the q-bit
    ones.  Noisy frames and words of uniformly random bits (every q-bit code,
    the clamped -Q-1 included); the bound is also reached or approached, so a
    looser constant would not pass unnoticed."""
    Q = oracle.q_max(q)
    s = 127 // Q
    R = len(gens)
    v = K - 1
    bm_span = 2 * Q * R
    offset = (127 - s * Q) * R
    spec = synth.CodeSpec("t", K, tuple(gens))
    rng = np.random.default_rng(q * 31 + K + R)
    m = 32 // q
    worst = 0
    for kind in ("noisy", "random", "clean"):
        if kind == "noisy":
            f = synth.make_packed_frame(spec, 3000, 0.0, q, seed=q + 7 * K)
            n = f.n_stages
            vals = oracle.unpack_soft(q, f.words, n * R).reshape(n, R)
        elif kind == "random":
            n = 3000
            words = rng.integers(0, 1 << 32, size=(n * R + m - 1) // m, dtype=np.uint64).astype(np.uint32)
            vals = oracle.unpack_soft(q, words, n * R).reshape(n, R)
        else:
            # the all-zero codeword received without noise: every other path
            # pays for each of its code bits, which spreads the metrics most
            n = 200
            vals = np.full((n, R), Q, dtype=np.int8)
        scaled = (np.maximum(vals.astype(np.int16), -Q) * s).astype(np.int8)
        _, _, _, pm = oracle.viterbi_full(K, gens, scaled, want_trace=True)
        spread = (pm.max(axis=1) - pm.min(axis=1))[v - 1:]
        assert np.all(spread % s == 0)
        assert int(spread.max()) // s <= v * bm_span, (kind, int(spread.max()) // s)
        worst = max(worst, int(spread.max()) // s)
        grow = np.diff(pm.min(axis=1)) - offset
        assert np.all(grow >= 0) and np.all(grow <= s * bm_span), kind
    assert 3 * worst >= 2 * v * bm_span, worst


def test_hard_decision_worked_example(golden_dir):
    """The hand-traced K=3 example read as hard decisions: every metric is the
    traced one divided by 127 (254 per differing bit becomes 2), the survivor
    bits are the traced ones, and the frame decodes to 1 0 1 1 0 0."""
    rows = {}
    stages = []
    with open(os.path.join(golden_dir, "k3_75_worked_example.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("stage"):
                _, pm, dec = line.split(":")
                stages.append(([int(x) for x in pm.split()], [int(x) for x in dec.split()]))
            else:
                k, v = line.split(None, 1)
                rows[k] = [int(x) for x in v.split()]
    vals = np.array([1 - 2 * b for b in rows["rx"]], np.int8).reshape(-1, 2)
    pm = np.array([0, oracle.BIG, oracle.BIG, oracle.BIG], np.int64)
    for s, (want_pm, want_dec) in enumerate(stages):
        pm, dec = oracle.acs_stage_q(3, K3, vals[s], 1, pm)
        assert dec.tolist() == want_dec, s
        big = [oracle.BIG if w >= oracle.BIG else 0 for w in want_pm]
        assert pm.tolist() == [b + (w - b) // 127 for w, b in zip(want_pm, big)], s
    bits = oracle.viterbi_block_q(3, K3, vals, 8, 4, 1)
    assert bits.tolist() == rows["decoded"]
