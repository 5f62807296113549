"""Pins for the block-form variants of the oracle:

  * argmin start: the traceback of each block starts from the state with the
    smallest metric at f1 (the start state S_E of the classic Viterbi
    algorithm, Sec. II) instead of S_0;
  * tail-biting frames (not in the paper): circular windows, stage s reads
    the soft values of s mod n, zero initial metrics in every block.

Each is checked against an exhaustive search over the paths of every block's
window, and against hand-traced values where the fixture has them."""
import numpy as np
import pytest

import oracle
from paper_1608_00066_gb300 import synth

from test_oracle_blocks import _geometry, _golden, _stage_metrics

K3 = (0o7, 0o5)
K5 = (0o23, 0o35)
K7 = (0o171, 0o133)


def search(K, gens, llr_rows, known_start, any_end):
    """Exhaustive search over the paths of a window given as its soft-value
    rows (stage t of the window = row t): smallest metric over paths that
    start in any state at zero cost (or in S_0 with a known start) and end in
    S_0 (or in any state), how many reach it, and the first minimiser's input
    bits."""
    R = len(gens)
    v = K - 1
    N = 1 << v
    m = len(llr_rows)
    table = oracle.output_table(K, gens)
    starts = np.array([0] if known_start else list(range(N)), dtype=np.int64)
    xs = np.arange(1 << m, dtype=np.int64)
    d = np.repeat(starts, 1 << m)
    x_all = np.tile(xs, len(starts))
    metric = np.zeros(d.shape, dtype=np.int64)
    for t in range(m):
        x = (x_all >> t) & 1
        metric += _stage_metrics(llr_rows[t], R)[table[d, x]]
        d = (d >> 1) | (x << (v - 1))
    ok = np.ones(d.shape, bool) if any_end else d == 0
    best = metric[ok].min()
    hits = np.flatnonzero(ok & (metric == best))
    first = int(x_all[hits[0]])
    return int(best), len(hits), [(first >> t) & 1 for t in range(m)]


def _windows(n, D, L, circular):
    nb = (n + D - 1) // D
    for b in range(nb):
        f0, f1, o0, o1 = _geometry(n, D, L, b)
        if circular:
            f0, f1 = o0 - L, o1 + L - 1
        yield b, f0, f1, o0, o1


def _check(K, gens, llr, D, L, argmin, circular):
    n = llr.shape[0]
    bits, pm_end = oracle.viterbi_block_variant(K, gens, llr, D, L, argmin=argmin, circular=circular)
    unique = 0
    for b, f0, f1, o0, o1 in _windows(n, D, L, circular):
        rows = [llr[s % n] for s in range(f0, f1 + 1)]
        best, count, path = search(K, gens, rows, known_start=(f0 == 0 and not circular), any_end=argmin)
        assert pm_end[b] == best, (K, D, L, b, argmin, circular)
        if count == 1:
            unique += 1
            assert bits[o0:o1].tolist() == path[o0 - f0:o1 - f0], (K, D, L, b, argmin, circular)
    return unique


CASES = [(3, K3, 12, 4, 2), (3, K3, 21, 8, 3), (3, K3, 13, 4, 5), (5, K5, 26, 8, 3),
         (7, K7, 22, 8, 2), (7, K7, 27, 4, 4), (4, (0o13, 0o16), 23, 4, 4)]


def test_default_flags_are_the_block_form():
    rng = np.random.default_rng(3)
    llr = rng.integers(-128, 128, size=(500, 2)).astype(np.int8)
    for D, L in ((64, 42), (8, 3), (512, 0)):
        a, pa = oracle.viterbi_block_variant(7, K7, llr, D, L)
        nb = (500 + D - 1) // D
        b, pb = oracle.viterbi_block_metrics(7, K7, llr, D, L, (0, nb))
        assert np.array_equal(a, b) and np.array_equal(pa, pb)


@pytest.mark.parametrize("K,gens,n,D,L", CASES)
@pytest.mark.parametrize("argmin,circular", [(True, False), (False, True), (True, True)])
def test_variants_equal_exhaustive_search(K, gens, n, D, L, argmin, circular):
    R = len(gens)
    rng = np.random.default_rng(10 * K + n + D + L + 2 * argmin + circular)
    unique = 0
    for trial in range(4):
        llr = rng.integers(-128, 128, size=(n, R)).astype(np.int8)
        unique += _check(K, gens, llr, D, L, argmin, circular)
    spec = synth.CodeSpec("t", K, tuple(gens))
    f = synth.make_frame(spec, n - (K - 1), ebn0_db=0.0, seed=n)
    unique += _check(K, gens, f.llr.reshape(-1, R), D, L, argmin, circular)
    assert unique > 0


def test_hand_traced_interior_block_argmin(golden_dir):
    """Block 1 of the hand-traced K=3 example in argmin mode: the cheapest
    state after stage 9 is S_3 (254), whose traceback gives 1 0 1 1."""
    kv, stages = _golden(golden_dir, "k3_75_interior_block.txt")
    llr = (127 - 254 * np.array(kv["rx"], dtype=np.int16)).astype(np.int8).reshape(-1, 2)
    b, D, L = kv["block"]
    bits, pm_end = oracle.viterbi_block_variant(3, K3, llr, D, L, argmin=True, blocks=(b, b + 1))
    last_pm = stages[-1][1]
    assert pm_end[0] == min(last_pm) == 254
    assert bits[b * D:(b + 1) * D].tolist() == kv["argmin_decoded"]


@pytest.mark.parametrize("K,gens", [(3, K3), (5, K5), (7, K7), (9, (0o557, 0o663, 0o711)), (4, (0o13, 0o16))])
def test_tailbiting_encoder(K, gens):
    """The encoder ends in the state it starts in, and its output is the
    circular convolution of the message with each generator over GF(2)."""
    spec = synth.CodeSpec("t", K, tuple(gens))
    rng = np.random.default_rng(K)
    for k in (K - 1, K, 37, 300):
        msg = rng.integers(0, 2, size=k, dtype=np.uint8)
        assert np.array_equal(oracle.encode_tailbiting(K, gens, msg), synth.conv_encode_tailbiting(spec, msg))
        # the same bits as the zero-start encoder run over the message twice
        twice = oracle.encode(K, gens, np.concatenate([msg, msg]))[k:2 * k]
        assert np.array_equal(oracle.encode_tailbiting(K, gens, msg), twice)


@pytest.mark.parametrize("name", ["K3_r1/2", "K7_r1/2", "K9_r1/3"])
def test_tailbiting_noiseless_round_trip(name):
    spec = synth.CODES[name]
    for k, D, L in ((3000, 64, 6 * spec.K), (40, 512, 6 * spec.K), (700, 8, 3 * spec.K)):
        f = synth.make_tailbiting_frame(spec, k, None, seed=k)
        for argmin in (False, True):
            bits, _ = oracle.viterbi_block_variant(spec.K, spec.gens, f.llr.reshape(-1, spec.R), D, L,
                                                   argmin=argmin, circular=True)
            assert np.array_equal(bits, f.msg), (name, k, D, L, argmin)


def test_argmin_ties_keep_the_lowest_state():
    """All-zero soft values tie every state at f1.  With L = 0 or 1 the last
    stages' bits are emitted, so the start state shows: the lowest index, S_0,
    gives all zeros (the highest would emit ones)."""
    for K, gens in ((3, K3), (7, K7), (9, (0o557, 0o663, 0o711))):
        R = len(gens)
        zeros = np.zeros((40, R), np.int8)
        for L in (0, 1):
            for circular in (False, True):
                bits, pm_end = oracle.viterbi_block_variant(K, gens, zeros, 8, L, argmin=True, circular=circular)
                assert not bits.any(), (K, L, circular)
