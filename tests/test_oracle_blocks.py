"""Pins for the block form of the oracle (Sec. III-A, Algorithm 1) that do not
reduce it to the full-frame decoder: every block, interior ones included, is
checked against an exhaustive search over all paths of its forward window.

What Sec. III-A fixes for a block b of a stream of n stages:
  * its forward range is [f0, f1], f0 = max(0, bD - L), f1 = min(n, (b+1)D + L) - 1;
  * its initial metrics are unknown and set to zero, so the search starts from
    every state at f0 with no cost -- except for a block whose range begins at
    stage 0, which starts from the encoder's known state S_0;
  * the traceback starts from S_0 at f1 with no metric comparison, so the
    path it follows is the cheapest path that ends in S_0 at f1;
  * the block emits the input bits of that path at stages [bD, min((b+1)D, n)).

The exhaustive search below enumerates (start state, input bits over the
window), sums the branch metrics along each path and keeps the paths that end
in S_0.  The oracle's PM(S_0) at f1 must equal the smallest sum, and its output
bits must equal the minimiser's input bits whenever the minimiser is unique.
"""
import numpy as np
import pytest

import oracle
from paper_1608_00066_gb300 import synth

K3 = (0o7, 0o5)
K5 = (0o23, 0o35)
K7 = (0o171, 0o133)


def _stage_metrics(llr_stage, R):
    """Distance of one stage's soft values to each of the 2^R codewords
    (c^(1) most significant), by the metric of Sec. II: sum of |lambda - mu|
    with mu(0) = +127, mu(1) = -127 and -128 read as -127."""
    lam = np.maximum(np.asarray(llr_stage, dtype=np.int64), -127)
    out = np.zeros(1 << R, dtype=np.int64)
    for c in range(1 << R):
        for r in range(R):
            mu = -127 if (c >> (R - 1 - r)) & 1 else 127
            out[c] += abs(int(lam[r]) - mu)
    return out


def brute_block(K, gens, llr, f0, f1, known_start):
    """Exhaustive search over the paths of the window [f0, f1].

    Returns (smallest metric of a path ending in S_0 at f1, number of paths
    reaching it, input bits of the first such path at stages f0..f1)."""
    R = len(gens)
    v = K - 1
    N = 1 << v
    m = f1 - f0 + 1
    table = oracle.output_table(K, gens)           # codeword c(S_d, x)
    starts = np.array([0] if known_start else list(range(N)), dtype=np.int64)
    xs = np.arange(1 << m, dtype=np.int64)          # bit t = input at stage f0 + t
    d = np.repeat(starts, 1 << m)
    x_all = np.tile(xs, len(starts))
    metric = np.zeros(d.shape, dtype=np.int64)
    for t in range(m):
        x = (x_all >> t) & 1
        bm = _stage_metrics(llr[f0 + t], R)
        metric += bm[table[d, x]]
        d = (d >> 1) | (x << (v - 1))               # butterfly of Sec. III-B
    ok = d == 0
    best = metric[ok].min()
    hits = np.flatnonzero(ok & (metric == best))
    first = x_all[hits[0]]
    bits = [(int(first) >> t) & 1 for t in range(m)]
    return int(best), len(hits), bits


def _geometry(n, D, L, b):
    f0 = max(0, b * D - L)
    f1 = min(n, (b + 1) * D + L) - 1
    return f0, f1, b * D, min((b + 1) * D, n)


def _check_all_blocks(K, gens, llr, D, L):
    """Every block of the stream against the exhaustive search; returns how
    many blocks had a unique minimiser (whose bits were compared)."""
    n = llr.shape[0]
    nb = (n + D - 1) // D
    bits, pm_end = oracle.viterbi_block_metrics(K, gens, llr, D, L, (0, nb))
    unique = 0
    for b in range(nb):
        f0, f1, o0, o1 = _geometry(n, D, L, b)
        best, count, path = brute_block(K, gens, llr, f0, f1, known_start=(f0 == 0))
        assert pm_end[b] == best, (K, D, L, b, pm_end[b], best)
        if count == 1:
            unique += 1
            want = path[o0 - f0:o1 - f0]
            assert bits[o0:o1].tolist() == want, (K, D, L, b)
    return unique


# (K, gens, n, D, L): windows of at most 16 stages so that the search stays small
CASES = [
    (3, K3, 12, 4, 2),
    (3, K3, 30, 8, 3),
    (3, K3, 21, 8, 0),
    (3, K3, 19, 4, 5),      # L > D: interior windows reach over two neighbours
    (5, K5, 26, 8, 3),
    (5, K5, 29, 4, 4),
    (7, K7, 22, 8, 2),
    (7, K7, 27, 4, 4),
    (7, (0o171, 0o165, 0o133), 18, 4, 3),   # R = 3
    (4, (0o13, 0o16), 23, 4, 4),           # g_{K-1} != g_0
]


@pytest.mark.parametrize("K,gens,n,D,L", CASES)
def test_blocks_equal_exhaustive_search_random_soft_values(K, gens, n, D, L):
    """Uniform random soft values: the start state that the search picks is
    rarely S_0, and the cheapest end state rarely S_0, so a block that started
    from the known state or traced back from the cheapest state would fail."""
    R = len(gens)
    rng = np.random.default_rng(100 * K + n + D + L)
    unique = 0
    for trial in range(4):
        llr = rng.integers(-128, 128, size=(n, R)).astype(np.int8)
        unique += _check_all_blocks(K, gens, llr, D, L)
    assert unique > 0


@pytest.mark.parametrize("K,gens,n,D,L", CASES[:8])
def test_blocks_equal_exhaustive_search_awgn(K, gens, n, D, L):
    """Soft values of a sent codeword over AWGN at low Eb/N0 (the workloads'
    recipe), message bits drawn at random: mostly unique minimisers."""
    spec = synth.CodeSpec("t", K, tuple(gens))
    unique = 0
    for seed in range(3):
        f = synth.make_frame(spec, n - (K - 1), ebn0_db=-1.0 + seed, seed=700 + seed)
        llr = f.llr.reshape(-1, spec.R)
        unique += _check_all_blocks(K, gens, llr, D, L)
    assert unique > 0


def test_interior_start_is_free_and_end_is_s0():
    """A hand-made case that separates the readings of Sec. III-A: block 1 of
    a K=3 stream whose window [2, 9] carries the noiseless codeword of a path
    that starts in S_3 and ends in S_3.  From free (zero) initial metrics the
    search finds that path's prefix at no cost; from the known start it could
    not; and the traceback from S_0 at f1 must leave the cheapest end state."""
    K, n, D, L = 3, 12, 4, 2
    # message bits x_0..x_9 then the tail; x_0 = x_1 = 1 leaves the encoder in S_3
    msg = [1, 1, 0, 1, 1, 0, 1, 1, 1, 1]
    code = synth.conv_encode(synth.CodeSpec("t", 3, K3), np.array(msg, np.uint8))
    llr = synth.noiseless_int8(code.reshape(-1)).reshape(-1, 2)
    f0, f1, o0, o1 = _geometry(n, D, L, 1)
    assert (f0, f1, o0, o1) == (2, 9, 4, 8)
    free_best, _, _ = brute_block(K, K3, llr, f0, f1, known_start=False)
    s0_best, _, _ = brute_block(K, K3, llr, f0, f1, known_start=True)
    assert free_best < s0_best           # the readings differ on this window
    bits, pm_end = oracle.viterbi_block_metrics(K, K3, llr, D, L, (1, 2))
    assert pm_end[0] == free_best
    best, count, path = brute_block(K, K3, llr, f0, f1, known_start=False)
    assert count == 1
    assert bits[o0:o1].tolist() == path[o0 - f0:o1 - f0]


# --------------------------------------------------- hand-traced interior block

def _golden(golden_dir, name):
    import os
    kv, stages = {}, []
    with open(os.path.join(golden_dir, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("stage"):
                head, pm, dec = line.split(":")
                stages.append((int(head.split()[1]), [int(x) for x in pm.split()],
                               [int(x) for x in dec.split()]))
            else:
                k, v = line.split(None, 1)
                kv[k] = [int(x) for x in v.split()]
    return kv, stages


def test_hand_traced_interior_block(golden_dir):
    """Block 1 of a K=3 stream, every metric and survivor bit traced by hand:
    zero initial metrics at f0 = 2, Eq. (1) over [2, 9], traceback from S_0 at
    f1 = 9.  The fixture also records what a known start or an argmin
    traceback would give; both differ from the block's result."""
    kv, stages = _golden(golden_dir, "k3_75_interior_block.txt")
    rx = np.array(kv["rx"], dtype=np.int16)
    llr = (127 - 254 * rx).astype(np.int8).reshape(-1, 2)
    assert llr.shape[0] == 12
    b, D, L = kv["block"]
    f0, f1 = kv["window"]
    assert _geometry(12, D, L, b)[:2] == (f0, f1)
    # the stage-by-stage recursion from zero metrics
    pm = np.zeros(4, dtype=np.int64)
    for s, want_pm, want_dec in stages:
        pm, dec = oracle.acs_stage(3, K3, llr[s], pm)
        assert pm.tolist() == want_pm, s
        assert dec.tolist() == want_dec, s
    # the block form end to end
    bits, pm_end = oracle.viterbi_block_metrics(3, K3, llr, D, L, (b, b + 1))
    assert pm_end[0] == kv["pm_end"][0]
    assert bits[b * D:(b + 1) * D].tolist() == kv["decoded"]
    # the readings the block must not follow
    pm = np.array([0, oracle.BIG, oracle.BIG, oracle.BIG], dtype=np.int64)
    for s in range(f0, f1 + 1):
        pm, _ = oracle.acs_stage(3, K3, llr[s], pm)
    assert pm[0] == kv["known_start_pm_end"][0] != kv["pm_end"][0]
    assert kv["argmin_decoded"] != kv["decoded"]
