"""Pins for the CPU oracle: each test checks it against something other than
itself -- the paper's Table 2, closed forms, a hand-traced example, the
maximum-likelihood definition by exhaustive search, and special cases in
which the block form must reduce to the full-frame Viterbi algorithm."""
import os

import numpy as np
import pytest

import oracle
from paper_1608_00066_gb300 import synth

K7 = (0o171, 0o133)
K9 = (0o557, 0o663, 0o711)
K3 = (0o7, 0o5)
# (13,16) has g_{K-1} != g_0 in its second generator, so it separates the
# input tap from the oldest-memory tap (all standard codes have both set).
CODES = [(3, K3), (7, K7), (9, K9), (5, (0o23, 0o35)), (7, (0o171, 0o165, 0o133)),
         (4, (0o13, 0o16))]


def _read(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as f:
        return [l.strip() for l in f if l.strip() and not l.startswith("#")]


# ----------------------------------------------------------------- Table 2

def test_table2_state_classification(golden_dir):
    """Table 2: butterflies of the (171,133) code grouped by alpha, with the
    beta/gamma/theta of each group.  Pins the encoder's bit conventions."""
    rows = _read(golden_dir, "table2_k7_171_133.txt")
    K = 7
    seen = set()
    for row in rows:
        head, states = row.split(":")
        _, a, b, g, t = head.split()
        states = [int(s) for s in states.split()]
        want = tuple(int(x, 2) for x in (a, b, g, t))
        assert len(states) == 16
        for s in states:
            j = s // 2
            got = (oracle.codeword(K, K7, 2 * j, 0), oracle.codeword(K, K7, 2 * j, 1),
                   oracle.codeword(K, K7, 2 * j + 1, 0), oracle.codeword(K, K7, 2 * j + 1, 1))
            assert got == want, (s, got, want)
            seen.add(s)
    assert seen == set(range(64))


@pytest.mark.parametrize("K,gens", CODES)
def test_butterfly_identities_eq3_to_eq6(K, gens):
    """Eqs. (3)-(6): beta = alpha^g_{K-1}, gamma = alpha^g_0,
    theta = alpha^g_{K-1}^g_0, for every butterfly."""
    R = len(gens)
    gK = sum(((g >> (K - 1)) & 1) << (R - 1 - r) for r, g in enumerate(gens))
    g0 = sum((g & 1) << (R - 1 - r) for r, g in enumerate(gens))
    for j in range(1 << (K - 2)):
        a = oracle.codeword(K, gens, 2 * j, 0)
        assert oracle.codeword(K, gens, 2 * j, 1) == a ^ gK
        assert oracle.codeword(K, gens, 2 * j + 1, 0) == a ^ g0
        assert oracle.codeword(K, gens, 2 * j + 1, 1) == a ^ gK ^ g0


@pytest.mark.parametrize("K", [3, 5, 7, 9])
def test_butterfly_transitions(K):
    """Sec. III-B: S_{2j}, S_{2j+1} go to S_j (x=0) and S_{j+2^{v-1}} (x=1)."""
    half = 1 << (K - 2)
    for j in range(half):
        for i in (2 * j, 2 * j + 1):
            assert oracle.next_state(K, i, 0) == j
            assert oracle.next_state(K, i, 1) == j + half


# ----------------------------------------------------------------- encoder

@pytest.mark.parametrize("K,gens", CODES)
def test_encoder_is_polynomial_product(K, gens):
    """The shift register of Eq. (2) equals c(D) = m(D) g(D) over GF(2)."""
    spec = synth.CodeSpec("t", K, tuple(gens))
    rng = np.random.default_rng(7)
    for k in (1, 5, 33, 200):
        msg = rng.integers(0, 2, size=k, dtype=np.uint8)
        assert np.array_equal(oracle.encode(K, gens, msg), synth.conv_encode(spec, msg))


def test_encoder_textbook_codeword(golden_dir):
    """(7,5) code, message 1011 + tail -> 11 10 00 01 01 11."""
    rows = dict(r.split(None, 1) for r in _read(golden_dir, "k3_75_worked_example.txt")
                if r.split()[0] in ("msg", "code"))
    msg = [int(x) for x in rows["msg"].split()][:4]
    code = [int(x) for x in rows["code"].split()]
    assert oracle.encode(3, K3, msg).reshape(-1).tolist() == code


# ---------------------------------------------------------------- metrics

def test_branch_metric_closed_forms():
    """Hard +-127 inputs: 254 x Hamming distance; erasures: 127 R;
    -128 reads as -127; general form 127R - sum(l) + 2 sum_{c_r=1} l_r."""
    rng = np.random.default_rng(3)
    for R in (1, 2, 3):
        for c in range(1 << R):
            for rx in range(1 << R):
                lam = [127 - 254 * ((rx >> (R - 1 - r)) & 1) for r in range(R)]
                assert oracle.branch_metric(lam, c) == 254 * bin(c ^ rx).count("1")
            assert oracle.branch_metric([0] * R, c) == 127 * R
            lam = rng.integers(-127, 128, size=R)
            want = 127 * R - int(lam.sum()) + 2 * sum(int(lam[r]) for r in range(R)
                                                       if (c >> (R - 1 - r)) & 1)
            assert oracle.branch_metric(lam, c) == want
            assert oracle.branch_metric([-128] * R, c) == oracle.branch_metric([-127] * R, c)


# ------------------------------------------------------- worked example

def test_hand_traced_k3_example(golden_dir):
    rows = _read(golden_dir, "k3_75_worked_example.txt")
    kv = {}
    stages = []
    for r in rows:
        if r.startswith("stage"):
            parts = r.split(":")
            stages.append(([int(x) for x in parts[1].split()], [int(x) for x in parts[2].split()]))
        else:
            k, v = r.split(None, 1)
            kv[k] = [int(x) for x in v.split()]
    rx = np.array(kv["rx"], dtype=np.uint8)
    llr = (127 - 254 * rx.astype(np.int16)).astype(np.int8).reshape(-1, 2)
    bits, fpm, dec, trace = oracle.viterbi_full(3, K3, llr, want_trace=True)
    for s, (pm, d) in enumerate(stages):
        assert trace[s].tolist() == pm, s
        assert dec[s].tolist() == d, s
    assert bits.tolist() == kv["decoded"]
    assert fpm[0] == 254


# ------------------------------------------------------------ brute force

@pytest.mark.parametrize("K,gens", [(3, K3), (7, K7), (5, (0o23, 0o35)), (9, K9)])
def test_full_frame_is_maximum_likelihood(K, gens):
    """Sec. II: the VA finds the minimum-metric terminated path.  Exhaustive
    search over all 2^k messages gives the same metric always, and the same
    message whenever the minimum is unique."""
    rng = np.random.default_rng(11 + K)
    spec = synth.CodeSpec("t", K, tuple(gens))
    unique = 0
    for trial in range(6):
        k = int(rng.integers(1, 13 if K < 9 else 9))
        f = synth.make_frame(spec, k, ebn0_db=float(rng.uniform(-2, 3)), seed=int(rng.integers(1 << 30)))
        llr = f.llr.reshape(-1, spec.R)
        bits, fpm = oracle.viterbi_full(K, gens, llr)
        best_msg, best_metric, n_best = oracle.brute_force(K, gens, llr, k)
        assert fpm[0] == best_metric
        if n_best == 1:
            unique += 1
            assert bits[:k].tolist() == best_msg.tolist()
        assert bits[k:].tolist() == [0] * (K - 1)
    assert unique > 0


def test_brute_force_noiseless():
    msg = np.array([1, 0, 0, 1, 1, 1, 0, 1, 0, 0, 1], dtype=np.uint8)
    llr = synth.noiseless_int8(oracle.encode(7, K7, msg))
    best, metric, nb = oracle.brute_force(7, K7, llr, len(msg))
    assert metric == 0 and nb == 1 and best.tolist() == msg.tolist()


def test_ties_keep_upper_branch():
    """All-zero soft values make every pair of candidates equal once the
    known-start offsets are gone: every survivor bit is 0 from stage v on, all
    metrics are equal, and the path traced from S_0 is all zeros."""
    for K, gens in ((3, K3), (7, K7), (9, K9)):
        R = len(gens)
        n = 40
        bits, fpm, dec, trace = oracle.viterbi_full(K, gens, np.zeros((n, R), np.int8), True)
        assert not dec[K - 1:].any()
        assert (trace[K - 1:] == trace[K - 1:, :1]).all()
        assert trace[-1, 0] == 127 * R * n
        assert not bits.any()


# -------------------------------------------------------------- round trips

@pytest.mark.parametrize("name", ["K3_r1/2", "K7_r1/2", "K9_r1/3", "K7_r3/4"])
def test_noiseless_round_trip(name):
    spec = synth.CODES[name]
    f = synth.make_frame(spec, 3000, None, seed=5)
    llr = _mother(spec, f)
    bits, fpm = oracle.viterbi_full(spec.K, spec.gens, llr)
    assert bits[:3000].tolist() == f.msg.tolist()
    # error-free: only erased (punctured) positions cost anything, 127 each
    assert fpm[0] == 127 * _erasure_count(spec, f)
    L = 6 * spec.K
    for D in (8, 64, 512):
        out = oracle.viterbi_block(spec.K, spec.gens, llr, D, L)
        assert out[:3000].tolist() == f.msg.tolist(), D
    out = oracle.viterbi_window(spec.K, spec.gens, llr, 64, L)
    assert out[:3000].tolist() == f.msg.tolist()


def _erasure_count(spec, f):
    return f.n_stages * spec.R - len(f.llr)


def _mother(spec, f):
    if spec.puncture is None:
        return f.llr.reshape(-1, spec.R)
    return oracle.depuncture(spec.pattern_array(), f.llr, f.n_stages)


# --------------------------------------------------------- block geometry

def test_block_geometry_clamps():
    """Sec. III-A: block b decodes [bD, (b+1)D) from a forward range that
    starts L stages earlier and ends L stages later, clamped to the stream."""
    n, D, L = 4102, 512, 42
    nb = (n + D - 1) // D
    assert nb == 9
    assert oracle.block_geometry(n, D, L, 0) == (0, 553, 0, 512)
    assert oracle.block_geometry(n, D, L, 1) == (470, 1065, 512, 1024)
    assert oracle.block_geometry(n, D, L, 6) == (3030, 3625, 3072, 3584)
    assert oracle.block_geometry(n, D, L, 7) == (3542, 4101, 3584, 4096)
    assert oracle.block_geometry(n, D, L, 8) == (4054, 4101, 4096, 4102)
    # D < L: the truncation range of early blocks reaches back to stage 0
    assert oracle.block_geometry(100, 8, 20, 2) == (0, 43, 16, 24)


@pytest.mark.parametrize("K,gens", [(3, K3), (7, K7), (9, K9)])
def test_block_reduces_to_full_frame(K, gens):
    """With D >= n there is one block covering the frame; with L >= n every
    block covers the frame.  Either way each output equals the full-frame VA."""
    spec = synth.CodeSpec("t", K, tuple(gens))
    f = synth.make_frame(spec, 700, 0.5, seed=21)
    llr = f.llr.reshape(-1, spec.R)
    full, _ = oracle.viterbi_full(K, gens, llr)
    assert np.array_equal(oracle.viterbi_block(K, gens, llr, 1024, 13), full)
    for D in (8, 96, 512):
        assert np.array_equal(oracle.viterbi_block(K, gens, llr, D, f.n_stages), full)
    assert np.array_equal(oracle.viterbi_window(K, gens, llr, 1024, 5), full)
    assert np.array_equal(oracle.viterbi_window(K, gens, llr, 64, f.n_stages), full)


def test_known_start_of_first_block():
    """The first block starts from the known encoder state S_0.  Soft values of
    a codeword that starts in another state make that visible: a decoder that
    ignored the known start would follow the other state's path."""
    spec = synth.K7_R12
    rng = np.random.default_rng(17)
    prefix = np.array([1, 0, 1, 1, 0, 1], dtype=np.uint8)  # leaves the encoder in state 45
    msg = rng.integers(0, 2, size=200, dtype=np.uint8)
    coded = synth.conv_encode(spec, np.concatenate([prefix, msg]))[6:]
    llr = synth.noiseless_int8(coded.reshape(-1)).reshape(-1, 2)
    full, fpm = oracle.viterbi_full(7, K7, llr)
    assert fpm[0] > 0  # the known start cannot reach the sent path for free
    blk = oracle.viterbi_block(7, K7, llr, 512, 42)
    assert np.array_equal(blk, full)
    assert not np.array_equal(blk[:200], msg)


def test_window_segments_equal_prefix_viterbi():
    """Carried-metric form: segment m = [mD, (m+1)D) is decided by traceback
    from S_0 at stage (m+1)D + L - 1, so it equals the full-frame VA run on the
    stream prefix that ends at that stage."""
    spec = synth.K7_R12
    f = synth.make_frame(spec, 900, -1.0, seed=33)
    llr = f.llr.reshape(-1, 2)
    n = f.n_stages
    for D, L in ((64, 3), (32, 7), (100, 0)):
        win = oracle.viterbi_window(7, K7, llr, D, L)
        m = 0
        while (m + 1) * D + L <= n - 1:
            e = (m + 1) * D + L
            pre, _ = oracle.viterbi_full(7, K7, llr[:e])
            assert np.array_equal(win[m * D:(m + 1) * D], pre[m * D:(m + 1) * D]), (D, L, m)
            m += 1
        full, _ = oracle.viterbi_full(7, K7, llr)
        assert np.array_equal(win[m * D:], full[m * D:])


def test_block_reads_only_its_window():
    """A block's bits depend only on the soft values in [f0, f1]."""
    spec = synth.K7_R12
    f = synth.make_frame(spec, 3000, 1.0, seed=9)
    llr = f.llr.reshape(-1, 2).copy()
    n, D, L = f.n_stages, 256, 35
    base = oracle.viterbi_block(7, K7, llr, D, L)
    rng = np.random.default_rng(1)
    for b in (0, 3, (n + D - 1) // D - 1):
        f0, f1, o0, o1 = oracle.block_geometry(n, D, L, b)
        pert = llr.copy()
        mask = np.ones(n, bool)
        mask[f0:f1 + 1] = False
        pert[mask] = rng.integers(-127, 128, size=(mask.sum(), 2))
        out = oracle.viterbi_block(7, K7, pert, D, L, blocks=(b, b + 1))
        assert np.array_equal(out[o0:o1], base[o0:o1])


def test_block_truncation_loss_is_small():
    """At moderate SNR the block form with L ~ 6K agrees with the full-frame
    VA on almost every bit (the block form is an approximation, Sec. III-A)."""
    spec = synth.K7_R12
    f = synth.make_frame(spec, 20000, 3.0, seed=1001)
    llr = f.llr.reshape(-1, 2)
    full, _ = oracle.viterbi_full(7, K7, llr)
    blk = oracle.viterbi_block(7, K7, llr, 512, 42)
    assert (full != blk).mean() < 1e-3
    assert (full[:20000] != f.msg).mean() < 5e-3


# --------------------------------------------------------------- puncture

def test_puncture_example(golden_dir):
    rows = dict(r.split(None, 1) for r in _read(golden_dir, "puncture_r34_example.txt"))
    pat = np.array([[int(x) for x in row.split()] for row in rows["pattern"].split("/")], np.uint8)
    bits = np.array([[int(x) for x in p.split()] for p in rows["bits"].split("/")], np.uint8)
    sent = [int(x) for x in rows["sent"].split()]
    assert oracle.puncture(pat, bits).tolist() == sent
    spec = synth.K7_R34
    assert synth.puncture_bits(spec, bits).tolist() == sent
    soft = (127 - 254 * np.array(sent)).astype(np.int8)
    full = oracle.depuncture(pat, soft, bits.shape[0])
    want = np.where(np.tile(pat.T, (2, 1)).astype(bool), 127 - 254 * bits.astype(int), 0)
    assert full.tolist() == want.tolist()


def test_puncture_matches_transmitter():
    spec = synth.K7_R34
    rng = np.random.default_rng(2)
    bits = rng.integers(0, 2, size=(1001, 2), dtype=np.uint8)
    assert np.array_equal(oracle.puncture(spec.pattern_array(), bits),
                          synth.puncture_bits(spec, bits))
    assert spec.sent_per_stage_prefix(1001) == len(synth.puncture_bits(spec, bits))


# ----------------------------------------------------------------- bounds

@pytest.mark.parametrize("K,gens", [(7, K7), (9, K9)])
def test_metric_spread_bound(K, gens):
    """The spread of the path metrics never exceeds BIG + v * 254 R, the bound
    that lets 16-bit renormalised metrics stay exact."""
    spec = synth.CodeSpec("t", K, tuple(gens))
    f = synth.make_frame(spec, 3000, -1.0, seed=4)
    _, _, _, trace = oracle.viterbi_full(K, gens, f.llr.reshape(-1, spec.R), True)
    spread = trace.max(axis=1) - trace.min(axis=1)
    assert spread.max() <= oracle.BIG + (K - 1) * 254 * spec.R
    assert spread[K - 1:].max() <= (K - 1) * 254 * spec.R
