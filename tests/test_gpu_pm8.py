"""8-bit path metrics (pbvd_decode_packed_pm8: four blocks per register) on
q-bit packed soft values: bit for bit against the q-bit block oracle (mu =
+-Q) and against the 16-bit path on the same words, over codes, q, block
geometries (L = 0, L > D so that several blocks start at stage 0, ragged
ends), uniformly random words (every q-bit code, the clamped -Q-1 included),
and the calls it refuses."""
import numpy as np
import pytest

import oracle
from paper_1608_00066_gb300 import pbvd, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K7_R13 = synth.CodeSpec("K7_r1/3", 7, (0o171, 0o165, 0o133))
K5_R12 = synth.CodeSpec("K5_r1/2", 5, (0o23, 0o35))
CODES = {"K7_r1/2": synth.K7_R12, "K7_r1/3": K7_R13, "K5_r1/2": K5_R12}
GEOMETRY = [(512, 42), (64, 100), (8, 0), (1024, 15), (16, 3)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1608_00066_gb300 import build
    build.build()
    pbvd.load()


def _words(f):
    return torch.from_numpy(f.words.view(np.int32).copy()).cuda()


def _want(spec, q, words, n, D, L):
    vals = oracle.unpack_soft(q, words, n * spec.R)
    return oracle.viterbi_block_q(spec.K, spec.gens, vals.reshape(n, spec.R), D, L, oracle.q_max(q))


def _bits(out, n):
    return np.unpackbits(out.cpu().numpy(), bitorder="little")[:n]


def _lanes(spec):
    """Threads per four blocks built for the code (two only for 64 states)."""
    return (1, 2) if spec.K == 7 else (1,)


@pytest.mark.parametrize("q", [1, 2, 3])
@pytest.mark.parametrize("name", list(CODES))
def test_pm8_matches_oracle(name, q):
    spec = CODES[name]
    for D, L in GEOMETRY:
        dec = pbvd.Decoder(spec.K, spec.gens, None, D, L)
        for k, eb in ((5000, 1.0), (777, 0.0), (1, 2.0)):
            f = synth.make_packed_frame(spec, k, eb, q, seed=k * 7 + q + D)
            want = _want(spec, q, f.words, f.n_stages, D, L)
            for lanes in _lanes(spec):
                dec.set_config(threads_per_pair=lanes)
                out = dec.decode_packed_pm8(_words(f), q, f.n_stages)
                torch.cuda.synchronize()
                got = _bits(out, f.n_stages)
                bad = np.flatnonzero(got != want)
                assert bad.size == 0, (name, q, D, L, k, lanes, bad[:8])
        dec.close()


@pytest.mark.parametrize("q", [1, 2, 3])
def test_pm8_random_words(q):
    """Words of uniformly random bits: every q-bit code equally likely (for
    q >= 2 the value -Q-1 too, read as -Q), metrics as spread as noise makes
    them; several ragged lengths, one and two threads per four blocks."""
    spec = synth.K7_R12
    rng = np.random.default_rng(100 + q)
    dec = pbvd.Decoder(spec.K, spec.gens, None, 256, 42)
    m = 32 // q
    for n in (9, 300, 4099, 70001):
        words = rng.integers(0, 1 << 32, size=(n * 2 + m - 1) // m, dtype=np.uint64).astype(np.uint32)
        want = _want(spec, q, words, n, 256, 42)
        for lanes in (1, 2):
            dec.set_config(threads_per_pair=lanes)
            out = dec.decode_packed_pm8(torch.from_numpy(words.view(np.int32)).cuda(), q, n)
            torch.cuda.synchronize()
            assert np.array_equal(_bits(out, n), want), (q, n, lanes)
    dec.close()


@pytest.mark.parametrize("q", [1, 3])
def test_pm8_equals_16bit_path_full_stream(q):
    """The 2^24-bit K=7 stream at D=512, L=42: identical to the 16-bit path's
    bits on the same words, and to the oracle on every block of the first 2^18
    stages (blocks of a prefix that end inside it decode as in the stream)."""
    spec = synth.K7_R12
    f = synth.make_packed_frame(spec, 1 << 24, 3.0, q, seed=2003 + q)
    n = f.n_stages
    dec = pbvd.Decoder(spec.K, spec.gens, None, 512, 42)
    w = _words(f)
    ref = _bits(dec.decode_packed(w, q, n), n)
    dec.set_config(threads_per_pair=1)
    one = _bits(dec.decode_packed_pm8(w, q, n), n)
    dec.set_config(threads_per_pair=0)
    got = _bits(dec.decode_packed_pm8(w, q, n), n)
    torch.cuda.synchronize()
    assert np.array_equal(got, ref)
    assert np.array_equal(one, ref)
    pre = 1 << 18
    want = oracle.viterbi_block_q(7, spec.gens, oracle.unpack_soft(q, f.words, pre * 2).reshape(pre, 2), 512, 42,
                                  oracle.q_max(q))
    full_blocks = (pre - 42) // 512  # blocks whose range [f0, f1] ends inside the prefix
    assert np.array_equal(got[:full_blocks * 512], want[:full_blocks * 512])
    assert int((got[:1 << 24] != f.msg).sum()) < (1 << 24) * 5e-2
    dec.close()


def test_pm8_refuses():
    spec = synth.K7_R12
    w = torch.zeros(4096, dtype=torch.int32, device="cuda")
    o = torch.zeros(4096, dtype=torch.uint8, device="cuda")

    def code(ctx, q, n=1000):
        try:
            pbvd.pbvd_decode_packed_pm8(ctx, w.data_ptr(), q, n, o.data_ptr(), 0)
        except pbvd.PbvdError as e:
            return e.code
        return pbvd.PBVD_OK

    dec = pbvd.Decoder(spec.K, spec.gens, None, 512, 42)
    for q in (4, 5, 8):  # 7 * 2QR >= 127
        assert code(dec.ctx, q) == pbvd.PBVD_EUNSUPPORTED
    for q in (0, 9):
        assert code(dec.ctx, q) == pbvd.PBVD_EINVAL
    assert code(dec.ctx, 3, n=0) == pbvd.PBVD_EINVAL
    dec.set_mode(argmin=True)
    assert code(dec.ctx, 3) == pbvd.PBVD_EUNSUPPORTED
    dec.close()
    for sp in (synth.K7_R34, synth.K9_R13):
        d = pbvd.Decoder(sp.K, sp.gens, sp.puncture, 512, 42)
        assert code(d.ctx, 1) == pbvd.PBVD_EUNSUPPORTED
        d.close()
    torch.cuda.synchronize()
