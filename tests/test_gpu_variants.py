"""The decoding variants on the GPU, bit for bit against their oracle forms:
the argmin traceback start (the classic VA's start state S_E, Sec. II) and
tail-biting frames (circular block windows), alone and together, over every
kernel configuration that honours them."""
import numpy as np
import pytest

import oracle
from paper_1608_00066_gb300 import pbvd, synth

from gpu_util import T_VALUES, gpu_bits, make_decoder, mother_llr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(1, 8, 0), (5, 8, 42), (300, 16, 35), (2000, 512, 42), (2999, 256, 64), (4093, 64, 0),
          (3000, 24, 100), (20000, 512, 42)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1608_00066_gb300 import build
    build.build()
    pbvd.load()


def _variant_Ts(name):
    # the one-warp latency kernel of the 64-state codes (T = 32) decodes the
    # plain scheme only
    Ts = T_VALUES[name]
    return [T for T in Ts if not (T == 32 and name.startswith("K7"))]


@pytest.mark.parametrize("name", ["K7_r1/2", "K7_r3/4", "K9_r1/3", "K3_r1/2"])
def test_argmin_start(name):
    spec = synth.CODES[name]
    rng = np.random.default_rng(len(name) + 5)
    for (k, D, L) in SHAPES:
        f = synth.make_frame(spec, k, float(rng.uniform(-1, 4)), seed=int(rng.integers(1 << 30)))
        want, _ = oracle.viterbi_block_variant(spec.K, spec.gens, mother_llr(spec, f.llr, f.n_stages), D, L,
                                               argmin=True)
        dec = make_decoder(spec, D, L)
        dec.set_mode(argmin=True)
        for T in _variant_Ts(name):
            for smem in (0, 1):
                got = gpu_bits(dec, f.llr, f.n_stages, threads_per_pair=T, survivors_in_smem=smem)
                bad = np.flatnonzero(got != want)
                assert bad.size == 0, (name, k, D, L, T, smem, bad[:10])
        got = gpu_bits(dec, f.llr, f.n_stages, threads_per_pair=0, cta_threads=0, survivors_in_smem=-1)
        assert np.array_equal(got, want), (name, k, D, L, "auto")
        dec.close()


def test_argmin_differs_from_s0_on_unterminated_streams():
    """A stream cut off without its tail: the argmin start recovers the last
    bits that the S_0 start gets wrong, and both equal their oracle forms."""
    spec = synth.K7_R12
    f = synth.make_frame(spec, 5000, 6.0, seed=3)
    n = 4000                      # cut inside the message, no tail
    llr = f.llr[:2 * n]
    dec = make_decoder(spec, 512, 42)
    s0 = gpu_bits(dec, llr, n)
    dec.set_mode(argmin=True)
    am = gpu_bits(dec, llr, n)
    want_am, _ = oracle.viterbi_block_variant(7, spec.gens, llr.reshape(-1, 2), 512, 42, argmin=True)
    assert np.array_equal(am, want_am)
    assert np.array_equal(s0, oracle.viterbi_block(7, spec.gens, llr.reshape(-1, 2), 512, 42))
    assert (am[-6:] != f.msg[n - 6:n]).sum() < (s0[-6:] != f.msg[n - 6:n]).sum() or \
        np.array_equal(am[-6:], f.msg[n - 6:n])
    dec.close()


@pytest.mark.parametrize("name", ["K7_r1/2", "K9_r1/3", "K3_r1/2"])
@pytest.mark.parametrize("argmin", [False, True])
def test_tailbiting(name, argmin):
    spec = synth.CODES[name]
    rng = np.random.default_rng(len(name) + 17 + argmin)
    for (k, D, L) in [(40, 8, 42), (700, 64, 35), (3000, 512, 42), (3001, 256, 64), (100, 512, 200),
                      (20000, 512, 42), (10, 8, 3)]:
        if k < spec.v:
            continue
        f = synth.make_tailbiting_frame(spec, k, float(rng.uniform(0, 4)), seed=int(rng.integers(1 << 30)))
        want, _ = oracle.viterbi_block_variant(spec.K, spec.gens, f.llr.reshape(-1, spec.R), D, L,
                                               argmin=argmin, circular=True)
        dec = make_decoder(spec, D, L)
        dec.set_mode(argmin=argmin, tailbiting=True)
        for T in _variant_Ts(name):
            for smem in (0, 1):
                got = gpu_bits(dec, f.llr, f.n_stages, threads_per_pair=T, survivors_in_smem=smem)
                bad = np.flatnonzero(got != want)
                assert bad.size == 0, (name, argmin, k, D, L, T, smem, bad[:10])
        got = gpu_bits(dec, f.llr, f.n_stages, threads_per_pair=0, cta_threads=0, survivors_in_smem=-1)
        assert np.array_equal(got, want), (name, argmin, k, D, L, "auto")
        dec.close()


def test_tailbiting_noiseless_and_runtime_code():
    for spec in (synth.K7_R12, synth.CodeSpec("K6_53_75", 6, (0o53, 0o75))):
        f = synth.make_tailbiting_frame(spec, 5000, None, seed=1)
        dec = make_decoder(spec, 256, 6 * spec.K)
        dec.set_mode(tailbiting=True)
        assert np.array_equal(gpu_bits(dec, f.llr, f.n_stages), f.msg)
        dec.close()


def test_mode_rejections():
    spec = synth.K7_R34
    dec = make_decoder(spec, 512, 42)
    with pytest.raises(pbvd.PbvdError) as ei:
        dec.set_mode(tailbiting=True)
    assert ei.value.code == pbvd.PBVD_EUNSUPPORTED
    with pytest.raises(pbvd.PbvdError) as ei:
        pbvd.pbvd_set_mode(dec.ctx, 4)
    assert ei.value.code == pbvd.PBVD_EINVAL
    dec.set_mode(argmin=True)
    assert pbvd.pbvd_get_mode(dec.ctx) == pbvd.PBVD_MODE_ARGMIN
    f = synth.make_frame(spec, 1000, 2.0, seed=5)
    d = torch.from_numpy(f.llr).cuda()
    o = torch.zeros((f.n_stages + 7) // 8, dtype=torch.uint8, device="cuda")
    with pytest.raises(pbvd.PbvdError) as ei:
        pbvd.pbvd_decode_batch([(dec.ctx, d.data_ptr(), f.n_stages, o.data_ptr())])
    assert ei.value.code == pbvd.PBVD_EUNSUPPORTED
    dec.close()
