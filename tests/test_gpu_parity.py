"""Parity of the CUDA decoder with the block-based CPU oracle: bit-exact on
every decoded bit (the method is integer arithmetic with a fixed tie rule).

Small cases compare every bit and span many blocks, a ragged last block and
the degenerate shapes (one stage, D < L, L = 0, a frame shorter than D); the
full-size cases (2^24 information bits) compare sampled blocks in the launch
configuration the benchmark uses."""
import numpy as np
import pytest

import oracle
from paper_1608_00066_gb300 import pbvd, synth

from gpu_util import T_VALUES, gpu_bits, make_decoder, mother_llr, oracle_bits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1608_00066_gb300 import build
    build.build()
    pbvd.load()


def test_worked_example_k3():
    """The hand-traced (7,5) example: received 11 11 00 01 01 11 decodes to
    1 0 1 1 0 0."""
    rx = np.array([1, 1, 1, 1, 0, 0, 0, 1, 0, 1, 1, 1], np.uint8)
    llr = (127 - 254 * rx.astype(np.int16)).astype(np.int8)
    for T in (1, 2):
        for smem in (0, 1):
            dec = make_decoder(synth.K3_R12, 8, 4)
            bits = gpu_bits(dec, llr, 6, threads_per_pair=T, survivors_in_smem=smem)
            assert bits.tolist() == [1, 0, 1, 1, 0, 0]


def test_latency_frame_all_configs():
    """K=7 r1/2, one frame of 4096 information bits at 3 dB, D=512, L=42."""
    spec = synth.K7_R12
    f = synth.make_frame(spec, 4096, 3.0, seed=1001)
    want = oracle_bits(spec, f.llr, f.n_stages, 512, 42)
    assert (want[:4096] != f.msg).sum() < 20
    dec = make_decoder(spec, 512, 42)
    for T in T_VALUES[spec.name]:
        for smem in (0, 1):
            got = gpu_bits(dec, f.llr, f.n_stages, threads_per_pair=T, survivors_in_smem=smem)
            assert np.array_equal(got, want), (T, smem)
    got = gpu_bits(dec, f.llr, f.n_stages, threads_per_pair=0, survivors_in_smem=-1)
    assert np.array_equal(got, want)


SHAPES = [
    # (k information bits, D, L)
    (1, 8, 0), (1, 8, 5), (5, 8, 42), (100, 8, 20), (300, 16, 35),
    (1000, 64, 3), (2000, 512, 42), (2999, 256, 64), (777, 1024, 42),
    (3000, 24, 100), (4093, 512, 0),
]


@pytest.mark.parametrize("name", ["K7_r1/2", "K7_r3/4", "K9_r1/3", "K3_r1/2"])
def test_random_shapes_all_configs(name):
    spec = synth.CODES[name]
    rng = np.random.default_rng(hash(name) % 1000)
    for (k, D, L) in SHAPES:
        f = synth.make_frame(spec, k, float(rng.uniform(-1, 4)), seed=int(rng.integers(1 << 30)))
        want = oracle_bits(spec, f.llr, f.n_stages, D, L)
        dec = make_decoder(spec, D, L)
        for T in T_VALUES[name]:
            for smem in (0, 1):
                got = gpu_bits(dec, f.llr, f.n_stages, threads_per_pair=T, survivors_in_smem=smem)
                bad = np.flatnonzero(got != want)
                assert bad.size == 0, (name, k, D, L, T, smem, bad[:10])
        dec.close()


def test_cta_shapes():
    """Several groups per CTA and partial CTAs give the same bits."""
    spec = synth.K7_R12
    f = synth.make_frame(spec, 20000, 2.0, seed=5)
    want = oracle_bits(spec, f.llr, f.n_stages, 256, 42)
    dec = make_decoder(spec, 256, 42)
    for T, cta in ((1, 32), (1, 64), (1, 128), (2, 128), (4, 96), (8, 256), (32, 64)):
        got = gpu_bits(dec, f.llr, f.n_stages, threads_per_pair=T, cta_threads=cta, survivors_in_smem=0)
        assert np.array_equal(got, want), (T, cta)


def test_extreme_soft_values_and_ties():
    """-128 reads as -127; all-zero soft values make every comparison a tie and
    decode to all zeros; saturated noise-free values decode the message."""
    spec = synth.K7_R12
    rng = np.random.default_rng(8)
    n = 3000
    llr = rng.choice(np.array([-128, -127, 127, 0, 1, -1], np.int8), size=n * 2)
    dec = make_decoder(spec, 64, 20)
    want = oracle_bits(spec, llr, n, 64, 20)
    for T in (1, 4, 32):
        assert np.array_equal(gpu_bits(dec, llr, n, threads_per_pair=T), want)
    zeros = np.zeros(n * 2, np.int8)
    for T in (1, 2, 8):
        assert not gpu_bits(dec, zeros, n, threads_per_pair=T).any()
    f = synth.make_frame(spec, 5000, None, seed=3)
    assert np.array_equal(gpu_bits(dec, f.llr, f.n_stages)[:5000], f.msg)


def test_zero_stages_rejected():
    dec = make_decoder(synth.K7_R12, 512, 42)
    d = torch.zeros(16, dtype=torch.int8, device="cuda")
    o = torch.zeros(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(pbvd.PbvdError):
        pbvd.pbvd_decode(dec.ctx, d.data_ptr(), 0, o.data_ptr(), 0)


def test_output_bytes_outside_range_untouched():
    """The decoder writes exactly ceil(n/8) bytes."""
    spec = synth.K7_R12
    f = synth.make_frame(spec, 1000, 2.0, seed=12)
    n = f.n_stages
    dec = make_decoder(spec, 64, 42)
    d = torch.from_numpy(f.llr).cuda()
    out = torch.full(((n + 7) // 8 + 64,), 0xA5, dtype=torch.uint8, device="cuda")
    dec.decode(d, n, out=out)
    torch.cuda.synchronize()
    tail = out[(n + 7) // 8:].cpu().numpy()
    assert (tail == 0xA5).all()


def _sampled_blocks(n, D, rng, count=24):
    nb = (n + D - 1) // D
    picks = set([0, 1, nb - 2, nb - 1])
    picks.update(int(x) for x in rng.integers(0, nb, size=count))
    return sorted(b for b in picks if 0 <= b < nb)


@pytest.mark.parametrize("name,ebn0,D,L,seed", [
    ("K7_r1/2", 3.0, 512, 42, 2003),
    ("K9_r1/3", 2.0, 1024, 64, 3001),
])
def test_full_size_stream_sampled(name, ebn0, D, L, seed):
    """2^24 information bits, the launch configuration of the benchmark; the
    oracle decodes a sample of blocks one by one."""
    spec = synth.CODES[name]
    k = 1 << 24
    f = synth.make_frame(spec, k, ebn0, seed=seed)
    n = f.n_stages
    dec = make_decoder(spec, D, L)
    got = gpu_bits(dec, f.llr, n)
    rng = np.random.default_rng(seed)
    mother = mother_llr(spec, f.llr, n)
    for b in _sampled_blocks(n, D, rng):
        want = oracle.viterbi_block(spec.K, spec.gens, mother, D, L, blocks=(b, b + 1))
        o0, o1 = b * D, min((b + 1) * D, n)
        assert np.array_equal(got[o0:o1], want[o0:o1]), b
    ber = float((got[:k] != f.msg).mean())
    assert ber < 1e-3, ber


def test_unaligned_soft_values():
    """Soft values starting at an odd address (no 2-byte loads) decode the
    same bits."""
    spec = synth.K7_R12
    f = synth.make_frame(spec, 30000, 1.5, seed=14)
    n = f.n_stages
    want = oracle_bits(spec, f.llr, n, 256, 42)
    dec = make_decoder(spec, 256, 42)
    big = torch.zeros(len(f.llr) + 1, dtype=torch.int8, device="cuda")
    big[1:] = torch.from_numpy(f.llr).cuda()
    view = big[1:]
    assert view.data_ptr() % 2 == 1
    for T in (1, 2, 4):
        dec.set_config(threads_per_pair=T)
        out = dec.decode(view, n)
        torch.cuda.synchronize()
        assert np.array_equal(np.unpackbits(out.cpu().numpy(), bitorder="little")[:n], want), T
