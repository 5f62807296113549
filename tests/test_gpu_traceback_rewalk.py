"""Parity where the traceback's guessed segments fail all the time: soft
values of pure noise (uniform int8, no transmitted codeword) and weak
signals, long blocks, every thread count built for the code (up to 32
segments per block), shared-memory and global survivors.  There a
segment's guess rarely meets the exact path within its warm-up, the
parallel re-walk round runs in most groups, and some re-walks end in a
different state than the first walk did, so the top-down check must walk
the segment below again.  Every bit is compared with the block oracle."""
import numpy as np
import pytest

from paper_1608_00066_gb300 import pbvd, synth

from gpu_util import T_VALUES, gpu_bits, make_decoder, oracle_bits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1608_00066_gb300 import build
    build.build()
    pbvd.load()


CASES = [
    # (code, D, L, stages)
    ("K7_r1/2", 1024, 42, 4 * 1024 + 37),
    ("K7_r1/2", 4096, 42, 2 * 4096 + 511),
    ("K7_r3/4", 2048, 42, 3 * 2048 + 5),
    ("K9_r1/3", 1024, 64, 4 * 1024 + 93),
    ("K9_r1/3", 2048, 64, 2 * 2048 + 8),
]


@pytest.mark.parametrize("name, D, L, n", CASES)
def test_noise_every_thread_count(name, D, L, n):
    spec = synth.CODES[name]
    rng = np.random.default_rng(D + L + n)
    dec = make_decoder(spec, D, L)
    llr = rng.integers(-127, 128, size=dec.llr_count(n), dtype=np.int16).astype(np.int8)
    want = oracle_bits(spec, llr, n, D, L)
    for T in T_VALUES[name]:
        for smem in (0, 1):
            try:
                got = gpu_bits(dec, llr, n, threads_per_pair=T, survivors_in_smem=smem)
            except pbvd.PbvdError as e:
                assert e.code == pbvd.PBVD_EINVAL and smem, (T, smem)  # records too large for shared memory
                continue
            bad = np.flatnonzero(got != want)
            assert bad.size == 0, (name, D, L, T, smem, bad[:8])
    dec.close()


@pytest.mark.parametrize("ebn0", [-2.0, 0.0])
def test_weak_signal_k7_every_thread_count(ebn0):
    """A transmitted stream at -2 and 0 dB: guesses fail often but not
    always, so some groups re-walk and others do not."""
    spec = synth.K7_R12
    f = synth.make_frame(spec, 20000, ebn0, seed=77 + int(ebn0))
    want = oracle_bits(spec, f.llr, f.n_stages, 2048, 42)
    dec = make_decoder(spec, 2048, 42)
    for T in T_VALUES[spec.name]:
        got = gpu_bits(dec, f.llr, f.n_stages, threads_per_pair=T, survivors_in_smem=0)
        assert np.array_equal(got, want), (ebn0, T)
    dec.close()


# Block lengths on both sides of the segment rule's switch (K=7, LAMBDA =
# 56 records of warm-up): lower segments of (J - LAMBDA) / T records when
# that is at least 2 LAMBDA, else the even split J / T, with J = D + L
# records per block; at two threads per pair the switch lies at J = 272, at
# four at J = 488.
@pytest.mark.parametrize("T, D", [(2, 224), (2, 232), (2, 240), (4, 440), (4, 448), (4, 456)])
def test_segment_rule_switch_k7(T, D):
    spec = synth.K7_R12
    L = 42
    f = synth.make_frame(spec, 24 * D + 13, 0.0, seed=500 + D)
    want = oracle_bits(spec, f.llr, f.n_stages, D, L)
    dec = make_decoder(spec, D, L)
    for smem in (0, 1):
        got = gpu_bits(dec, f.llr, f.n_stages, threads_per_pair=T, survivors_in_smem=smem)
        bad = np.flatnonzero(got != want)
        assert bad.size == 0, (T, D, smem, bad[:8])
    dec.close()
