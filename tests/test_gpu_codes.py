"""Codes beyond the benchmark's three, bit for bit against the block oracle.

Sec. III-B states the method for any (R,1,K) code and names the widely used
rate-1/2 codes with K = 5, 7, 9 and rate-1/3 codes with K = 7, 9.  The
library has compiled kernels for the (3,1,7) (171,165,133) and (2,1,5)
(23,35) codes; every other valid code is compiled at run time from the same
kernel template on its first decode.  The run-time codes below include one
whose generators do not all tap the oldest cell (no complement symmetry of
the branch metrics), one with a generator that skips the input tap, and a
punctured one."""
import numpy as np
import pytest

from paper_1608_00066_gb300 import pbvd, synth

from gpu_util import gpu_bits, make_decoder, oracle_bits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(1, 8, 0), (5, 8, 42), (300, 16, 35), (2000, 512, 42), (2999, 256, 64), (4093, 64, 0),
          (20000, 512, 42)]

BUILT = [
    (synth.CodeSpec("K7_r1/3", 7, (0o171, 0o165, 0o133)), (1, 2, 4, 8, 16, 32)),
    (synth.CodeSpec("K5_r1/2", 5, (0o23, 0o35)), (1, 2, 4, 8)),
]

RUNTIME = [
    synth.CodeSpec("K4_13_16", 4, (0o13, 0o16)),             # g_0 taps only one generator
    synth.CodeSpec("K3_3_7", 3, (0o3, 0o7)),                 # first generator skips the input tap
    synth.CodeSpec("K6_53_75", 6, (0o53, 0o75)),
    synth.CodeSpec("K8_247_371", 8, (0o247, 0o371)),
    synth.CodeSpec("K9_561_753", 9, (0o561, 0o753)),         # rate-1/2 256-state code
    synth.CodeSpec("K5_25_33_37", 5, (0o25, 0o33, 0o37)),
    synth.CodeSpec("K6_53_75_p23", 6, (0o53, 0o75), ((1, 1), (1, 0))),  # punctured to rate 2/3
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1608_00066_gb300 import build
    build.build()
    pbvd.load()


def _check(spec, Ts, shapes, seed):
    rng = np.random.default_rng(seed)
    for (k, D, L) in shapes:
        f = synth.make_frame(spec, k, float(rng.uniform(-1, 4)), seed=int(rng.integers(1 << 30)))
        want = oracle_bits(spec, f.llr, f.n_stages, D, L)
        dec = make_decoder(spec, D, L)
        for T in Ts:
            for smem in (0, 1):
                got = gpu_bits(dec, f.llr, f.n_stages, threads_per_pair=T, survivors_in_smem=smem)
                bad = np.flatnonzero(got != want)
                assert bad.size == 0, (spec.name, k, D, L, T, smem, bad[:10])
        got = gpu_bits(dec, f.llr, f.n_stages, threads_per_pair=0, cta_threads=0, survivors_in_smem=-1)
        assert np.array_equal(got, want), (spec.name, k, D, L, "auto")
        dec.close()


@pytest.mark.parametrize("spec,Ts", BUILT, ids=[s.name for s, _ in BUILT])
def test_built_in_codes(spec, Ts):
    _check(spec, Ts, SHAPES, seed=len(spec.name))


def _runtime_Ts(spec):
    N = 1 << (spec.K - 1)
    return [T for T in (1, 2, 4, 8, 16) if T <= N // 2 and N // T <= 64]


@pytest.mark.parametrize("spec", RUNTIME, ids=[s.name for s in RUNTIME])
def test_runtime_compiled_codes(spec):
    Ts = _runtime_Ts(spec)
    # the smallest and largest thread counts of every code, all of them for two
    _check(spec, Ts if spec.K in (4, 6) else [Ts[0], Ts[-1]], SHAPES[1:6], seed=spec.K * 7)


def test_runtime_code_noiseless_round_trip_and_host_pipeline():
    """A run-time code decodes an error-free frame to its message, and the
    host-memory pipeline gives the device decode's bits."""
    spec = RUNTIME[4]
    f = synth.make_frame(spec, 50000, None, seed=9)
    dec = make_decoder(spec, 512, 48)
    got = gpu_bits(dec, f.llr, f.n_stages)
    assert np.array_equal(got[:50000], f.msg)
    h_llr = torch.from_numpy(f.llr).pin_memory()
    h_out = torch.zeros((f.n_stages + 7) // 8, dtype=torch.uint8).pin_memory()
    dec.decode_host(h_llr, f.n_stages, out=h_out, segments=3)
    torch.cuda.synchronize()
    assert np.array_equal(np.unpackbits(h_out.numpy(), bitorder="little")[:f.n_stages], got)
    dec.close()


def test_runtime_codes_are_not_batched():
    """The persistent batch kernel covers the benchmark's codes only."""
    spec = RUNTIME[2]
    f = synth.make_frame(spec, 1000, 2.0, seed=5)
    dec = make_decoder(spec, 512, 42)
    d = torch.from_numpy(f.llr).cuda()
    o = torch.zeros((f.n_stages + 7) // 8, dtype=torch.uint8, device="cuda")
    with pytest.raises(pbvd.PbvdError) as ei:
        pbvd.pbvd_decode_batch([(dec.ctx, d.data_ptr(), f.n_stages, o.data_ptr())])
    assert ei.value.code == pbvd.PBVD_EUNSUPPORTED
    dec.close()
