"""The paper's two-kernel design (K1 forward with one thread per butterfly
group, K2 traceback with one thread per block; Algorithm 1, Table 1), kept
as an ablation: the same bits as the block oracle and as the fused kernel."""
import numpy as np
import pytest

from paper_1608_00066_gb300 import pbvd, synth

from gpu_util import gpu_bits, make_decoder, oracle_bits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(1, 8, 0), (5, 8, 42), (100, 8, 20), (300, 16, 35), (2000, 512, 42), (2999, 256, 64),
          (777, 1024, 42), (3000, 24, 100), (4093, 512, 0), (40000, 512, 42)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1608_00066_gb300 import build
    build.build()
    pbvd.load()


def _two_kernel_bits(dec, llr, n):
    d = torch.from_numpy(np.ascontiguousarray(llr)).cuda()
    out = torch.full(((n + 7) // 8,), 0xA5, dtype=torch.uint8, device="cuda")
    pbvd.pbvd_decode_two_kernel(dec.ctx, d.data_ptr(), n, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return np.unpackbits(out.cpu().numpy(), bitorder="little")[:n]


@pytest.mark.parametrize("name", ["K7_r1/2", "K9_r1/3"])
def test_two_kernel_equals_oracle(name):
    spec = synth.CODES[name]
    rng = np.random.default_rng(77 + len(name))
    for (k, D, L) in SHAPES:
        f = synth.make_frame(spec, k, float(rng.uniform(-1, 4)), seed=int(rng.integers(1 << 30)))
        want = oracle_bits(spec, f.llr, f.n_stages, D, L)
        dec = make_decoder(spec, D, L)
        got = _two_kernel_bits(dec, f.llr, f.n_stages)
        bad = np.flatnonzero(got != want)
        assert bad.size == 0, (name, k, D, L, bad[:10])
        dec.close()


def test_two_kernel_equals_fused_on_the_benchmark_stream():
    spec = synth.K7_R12
    f = synth.make_frame(spec, 1 << 24, 3.0, seed=2003)
    dec = make_decoder(spec, 512, 42)
    fused = gpu_bits(dec, f.llr, f.n_stages)
    two = _two_kernel_bits(dec, f.llr, f.n_stages)
    assert np.array_equal(two, fused)
    dec.close()


def test_two_kernel_rejects_other_codes_and_modes():
    for spec in (synth.K7_R34, synth.K3_R12):
        dec = make_decoder(spec, 512, 42)
        with pytest.raises(pbvd.PbvdError) as ei:
            _two_kernel_bits(dec, np.zeros(4000, np.int8), 1000)
        assert ei.value.code == pbvd.PBVD_EUNSUPPORTED
        dec.close()
    dec = make_decoder(synth.K7_R12, 512, 42)
    dec.set_mode(argmin=True)
    with pytest.raises(pbvd.PbvdError) as ei:
        _two_kernel_bits(dec, np.zeros(4000, np.int8), 1000)
    assert ei.value.code == pbvd.PBVD_EUNSUPPORTED
    dec.close()
