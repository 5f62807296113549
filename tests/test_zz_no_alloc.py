"""The allocation-free entry point, pbvd_decode_noalloc, for callers that may
not allocate device memory while decoding (stream capture, real-time chains
with memory reserved up front, hosts with their own pool allocator).  It must
give exactly the bits of pbvd_decode, call after call, although every call
reuses the same fixed survivor array, and must refuse sizes beyond that
array.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1608_00066_gb300 import pbvd, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1608_00066_gb300 import build
    build.build()
    pbvd.load()


def _decode(fn, dec, llr, n):
    d = torch.from_numpy(np.ascontiguousarray(llr)).cuda()
    out = torch.full(((n + 7) // 8,), 0x5A, dtype=torch.uint8, device="cuda")
    fn(dec.ctx, d.data_ptr(), n, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_decode_on_consecutive_calls():
    spec = synth.K7_R12
    dec = pbvd.Decoder(spec.K, spec.gens, None, 512, 42)
    frames = [synth.make_frame(spec, 300000, 2.0, seed=71), synth.make_frame(spec, 123457, 1.0, seed=72)]
    # two calls in a row on the same input, then a call on another input
    for f in (frames[0], frames[0], frames[1]):
        want = _decode(pbvd.pbvd_decode, dec, f.llr, f.n_stages)
        got = _decode(pbvd.pbvd_decode_noalloc, dec, f.llr, f.n_stages)
        assert np.array_equal(got, want)
    dec.close()


def test_noalloc_punctured_and_k9():
    for spec, k in ((synth.K7_R34, 50000), (synth.K9_R13, 40000)):
        dec = pbvd.Decoder(spec.K, spec.gens, spec.puncture, 256, 48)
        f = synth.make_frame(spec, k, 2.5, seed=73)
        want = _decode(pbvd.pbvd_decode, dec, f.llr, f.n_stages)
        for _ in range(2):
            got = _decode(pbvd.pbvd_decode_noalloc, dec, f.llr, f.n_stages)
            assert np.array_equal(got, want)
        dec.close()


def test_noalloc_rejects_sizes_beyond_the_array():
    spec = synth.K7_R12
    dec = pbvd.Decoder(spec.K, spec.gens, None, 512, 42)
    dec.set_config(threads_per_pair=2, cta_threads=64, survivors_in_smem=0)
    cap = pbvd.pbvd_noalloc_max_survivor_bytes()
    assert cap == 16 << 20
    # 554 records of 16 bytes per pair of blocks at T = 2
    n = (cap // (554 * 16) + 64) * 1024
    d = torch.zeros(n * 2, dtype=torch.int8, device="cuda")
    out = torch.zeros((n + 7) // 8, dtype=torch.uint8, device="cuda")
    with pytest.raises(pbvd.PbvdError) as ei:
        pbvd.pbvd_decode_noalloc(dec.ctx, d.data_ptr(), n, out.data_ptr(), 0)
    assert ei.value.code == pbvd.PBVD_EINVAL
    dec.close()
