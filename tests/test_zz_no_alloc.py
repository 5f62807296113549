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


def _records_per_pair(D, L):
    """Survivor records per pair of blocks: D + L stages rounded up to whole
    blocks of eight (the size the library reserves)."""
    return (D + L + 7) // 8 * 8


def test_noalloc_rejects_sizes_beyond_the_array():
    spec = synth.K7_R12
    dec = pbvd.Decoder(spec.K, spec.gens, None, 512, 42)
    dec.set_config(threads_per_pair=2, cta_threads=64, survivors_in_smem=0)
    cap = pbvd.pbvd_noalloc_max_survivor_bytes()
    assert cap == 16 << 20
    # at T = 2 a record is 16 bytes, 560 records per pair of 512-stage blocks
    per_pair = _records_per_pair(512, 42) * 16
    pairs = cap // per_pair
    n_ok = pairs * 1024              # the largest whole number of pairs that fits
    n_bad = n_ok + 1                 # one more block, one more pair
    d = torch.zeros(n_bad * 2, dtype=torch.int8, device="cuda")
    out = torch.zeros((n_bad + 7) // 8, dtype=torch.uint8, device="cuda")
    pbvd.pbvd_decode_noalloc(dec.ctx, d.data_ptr(), n_ok, out.data_ptr(), 0)
    torch.cuda.synchronize()
    with pytest.raises(pbvd.PbvdError) as ei:
        pbvd.pbvd_decode_noalloc(dec.ctx, d.data_ptr(), n_bad, out.data_ptr(), 0)
    assert ei.value.code == pbvd.PBVD_EINVAL
    dec.close()


def test_noalloc_accepts_a_stream_just_under_the_limit():
    """The largest stream that fits at T = 2 decodes to pbvd_decode's bits."""
    spec = synth.K7_R12
    dec = pbvd.Decoder(spec.K, spec.gens, None, 512, 42)
    dec.set_config(threads_per_pair=2, cta_threads=64, survivors_in_smem=0)
    pairs = pbvd.pbvd_noalloc_max_survivor_bytes() // (_records_per_pair(512, 42) * 16)
    n = pairs * 1024
    f = synth.make_frame(spec, n - spec.v, 2.0, seed=75)
    want = _decode(pbvd.pbvd_decode, dec, f.llr, f.n_stages)
    for _ in range(2):
        assert np.array_equal(_decode(pbvd.pbvd_decode_noalloc, dec, f.llr, f.n_stages), want)
    dec.close()


def test_noalloc_falls_back_to_fewer_threads_per_pair():
    """K=7, D=64, L=42: for 2,432 pairs of blocks the automatic configuration
    uses 16 threads per pair (16-word records: 17.4 MB of survivor bits, more
    than the array holds); the entry point falls back to 8 threads per pair
    (8-word records, 8.7 MB) and must still give pbvd_decode's bits."""
    spec = synth.K7_R12
    D, L = 64, 42
    n = 2432 * 2 * D
    dec = pbvd.Decoder(spec.K, spec.gens, None, D, L)
    cfg = dec.get_config(n)
    assert cfg["threads_per_pair"] == 16 and cfg["survivors_in_smem"] == 0
    assert _records_per_pair(D, L) * 2432 * 16 * 4 > pbvd.pbvd_noalloc_max_survivor_bytes()
    f = synth.make_frame(spec, n - spec.v, 1.0, seed=76)
    want = _decode(pbvd.pbvd_decode, dec, f.llr, f.n_stages)
    for _ in range(2):
        assert np.array_equal(_decode(pbvd.pbvd_decode_noalloc, dec, f.llr, f.n_stages), want)
    dec.close()


def test_noalloc_keeps_shared_memory_survivors_for_short_frames():
    """One 4096-bit frame: the automatic configuration keeps the survivors in
    shared memory, which needs no allocation either."""
    spec = synth.K7_R12
    dec = pbvd.Decoder(spec.K, spec.gens, None, 512, 42)
    f = synth.make_frame(spec, 4096, 3.0, seed=1001)
    assert dec.get_config(f.n_stages)["survivors_in_smem"] == 1
    want = _decode(pbvd.pbvd_decode, dec, f.llr, f.n_stages)
    for _ in range(2):
        assert np.array_equal(_decode(pbvd.pbvd_decode_noalloc, dec, f.llr, f.n_stages), want)
    dec.close()


def test_noalloc_needs_run_time_kernels_loaded_first():
    """A code without a built-in kernel is compiled at run time, and loading
    that kernel allocates device memory: the allocation-free call refuses it
    until pbvd_decode has loaded it, then gives the same bits."""
    # a code no other test decodes, so that its kernel is not loaded yet even
    # when the whole suite ran before in this process
    spec = synth.CodeSpec("K6_65_57", 6, (0o65, 0o57))
    dec = pbvd.Decoder(spec.K, spec.gens, None, 256, 36)
    dec.set_config(threads_per_pair=4, cta_threads=64, survivors_in_smem=0)
    f = synth.make_frame(spec, 20000, 2.0, seed=77)
    with pytest.raises(pbvd.PbvdError) as ei:
        _decode(pbvd.pbvd_decode_noalloc, dec, f.llr, f.n_stages)
    assert ei.value.code == pbvd.PBVD_EUNSUPPORTED
    want = _decode(pbvd.pbvd_decode, dec, f.llr, f.n_stages)
    for _ in range(2):
        assert np.array_equal(_decode(pbvd.pbvd_decode_noalloc, dec, f.llr, f.n_stages), want)
    dec.close()
