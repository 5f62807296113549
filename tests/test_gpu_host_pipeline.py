"""pbvd_decode_host: a stream in host memory, cut into runs of blocks whose
copies overlap the decoding (Sec. IV-C), or read and written in place by the
kernel (direct access to page-locked buffers), must give exactly the bits of
pbvd_decode on the same soft values (and so the block oracle's), for any
number of runs, ragged last runs, direct access, punctured codes, the
256-state code, page-locked and pageable host buffers, and calls in a row."""
import numpy as np
import pytest

from paper_1608_00066_gb300 import pbvd, synth

from gpu_util import make_decoder, oracle_bits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1608_00066_gb300 import build
    build.build()
    pbvd.load()


def _device_bits(dec, f):
    d = torch.from_numpy(f.llr).cuda()
    out = dec.decode(d, f.n_stages)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _host_bits(dec, f, segments, pinned=True):
    h = torch.from_numpy(f.llr.copy())
    if pinned:
        h = h.pin_memory()
    nbytes = (f.n_stages + 7) // 8
    out = torch.full((nbytes,), 0xA5, dtype=torch.uint8)
    if pinned:
        out = out.pin_memory()
    dec.decode_host(h, f.n_stages, out=out, segments=segments)
    torch.cuda.synchronize()
    return out.numpy().copy()


@pytest.mark.parametrize("name,k,D,L", [
    ("K7_r1/2", 300000, 512, 42),
    ("K7_r1/2", 123457, 256, 35),
    ("K7_r3/4", 200001, 512, 42),
    ("K9_r1/3", 100003, 1024, 64),
    ("K7_r1/2", 140001, 64, 42),    # 2188 blocks: two automatic runs
])
def test_matches_device_decode(name, k, D, L):
    spec = synth.CODES[name]
    f = synth.make_frame(spec, k, 2.0, seed=k)
    dec = make_decoder(spec, D, L)
    want = _device_bits(dec, f)
    for segments in (0, -1, 1, 2, 3, 7, 64):
        got = _host_bits(dec, f, segments)
        assert np.array_equal(got, want), segments
    dec.close()


def test_small_and_ragged_against_oracle():
    spec = synth.K7_R12
    for k, D, L, segments in ((1, 8, 5, 0), (50, 16, 20, 3), (3001, 64, 42, 64), (4000, 512, 42, 5),
                              (2, 8, 5, -1), (777, 16, 20, -1)):
        f = synth.make_frame(spec, k, 1.5, seed=100 + k)
        dec = make_decoder(spec, D, L)
        want = np.packbits(oracle_bits(spec, f.llr, f.n_stages, D, L), bitorder="little")
        got = _host_bits(dec, f, segments)
        assert np.array_equal(got, want), (k, D, L, segments)
        dec.close()


def test_pageable_buffers_and_calls_in_a_row():
    spec = synth.K7_R12
    dec = make_decoder(spec, 512, 42)
    frames = [synth.make_frame(spec, k, 2.5, seed=k) for k in (250000, 70001, 250000)]
    for f in frames:
        want = _device_bits(dec, f)
        assert np.array_equal(_host_bits(dec, f, 0, pinned=False), want)
        assert np.array_equal(_host_bits(dec, f, 6, pinned=True), want)
    dec.close()


def test_direct_access_needs_mapped_buffers():
    """segments = -1 with a pageable buffer is refused on the host, before
    anything is enqueued; the copy pipeline takes any mix of buffers."""
    spec = synth.K7_R12
    f = synth.make_frame(spec, 5000, 2.0, seed=77)
    dec = make_decoder(spec, 512, 42)
    want = _device_bits(dec, f)
    h = torch.from_numpy(f.llr.copy())
    out = torch.zeros((f.n_stages + 7) // 8, dtype=torch.uint8)
    with pytest.raises(pbvd.PbvdError):
        dec.decode_host(h, f.n_stages, out=out, segments=-1)
    with pytest.raises(pbvd.PbvdError):
        dec.decode_host(h.pin_memory(), f.n_stages, out=out, segments=-1)
    dec.decode_host(h, f.n_stages, out=out, segments=0)
    torch.cuda.synchronize()
    assert np.array_equal(out.numpy(), want)
    out.zero_()
    dec.decode_host(h.pin_memory(), f.n_stages, out=out, segments=0)
    torch.cuda.synchronize()
    assert np.array_equal(out.numpy(), want)
    dec.close()


def test_two_contexts_in_flight():
    """Calls on two contexts and two CUDA streams overlap on the GPU (one
    call's copies with the other's decoding); every output stays exact."""
    spec = synth.K7_R12
    frames = [synth.make_frame(spec, 200000 + 1000 * i, 2.5, seed=300 + i) for i in range(6)]
    decs = [make_decoder(spec, 512, 42) for _ in range(2)]
    streams = [torch.cuda.Stream() for _ in range(2)]
    want = [_device_bits(decs[0], f) for f in frames]
    hins = [torch.from_numpy(f.llr.copy()).pin_memory() for f in frames]
    outs = [torch.zeros((f.n_stages + 7) // 8, dtype=torch.uint8).pin_memory() for f in frames]
    for i, f in enumerate(frames):
        decs[i & 1].decode_host(hins[i], f.n_stages, out=outs[i], stream=streams[i & 1])
    torch.cuda.synchronize()
    for i in range(len(frames)):
        assert np.array_equal(outs[i].numpy(), want[i]), i
    for d in decs:
        d.close()
