"""Batched decode of mixed-code frames in one persistent launch: every frame
equals its block-based oracle result and its plain single-frame decode,
bit for bit; the prepared batch replays under a CUDA graph."""
import numpy as np
import pytest

import oracle
from paper_1608_00066_gb300 import pbvd, synth

from gpu_util import mother_llr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DL = {"K7_r1/2": (512, 42), "K7_r3/4": (512, 42), "K9_r1/3": (1024, 64)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1608_00066_gb300 import build
    build.build()
    pbvd.load()


def _setup(frames):
    decs = {name: pbvd.Decoder(synth.CODES[name].K, synth.CODES[name].gens, synth.CODES[name].puncture,
                               *DL[name]) for name in DL}
    llrs, outs, items = [], [], []
    for f in frames:
        d = torch.from_numpy(f.llr).cuda()
        o = torch.full(((f.n_stages + 7) // 8,), 0xA5, dtype=torch.uint8, device="cuda")
        llrs.append(d)
        outs.append(o)
        items.append((decs[f.spec.name].ctx, d.data_ptr(), f.n_stages, o.data_ptr()))
    return decs, llrs, outs, items


def _bits(o, n):
    return np.unpackbits(o.cpu().numpy(), bitorder="little")[:n]


def test_batch_equals_oracle_and_plain():
    frames = synth.batch_frames(160, seed=4001, k_range=(1, 6144))
    decs, llrs, outs, items = _setup(frames)
    pbvd.pbvd_decode_batch(items)
    torch.cuda.synchronize()
    for f, o, d in zip(frames, outs, llrs):
        D, L = DL[f.spec.name]
        want = oracle.viterbi_block(f.spec.K, f.spec.gens, mother_llr(f.spec, f.llr, f.n_stages), D, L)
        got = _bits(o, f.n_stages)
        assert np.array_equal(got, want), (f.spec.name, f.n_stages)
        alone = decs[f.spec.name].decode(d, f.n_stages)
        torch.cuda.synchronize()
        assert np.array_equal(_bits(alone, f.n_stages), got)
    # a second call reuses the lead context's work list
    for o in outs:
        o.fill_(0)
    pbvd.pbvd_decode_batch(items[::-1])
    torch.cuda.synchronize()
    for f, o in zip(frames, outs):
        D, L = DL[f.spec.name]
        want = oracle.viterbi_block(f.spec.K, f.spec.gens, mother_llr(f.spec, f.llr, f.n_stages), D, L)
        assert np.array_equal(_bits(o, f.n_stages), want)


def test_batch_graph_replay_and_single_code():
    frames = synth.batch_frames(60, seed=4002, codes=(synth.K7_R12,))
    decs, llrs, outs, items = _setup(frames)
    b = pbvd.pbvd_batch_prepare(items)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        pbvd.pbvd_batch_run(b, s.cuda_stream)
    for rep in range(2):
        for o in outs:
            o.fill_(0)
        g.replay()
        torch.cuda.synchronize()
        for f, o in zip(frames, outs):
            want = oracle.viterbi_block(7, f.spec.gens, f.llr.reshape(-1, 2), 512, 42)
            assert np.array_equal(_bits(o, f.n_stages), want), rep
    pbvd.pbvd_batch_destroy(b)


def test_batch_rejects_mixed_geometry_and_unknown_codes():
    f = synth.make_frame(synth.K7_R12, 1000, 2.0, seed=5)
    d = torch.from_numpy(f.llr).cuda()
    o = torch.zeros((f.n_stages + 7) // 8, dtype=torch.uint8, device="cuda")
    a = pbvd.Decoder(7, synth.K7_R12.gens, None, 512, 42)
    b = pbvd.Decoder(7, synth.K7_R12.gens, None, 256, 42)
    with pytest.raises(pbvd.PbvdError) as ei:
        pbvd.pbvd_decode_batch([(a.ctx, d.data_ptr(), f.n_stages, o.data_ptr()),
                                (b.ctx, d.data_ptr(), f.n_stages, o.data_ptr())])
    assert ei.value.code == pbvd.PBVD_EINVAL
    k3 = pbvd.Decoder(3, (0o7, 0o5), None, 64, 10)
    with pytest.raises(pbvd.PbvdError) as ei:
        pbvd.pbvd_decode_batch([(k3.ctx, d.data_ptr(), 100, o.data_ptr())])
    assert ei.value.code == pbvd.PBVD_EUNSUPPORTED
