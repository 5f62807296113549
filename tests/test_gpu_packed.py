"""q-bit packed soft inputs (Sec. IV-C) and hard decisions (q = 1) on the
GPU: pbvd_decode_packed and pbvd_decode_host_packed against the q-bit block
oracle (mu = +-Q), bit for bit."""
import numpy as np
import pytest

import oracle
from paper_1608_00066_gb300 import pbvd, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DL = {"K7_r1/2": (512, 42), "K7_r3/4": (256, 42), "K9_r1/3": (1024, 64), "K3_r1/2": (64, 15)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1608_00066_gb300 import build
    build.build()
    pbvd.load()


def _want(spec, f, D, L):
    n = f.n_stages
    vals = oracle.unpack_soft(f.q, f.words, len(f.values))
    if spec.puncture is not None:
        vals = oracle.depuncture(spec.pattern_array(), vals, n)
    return oracle.viterbi_block_q(spec.K, spec.gens, vals.reshape(n, spec.R), D, L, oracle.q_max(f.q))


def _words_tensor(f):
    return torch.from_numpy(f.words.view(np.int32).copy())


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5, 8])
@pytest.mark.parametrize("name", ["K7_r1/2", "K7_r3/4", "K9_r1/3", "K3_r1/2"])
def test_packed_device_decode(q, name):
    spec = synth.CODES[name]
    D, L = DL[name]
    dec = pbvd.Decoder(spec.K, spec.gens, spec.puncture, D, L)
    for k, eb in ((20000, 2.0), (777, 0.0), (3, 1.0)):
        f = synth.make_packed_frame(spec, k, eb, q, seed=k + q)
        want = _want(spec, f, D, L)
        out = dec.decode_packed(_words_tensor(f).cuda(), q, f.n_stages)
        torch.cuda.synchronize()
        got = np.unpackbits(out.cpu().numpy(), bitorder="little")[:f.n_stages]
        bad = np.flatnonzero(got != want)
        assert bad.size == 0, (name, q, k, bad[:8])
    dec.close()


@pytest.mark.parametrize("q", [1, 3, 4])
def test_packed_host_pipeline(q):
    """Host-memory packed input through the copy pipeline (several runs)
    equals the device decode and the oracle."""
    spec = synth.K7_R12
    f = synth.make_packed_frame(spec, 1 << 20, 3.0, q, seed=q)
    want = _want(spec, f, 512, 42)
    dec = pbvd.Decoder(spec.K, spec.gens, None, 512, 42)
    h_words = _words_tensor(f).pin_memory()
    h_out = torch.zeros((f.n_stages + 7) // 8, dtype=torch.uint8).pin_memory()
    for seg in (0, 1, 5):
        h_out.zero_()
        pbvd.pbvd_decode_host_packed(dec.ctx, h_words.data_ptr(), q, f.n_stages, h_out.data_ptr(), seg,
                                     torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        got = np.unpackbits(h_out.numpy(), bitorder="little")[:f.n_stages]
        assert np.array_equal(got, want), (q, seg)
    dec.close()


def test_packed_rejects_bad_q():
    spec = synth.K7_R12
    dec = pbvd.Decoder(spec.K, spec.gens, None, 512, 42)
    w = torch.zeros(64, dtype=torch.int32, device="cuda")
    o = torch.zeros(64, dtype=torch.uint8, device="cuda")
    for q in (0, 9):
        with pytest.raises(pbvd.PbvdError) as ei:
            pbvd.pbvd_decode_packed(dec.ctx, w.data_ptr(), q, 100, o.data_ptr(), 0)
        assert ei.value.code == pbvd.PBVD_EINVAL
    dec.close()
