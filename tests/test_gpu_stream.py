"""Continuous streams with device-resident path metrics: whatever the chunking,
the bits equal the oracle's carried-metric window form (Eq. (1) run once over
the whole stream, segment m released by traceback from S_0 at stage
(m+1)D + L - 1, the rest at the end), bit for bit; bits reported released
are final when reported."""
import numpy as np
import pytest

import oracle
from paper_1608_00066_gb300 import pbvd, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STREAM_CODES = ("K7_r1/2", "K9_r1/3")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1608_00066_gb300 import build
    build.build()
    pbvd.load()


def _chunks(rng, n, max_push, mode):
    if mode == "even":
        sizes = [max_push] * (n // max_push) + ([n % max_push] if n % max_push else [])
    elif mode == "tiny":
        sizes = list(rng.integers(0, 5, size=4 * n // 2))
    else:
        sizes = list(rng.integers(0, max_push + 1, size=4 * n // max(1, max_push // 2) + 8))
    out, t = [], 0
    for c in sizes:
        c = int(min(c, n - t))
        out.append(c)
        t += c
        if t == n:
            break
    if t < n:
        while t < n:
            c = min(max_push, n - t)
            out.append(c)
            t += c
    return out


def _run_stream(spec, llr, D, L, chunks, max_push, check_released=True):
    n = llr.shape[0]
    dec = pbvd.Decoder(spec.K, spec.gens, None, D, L)
    st = pbvd.Stream(dec, n, max_push)
    st.out.fill_(0xA5)
    d = torch.from_numpy(np.ascontiguousarray(llr).reshape(-1)).cuda()
    ref = oracle.viterbi_window(spec.K, spec.gens, llr, D, L)
    t = 0
    for c in chunks:
        st.push(d[t * spec.R:(t + c) * spec.R] if c else d[:0], c)
        t += c
        if check_released:
            torch.cuda.synchronize()
            rel = st.released
            assert 0 <= rel <= t
            assert rel % D == 0
            # every segment whose trigger stage has been decoded is released
            # (up to P - 1 < 8 pushed stages wait in the carry buffer)
            assert t - 7 < rel + D + L
            if rel:
                got = np.unpackbits(st.out.cpu().numpy(), bitorder="little")[:rel]
                assert np.array_equal(got, ref[:rel])
    st.close()
    torch.cuda.synchronize()
    assert st.released == n
    got = np.unpackbits(st.out.cpu().numpy(), bitorder="little")[:n]
    st.destroy()
    dec.close()
    return got, ref


@pytest.mark.parametrize("name", STREAM_CODES)
@pytest.mark.parametrize("mode", ["even", "random", "tiny"])
def test_stream_matches_window_oracle(name, mode):
    spec = synth.CODES[name]
    D, L = (512, 42) if spec.K == 7 else (1024, 64)
    k = 6000 if mode != "tiny" else 700
    f = synth.make_frame(spec, k, 2.0, seed=7001 + len(mode))
    llr = f.llr.reshape(f.n_stages, spec.R)
    rng = np.random.default_rng(11)
    max_push = 1000
    chunks = _chunks(rng, f.n_stages, max_push, mode)
    got, ref = _run_stream(spec, llr, D, L, chunks, max_push, check_released=(mode != "tiny"))
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("name", STREAM_CODES)
@pytest.mark.parametrize("D,L", [(8, 0), (16, 42), (64, 7), (2048, 96)])
def test_stream_geometries(name, D, L):
    spec = synth.CODES[name]
    f = synth.make_frame(spec, 3000, 1.0, seed=7100 + D + L)
    llr = f.llr.reshape(f.n_stages, spec.R)
    rng = np.random.default_rng(D * 1000 + L)
    chunks = _chunks(rng, f.n_stages, 257, "random")
    got, ref = _run_stream(spec, llr, D, L, chunks, 257)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 9, 41, 50])
def test_stream_short(n):
    spec = synth.K7_R12
    rng = np.random.default_rng(n)
    llr = rng.integers(-128, 128, size=(n, 2), dtype=np.int8)
    got, ref = _run_stream(spec, llr, 16, 42, [1] * n, 4)
    assert np.array_equal(got, ref)


def test_stream_extreme_values():
    # saturated soft values and ties over a long stream: the carried metrics
    # are renormalised across pushes and stay exact
    spec = synth.K7_R12
    rng = np.random.default_rng(3)
    n = 40000
    llr = rng.choice(np.array([-128, -127, 0, 127], np.int8), size=(n, 2))
    chunks = _chunks(rng, n, 4096, "random")
    got, ref = _run_stream(spec, llr, 512, 42, chunks, 4096, check_released=False)
    assert np.array_equal(got, ref)


def test_push_many_mixed_lengths_equal_alone():
    spec = synth.K7_R12
    D, L = 256, 42
    nstreams = 150          # more than one launch of descriptors
    rng = np.random.default_rng(5)
    max_push = 300
    lens = rng.integers(500, 3000, size=nstreams)
    frames = [synth.make_frame(spec, int(k) - 6, 2.5, seed=7200 + i) for i, k in enumerate(lens)]
    dec = pbvd.Decoder(spec.K, spec.gens, None, D, L)
    sts = [pbvd.Stream(dec, f.n_stages, max_push) for f in frames]
    dls = [torch.from_numpy(f.llr).cuda() for f in frames]
    pos = [0] * nstreams
    while True:
        hs, ps, ns = [], [], []
        for i, f in enumerate(frames):
            c = int(min(rng.integers(0, max_push + 1), f.n_stages - pos[i]))
            hs.append(sts[i].handle)
            ps.append(dls[i][pos[i] * 2:].data_ptr() if c else 0)
            ns.append(c)
            pos[i] += c
        pbvd.pbvd_stream_push_many(hs, ps, ns, close=False, stream=torch.cuda.current_stream().cuda_stream)
        if all(p == f.n_stages for p, f in zip(pos, frames)):
            break
    pbvd.pbvd_stream_push_many([s.handle for s in sts], [0] * nstreams, [0] * nstreams, close=True,
                               stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for i, f in enumerate(frames):
        got = np.unpackbits(sts[i].out.cpu().numpy(), bitorder="little")[:f.n_stages]
        ref = oracle.viterbi_window(spec.K, spec.gens, f.llr.reshape(-1, 2), D, L)
        assert np.array_equal(got, ref), i
        if i % 37 == 0:
            alone, _ = _run_stream(spec, f.llr.reshape(-1, 2), D, L, [f.n_stages], f.n_stages,
                                   check_released=False)
            assert np.array_equal(alone, got)
    for s in sts:
        s.destroy()
    dec.close()


def test_stream_large():
    # 2^20 stages in 64 Ki-stage pushes; the whole stream checked
    spec = synth.K7_R12
    f = synth.make_frame(spec, (1 << 20) - 6, 3.0, seed=7300)
    llr = f.llr.reshape(f.n_stages, 2)
    got, ref = _run_stream(spec, llr, 512, 42, [1 << 16] * 16, 1 << 16, check_released=False)
    assert np.array_equal(got, ref)


def test_stream_errors():
    import ctypes
    spec = synth.K7_R12
    dec = pbvd.Decoder(spec.K, spec.gens, None, 512, 42)
    out = torch.zeros(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(pbvd.PbvdError) as e:
        pbvd.pbvd_stream_open(dec.ctx, 0, out.data_ptr(), 128)
    assert e.value.code == pbvd.PBVD_EINVAL
    p34 = synth.K7_R34
    dp = pbvd.Decoder(p34.K, p34.gens, p34.puncture, 512, 42)
    with pytest.raises(pbvd.PbvdError) as e:
        pbvd.pbvd_stream_open(dp.ctx, 64, out.data_ptr(), 128)
    assert e.value.code == pbvd.PBVD_EUNSUPPORTED
    k3 = synth.K3_R12
    d3 = pbvd.Decoder(k3.K, k3.gens, None, 16, 18)
    with pytest.raises(pbvd.PbvdError) as e:
        pbvd.pbvd_stream_open(d3.ctx, 64, out.data_ptr(), 128)
    assert e.value.code == pbvd.PBVD_EUNSUPPORTED
    h = pbvd.pbvd_stream_open(dec.ctx, 64, out.data_ptr(), 128)
    llr = torch.zeros(200, dtype=torch.int8, device="cuda")
    # more than max_push stages, more than the output capacity
    with pytest.raises(pbvd.PbvdError):
        pbvd.pbvd_stream_push(h, llr.data_ptr(), 65)
    pbvd.pbvd_stream_push(h, llr.data_ptr(), 64)
    pbvd.pbvd_stream_push(h, llr.data_ptr(), 64)
    with pytest.raises(pbvd.PbvdError):
        pbvd.pbvd_stream_push(h, llr.data_ptr(), 1)
    # the same stream twice in one launch
    with pytest.raises(pbvd.PbvdError):
        pbvd.pbvd_stream_push_many([h, h], [0, 0], [0, 0])
    pbvd.pbvd_stream_close(h)
    with pytest.raises(pbvd.PbvdError):
        pbvd.pbvd_stream_close(h)
    torch.cuda.synchronize()
    assert pbvd.pbvd_stream_released(h) == 128
    pbvd.pbvd_stream_destroy(h)
    del ctypes
    for d in (dec, dp, d3):
        d.close()


@pytest.mark.parametrize("name", STREAM_CODES)
def test_carried_metrics_equal_oracle_up_to_a_shift(name):
    """The stream's 16-bit renormalised path metrics after every push equal
    the oracle's exact int64 metrics of Eq. (1) after the same stage (known
    start S_0, full-frame form) up to one common offset per stage, over
    pushes of uneven sizes, noisy and noiseless stretches and the first
    stages where only part of the states are reachable."""
    spec = synth.CODES[name]
    rng = np.random.default_rng(31 + spec.K)
    n = 20000
    f = synth.make_frame(spec, n - spec.v, 1.0, seed=spec.K)
    llr = np.asarray(f.llr, np.int8).reshape(n, spec.R).copy()
    llr[8000:9000] = rng.integers(-127, 128, size=(1000, spec.R), dtype=np.int16).astype(np.int8)
    _, _, _, pm_trace = oracle.viterbi_full(spec.K, spec.gens, llr, want_trace=True)
    dec = pbvd.Decoder(spec.K, spec.gens, None, 512, 42)
    st = pbvd.Stream(dec, n, 4096)
    d = torch.from_numpy(llr.reshape(-1)).cuda()
    t, checked = 0, 0
    for c in [1, 2, 3, 5, 7, 64, 1000, 4096, 300, 4096, 4096, 4096, 2000]:
        c = min(c, n - t)
        if c == 0:
            break
        st.push(d[t * spec.R:(t + c) * spec.R], c)
        t += c
        done, pm = st.metrics()
        if done == 0:
            continue
        want = pm_trace[done - 1]
        assert np.array_equal(pm.astype(np.int64) - pm[0], want - want[0]), (name, done)
        checked += 1
    assert checked >= 8
    st.destroy()
    dec.close()
