"""Parity at the configurations the kernels are tuned and benchmarked in,
bit for bit against the block-based CPU oracle on every block:

  * long blocks, D in {2048, 4096, 8192} (the geometry tuner's candidates),
    through pbvd_decode, pbvd_decode_batch and pbvd_decode_host;
  * long overlaps, L in {256, 1024, 4096} (the renormalisation interval and
    the survivor ring sizes depend on L);
  * the full-size streams of 2^24 information bits (K=7 r1/2 and r3/4 at
    D=512 L=42, K=9 r1/3 at D=1024 L=64) in the benchmark's launch
    configuration;
  * the 10,000-frame mixed-code batch at the geometry the tuner picks.

The oracle decodes the large cases with its blocks spread over the host
cores (spawned processes)."""
import numpy as np
import pytest

from paper_1608_00066_gb300 import pbvd, synth, tune

from gpu_util import T_VALUES, batch_oracle_job, gpu_bits, make_decoder, oracle_bits, oracle_bits_parallel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEPTH = {"K7_r1/2": 42, "K7_r3/4": 42, "K9_r1/3": 64}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1608_00066_gb300 import build
    build.build()
    pbvd.load()


def _bits(o, n):
    return np.unpackbits(o.cpu().numpy(), bitorder="little")[:n]


@pytest.mark.parametrize("name", ["K7_r1/2", "K7_r3/4", "K9_r1/3"])
@pytest.mark.parametrize("D", [2048, 4096, 8192])
def test_long_blocks_decode(name, D):
    """Every built T with survivors in the workspace, and the automatic
    configuration (which keeps the survivors of few pairs in shared memory
    when they fit), on three full blocks and a ragged fourth."""
    spec = synth.CODES[name]
    L = DEPTH[name]
    k = 3 * D + 1237
    f = synth.make_frame(spec, k, 1.5, seed=D + len(name))
    want = oracle_bits(spec, f.llr, f.n_stages, D, L)
    dec = make_decoder(spec, D, L)
    for T in T_VALUES[name]:
        got = gpu_bits(dec, f.llr, f.n_stages, threads_per_pair=T, survivors_in_smem=0)
        assert np.array_equal(got, want), (name, D, T)
    got = gpu_bits(dec, f.llr, f.n_stages, threads_per_pair=0, cta_threads=0, survivors_in_smem=-1)
    assert np.array_equal(got, want), (name, D, "auto")
    dec.close()


@pytest.mark.parametrize("D", [2048, 4096, 8192])
def test_long_blocks_batch_and_host(D):
    """Mixed-code batch and the host-memory pipeline at long D."""
    frames = synth.batch_frames(24, seed=4100 + D, k_range=(D // 2, 3 * D))
    decs = {nm: make_decoder(synth.CODES[nm], D, DEPTH[nm]) for nm in DEPTH}
    llrs, outs, items = [], [], []
    for f in frames:
        d = torch.from_numpy(f.llr).cuda()
        o = torch.full(((f.n_stages + 7) // 8,), 0xA5, dtype=torch.uint8, device="cuda")
        llrs.append(d)
        outs.append(o)
        items.append((decs[f.spec.name].ctx, d.data_ptr(), f.n_stages, o.data_ptr()))
    pbvd.pbvd_decode_batch(items)
    torch.cuda.synchronize()
    for f, o in zip(frames, outs):
        want = oracle_bits(f.spec, f.llr, f.n_stages, D, DEPTH[f.spec.name])
        assert np.array_equal(_bits(o, f.n_stages), want), (f.spec.name, f.n_stages, D)
        h_llr = torch.from_numpy(f.llr).pin_memory()
        h_out = torch.zeros((f.n_stages + 7) // 8, dtype=torch.uint8).pin_memory()
        for seg in (0, 3):
            h_out.zero_()
            decs[f.spec.name].decode_host(h_llr, f.n_stages, out=h_out, segments=seg)
            torch.cuda.synchronize()
            got = np.unpackbits(h_out.numpy(), bitorder="little")[:f.n_stages]
            assert np.array_equal(got, want), (f.spec.name, f.n_stages, D, seg)
    for d in decs.values():
        d.close()


@pytest.mark.parametrize("name", ["K7_r1/2", "K7_r3/4", "K9_r1/3"])
@pytest.mark.parametrize("L", [256, 1024, 4096])
def test_long_overlaps(name, L):
    """L far above the decoding depth: forward ranges of D + 2L stages, many
    renormalisations per block, survivor records for D + L stages."""
    spec = synth.CODES[name]
    n_target = 12000 if L == 4096 else 20000
    f = synth.make_frame(spec, n_target - spec.v, 0.5, seed=L + len(name))
    n = f.n_stages
    for D in (64, 512):
        want = oracle_bits_parallel(spec, f.llr, n, D, L)
        dec = make_decoder(spec, D, L)
        Ts = T_VALUES[name] if L < 4096 else T_VALUES[name][:1] + T_VALUES[name][-2:]
        for T in Ts:
            got = gpu_bits(dec, f.llr, n, threads_per_pair=T, survivors_in_smem=0)
            assert np.array_equal(got, want), (name, L, D, T)
        got = gpu_bits(dec, f.llr, n, threads_per_pair=0, cta_threads=0, survivors_in_smem=-1)
        assert np.array_equal(got, want), (name, L, D, "auto")
        dec.close()


@pytest.mark.parametrize("name,ebn0,D,L,seed", [
    ("K7_r1/2", 3.0, 512, 42, 2003),
    ("K7_r3/4", 4.0, 512, 42, 2103),
    ("K9_r1/3", 2.0, 1024, 64, 3001),
])
def test_full_size_stream_every_block(name, ebn0, D, L, seed):
    """2^24 information bits in the benchmark's launch configuration (the
    library's automatic one), every one of the 16,385-32,769 blocks."""
    spec = synth.CODES[name]
    k = 1 << 24
    f = synth.make_frame(spec, k, ebn0, seed=seed)
    n = f.n_stages
    dec = make_decoder(spec, D, L)
    got = gpu_bits(dec, f.llr, n)
    dec.close()
    want = oracle_bits_parallel(spec, f.llr, n, D, L)
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, (name, bad.size, bad[:8].tolist())
    # the punctured rate-3/4 code is the weakest of the three at these Eb/N0
    assert float((got[:k] != f.msg).mean()) < (1e-2 if spec.puncture else 1e-3)


def test_full_batch_at_tuned_geometry():
    """The 10,000-frame batched workload (k ~ U[40, 6144], mixed codes, Eb/N0
    ~ U[1, 5] dB) at the D per code the geometry tuner picks, one persistent
    launch replayed from a CUDA graph: every frame against the oracle."""
    import multiprocessing as mp
    import os
    frames = synth.batch_frames(10000, seed=4001)
    flat = np.concatenate([f.llr for f in frames])
    d_all = torch.from_numpy(flat).cuda()
    sizes = [(f.n_stages + 7) // 8 for f in frames]
    outs = torch.zeros(sum(sizes), dtype=torch.uint8, device="cuda")
    lp, op, off, ooff = [], [], 0, 0
    for f, sz in zip(frames, sizes):
        lp.append(d_all.data_ptr() + off)
        op.append(outs.data_ptr() + ooff)
        off += len(f.llr)
        ooff += sz
    choice, _, _ = tune.tune_batch_geometry(frames, lp, op, candidates=(512, 1024, 2048, 4096), reps=2)
    decs = {nm: pbvd.Decoder(synth.CODES[nm].K, synth.CODES[nm].gens, synth.CODES[nm].puncture, *choice[nm])
            for nm in choice}
    items = tune.make_items(frames, decs, lp, op)
    b = pbvd.pbvd_batch_prepare(items)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        pbvd.pbvd_batch_run(b, s.cuda_stream)
    outs.zero_()
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    host = outs.cpu().numpy()
    pbvd.pbvd_batch_destroy(b)
    procs = os.cpu_count() or 1
    step = (len(frames) + 4 * procs - 1) // (4 * procs)
    jobs = [(a, min(len(frames), a + step), 4001, dict(choice)) for a in range(0, len(frames), step)]
    with mp.get_context("spawn").Pool(procs) as pool:
        results = [r for part in pool.imap_unordered(batch_oracle_job, jobs) for r in part]
    starts = np.concatenate([[0], np.cumsum(sizes)])
    bad = []
    for i, want in results:
        f = frames[i]
        got = np.unpackbits(host[starts[i]:starts[i + 1]], bitorder="little")[:f.n_stages]
        if not np.array_equal(got, want):
            bad.append(i)
    assert len(results) == len(frames)
    assert not bad, (choice, bad[:10])
