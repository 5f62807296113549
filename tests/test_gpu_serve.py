"""Serving loop on the GPU: every request decoded under continuous batching
(admission by device memory, rotating CUDA streams, arena wrap-around) equals
its decode alone and the block oracle; continuous streams pushed alongside
equal the carried-metric window oracle; under overload every request is
either completed or rejected, and admitted ones were admitted in time."""
import numpy as np
import pytest

import oracle
from paper_1608_00066_gb300 import pbvd, serve, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1608_00066_gb300 import build
    build.build()
    pbvd.load()


def _mother(spec, llr, n):
    if spec.puncture is None:
        return np.asarray(llr, np.int8).reshape(n, spec.R)
    return oracle.depuncture(spec.pattern_array(), llr, n)


def test_serve_outputs_exact():
    pool = serve.build_request_pool(150, seed=5001, k_range=(100, 20000))
    cfg = serve.ServeConfig(arena_bytes=1 << 20, inflight=3, max_batch_bits=150000, max_wait_ms=None)
    srv = serve.Server(pool, cfg)
    arrivals = serve.poisson_arrivals(40000.0, 1.0, seed=5002)[:pool.n]
    assert arrivals.shape[0] == pool.n
    k7 = srv.decoders["K7_r1/2"]
    feeder = serve.StreamFeeder(k7, synth.K7_R12, n_streams=4, chunk=1024, period=3e-4, n_chunks=12, seed=5003)
    res = srv.run(arrivals, feeder)
    assert res["admitted"] == pool.n and res["rejected"] == 0
    assert res["batches"] > 3           # several batches, some in flight together
    assert np.all(srv.status == serve.DONE)
    for j in range(pool.n):
        name = pool.code_names[pool.code[j]]
        spec = synth.CODES[name]
        n = int(pool.n_stages[j])
        got = srv.output_bits(j)
        d = torch.from_numpy(pool.llr[j]).cuda()
        alone = srv.decoders[name].decode(d, n)
        torch.cuda.synchronize()
        alone = np.unpackbits(alone.cpu().numpy(), bitorder="little")[:n]
        assert np.array_equal(got, alone), j
        if j % 10 == 0:
            D, L = cfg.geometry[name]
            ref = oracle.viterbi_block(spec.K, spec.gens, _mother(spec, pool.llr[j], n), D, L)
            assert np.array_equal(got, ref), j
    D, L = k7.D, k7.L
    for s in range(feeder.S):
        ref = oracle.viterbi_window(7, synth.K7_R12.gens, feeder.fed_llr(s).reshape(-1, 2), D, L)
        assert np.array_equal(feeder.bits(s), ref), s
    lat = res["streams"]["latency_us"]
    assert lat["p50"] is not None and lat["p50"] <= lat["p99"]
    feeder.destroy()
    srv.close()


def test_serve_overload_rejects_and_bounds_queueing():
    pool = serve.build_request_pool(64, seed=5004, k_range=(100, 100000))
    max_wait_ms = 2.0
    cfg = serve.ServeConfig(arena_bytes=512 << 10, inflight=2, max_batch_bits=1 << 20, max_wait_ms=max_wait_ms)
    srv = serve.Server(pool, cfg)
    arrivals = serve.poisson_arrivals(1.0e6, 0.004, seed=5005)
    res = srv.run(arrivals)
    st = srv.status
    assert np.all((st == serve.DONE) | (st == serve.REJECTED))
    assert res["rejected"] > 0 and res["admitted"] > 0
    assert res["admitted"] + res["rejected"] == arrivals.shape[0]
    done = st == serve.DONE
    wait = srv.t_admit[done] - arrivals[done]
    assert np.all(wait >= 0)
    assert np.all(wait <= max_wait_ms * 1e-3 + 1e-3)
    assert np.all(srv.t_done[done] >= srv.t_admit[done])
    srv.close()
