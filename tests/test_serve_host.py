"""Host-side serving logic on the CPU: the arrival process, FIFO admission
under byte / bit / item budgets with expiry, the arena ring and the request
pool layout."""
import math

import numpy as np
import pytest

from paper_1608_00066_gb300 import serve, synth


def test_poisson_arrivals_rate_and_gaps():
    t = serve.poisson_arrivals(20000.0, 2.0, seed=5001)
    assert np.all(np.diff(t) > 0) and t[0] >= 0 and t[-1] < 2.0
    # count within 5 sigma of rate * duration
    assert abs(t.shape[0] - 40000) < 5 * math.sqrt(40000)
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 20000.0) < 0.05 / 20000.0
    # exponential gaps: coefficient of variation 1
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05
    assert np.array_equal(t, serve.poisson_arrivals(20000.0, 2.0, seed=5001))
    assert serve.poisson_arrivals(0.0, 1.0, 1).shape == (0,)


def test_thinning_keeps_fraction():
    t = serve.poisson_arrivals(50000.0, 1.0, seed=1)
    k = serve.thin(t, 0.25, seed=2)
    assert set(k.tolist()) <= set(t.tolist())
    assert abs(k.shape[0] / t.shape[0] - 0.25) < 0.02


def test_log_uniform_k_mean():
    rng = np.random.default_rng(3)
    k = serve.log_uniform_k(rng, 100, 100000, size=200000)
    assert k.min() >= 100 and k.max() <= 100000
    # mean of a log-uniform law on [a, b]: (b - a) / ln(b / a)
    assert abs(k.mean() - (100000 - 100) / math.log(1000)) < 0.02 * 14462


def test_admission_fifo_budgets_and_expiry():
    arr = np.array([0.0, 0.1, 0.2, 0.3, 0.4, 0.5])
    nbytes = np.array([10, 10, 10, 50, 10, 10])
    bits = np.array([5, 5, 5, 5, 100, 5])
    q = serve.AdmissionQueue(arr, nbytes, bits, max_wait=0.25)
    assert q.advance(0.05) == (0, 0)
    assert q.queued() == 1
    assert q.take(100, 100, 10) == (0, 1)
    q.advance(0.25)
    # bytes cap: 10 + 10 fit, bits fine
    assert q.take(20, 100, 10) == (1, 3)
    q.advance(0.45)
    # request 3 needs 50 bytes: the head does not fit, nothing is admitted
    assert q.take(40, 1000, 10) == (3, 3)
    # item cap
    assert q.take(1000, 1000, 1) == (3, 4)
    # request 4 alone exceeds the bit cap but still goes alone
    assert q.take(1000, 50, 10) == (4, 5)
    # request 5 arrives at 0.5 and expires after 0.75
    q.advance(0.8)
    assert q.finished()
    assert q.status.tolist() == [1, 1, 1, 1, 1, 2]


def test_admission_expiry_only_of_arrived():
    arr = np.array([0.0, 0.01, 1.0])
    q = serve.AdmissionQueue(arr, np.ones(3), np.ones(3), max_wait=0.1)
    assert q.advance(0.5) == (0, 2)
    assert q.status.tolist() == [2, 2, 0]
    assert not q.finished()
    assert q.advance(1.05) == (2, 2)
    assert q.take(10, 10, 10) == (2, 3)


@pytest.mark.parametrize("seed", range(5))
def test_ring_arena_never_overlaps(seed):
    rng = np.random.default_rng(seed)
    cap = 4096
    a = serve.RingArena(cap)
    live = []
    for step in range(3000):
        if live and (rng.random() < 0.45 or not a.largest_free()):
            off, n = live.pop(0)
            a.release()
        else:
            n = int(rng.integers(1, 900))
            fits = serve.align_up(n) <= a.largest_free()
            off = a.alloc(n)
            assert (off is not None) == fits
            if off is None:
                continue
            n = serve.align_up(n)
            assert off % serve.ALIGN == 0 and 0 <= off and off + n <= cap
            for o2, n2 in live:
                assert off + n <= o2 or o2 + n2 <= off
            live.append((off, n))
        assert a.used() == sum(n for _, n in live)


def test_ring_arena_wraps():
    a = serve.RingArena(100 * 16)
    offs = [a.alloc(400) for _ in range(4)]
    assert offs == [0, 400, 800, 1200]
    assert a.alloc(16) is None
    a.release()
    a.release()
    assert a.largest_free() == 800
    assert a.alloc(800) == 0
    assert a.alloc(16) is None
    a.release()
    a.release()
    assert a.largest_free() == 800


def test_request_pool_layout():
    p = serve.build_request_pool(12, seed=5001, k_range=(100, 2000))
    assert p.n == 12
    assert np.all(p.in_off % serve.ALIGN == 0) and np.all(p.out_off % serve.ALIGN == 0)
    assert np.all(np.diff(p.in_off) == p.in_len[:-1])
    for j in range(p.n):
        spec = synth.CODES[p.code_names[p.code[j]]]
        assert p.n_stages[j] == p.info_bits[j] + spec.K - 1
        x = p.llr[j]
        assert np.array_equal(p.host_in[p.in_off[j]:p.in_off[j] + x.shape[0]].view(np.int8), x)
        assert p.out_len[j] >= (p.n_stages[j] + 7) // 8
    # reproducible from the seed
    q = serve.build_request_pool(12, seed=5001, k_range=(100, 2000))
    assert np.array_equal(p.host_in, q.host_in)


def test_percentiles():
    r = serve.percentiles_us(np.arange(1, 101) * 1e-6)
    assert r["p50"] == pytest.approx(50.5) and r["p99"] == pytest.approx(99.0)
    assert serve.percentiles_us(np.zeros(0))["p50"] is None
