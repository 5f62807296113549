"""Serving loop: continuous batching of frame requests and continuous streams
on one GPU.

Frame requests arrive as a Poisson process, each a frame of one of the codes
(k information bits, log-uniform).  The server admits them in arrival order
into a device arena (a byte ring of fixed size: admission by device memory),
copies the admitted requests' soft values host -> device, decodes them in one
persistent batched launch (every frame decoded exactly as it would be alone,
Sec. III-A geometry), copies the packed bits back and completes the requests
when that copy has finished.  Iterations run on rotating CUDA streams, so the
copies of one batch overlap the decoding of another.  A request that waited
longer than ``max_wait_ms`` without being admitted is rejected.

Alongside, S continuous streams deliver a chunk of soft values every period;
the chunks that are due are pushed to all streams in one launch on a
high-priority CUDA stream, with each stream's path metrics kept on the device
between pushes.

The host-side pieces (arrival process, FIFO admission with a byte budget,
the arena ring, latency statistics) are plain Python/numpy and are tested on
the CPU; ``Server`` drives the GPU through the C ABI.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import pbvd, synth

ALIGN = 16


def align_up(x, a: int = ALIGN):
    return (x + a - 1) // a * a


# ------------------------------------------------------------- workload ----

def poisson_arrivals(rate: float, duration: float, seed: int) -> np.ndarray:
    """Arrival times (s, increasing) of a Poisson process of ``rate`` per
    second over [0, duration)."""
    if rate <= 0 or duration <= 0:
        return np.zeros(0)
    rng = np.random.default_rng(seed)
    mean = rate * duration
    n = int(mean + 10 * math.sqrt(mean) + 16)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    while t[-1] < duration:
        t = np.concatenate([t, t[-1] + np.cumsum(rng.exponential(1.0 / rate, size=n))])
    return t[t < duration]


def thin(arrivals: np.ndarray, keep: float, seed: int) -> np.ndarray:
    """Independent thinning: keeps each arrival with probability ``keep``
    (a Poisson process of rate keep * rate)."""
    rng = np.random.default_rng(seed)
    return arrivals[rng.random(arrivals.shape[0]) < keep]


def log_uniform_k(rng, lo: int, hi: int, size=None):
    return np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=size))).astype(np.int64)


@dataclasses.dataclass
class RequestPool:
    """Frames that requests draw from (request i uses entry i mod n), with
    their soft values packed into one host buffer at 16-byte aligned offsets."""
    code_names: List[str]
    code: np.ndarray        # code index per entry
    n_stages: np.ndarray
    info_bits: np.ndarray
    in_off: np.ndarray      # byte offset in host_in
    in_len: np.ndarray      # aligned byte length
    out_off: np.ndarray     # byte offset in the host output buffer
    out_len: np.ndarray     # aligned byte length of the packed bits
    host_in: np.ndarray     # uint8
    llr: list               # per entry int8 soft values (for checks)

    @property
    def n(self) -> int:
        return int(self.code.shape[0])

    @property
    def in_bytes(self) -> int:
        return int(self.in_off[-1] + self.in_len[-1])

    @property
    def out_bytes(self) -> int:
        return int(self.out_off[-1] + self.out_len[-1])


def build_request_pool(n: int, seed: int, k_range=(100, 100000), ebn0_range=(1.0, 5.0),
                       codes: Sequence[synth.CodeSpec] = (synth.K7_R12, synth.K7_R34, synth.K9_R13)
                       ) -> RequestPool:
    names = [c.name for c in codes]
    code = np.zeros(n, np.int64)
    n_stages = np.zeros(n, np.int64)
    info = np.zeros(n, np.int64)
    llrs = []
    for j in range(n):
        rng = np.random.default_rng(np.random.SeedSequence([seed, j]))
        ci = int(rng.integers(len(codes)))
        k = int(log_uniform_k(rng, *k_range))
        eb = float(rng.uniform(*ebn0_range))
        f = synth.make_frame(codes[ci], k, eb, seed=np.random.SeedSequence([seed, j, 1]))
        code[j], n_stages[j], info[j] = ci, f.n_stages, k
        llrs.append(f.llr)
    in_len = align_up(np.array([x.shape[0] for x in llrs], np.int64))
    out_len = align_up((n_stages + 7) // 8)
    in_off = np.concatenate([[0], np.cumsum(in_len)[:-1]]).astype(np.int64)
    out_off = np.concatenate([[0], np.cumsum(out_len)[:-1]]).astype(np.int64)
    host_in = np.zeros(int(in_off[-1] + in_len[-1]), np.uint8)
    for j, x in enumerate(llrs):
        host_in[in_off[j]:in_off[j] + x.shape[0]] = x.view(np.uint8)
    return RequestPool(names, code, n_stages, info, in_off, in_len, out_off, out_len, host_in, llrs)


# ------------------------------------------------------------ admission ----

PENDING, ADMITTED, REJECTED, DONE = 0, 1, 2, 3


class AdmissionQueue:
    """Requests in arrival order.  A request becomes visible at its arrival
    time; the head of the queue is admitted in runs that fit a byte budget, a
    bit cap and an item cap; a request that waited longer than ``max_wait``
    seconds without being admitted is rejected."""

    def __init__(self, arrival: np.ndarray, nbytes: np.ndarray, bits: np.ndarray,
                 max_wait: Optional[float] = None):
        self.arrival = np.asarray(arrival, np.float64)
        self.nbytes = np.asarray(nbytes, np.int64)
        self.bits = np.asarray(bits, np.int64)
        self.max_wait = max_wait
        self.status = np.zeros(self.arrival.shape[0], np.int8)
        self.head = 0          # first request not yet admitted or rejected
        self.visible = 0       # requests that have arrived

    @property
    def n(self) -> int:
        return int(self.arrival.shape[0])

    def queued(self) -> int:
        return self.visible - self.head

    def finished(self) -> bool:
        return self.head >= self.n

    def advance(self, now: float):
        """Makes arrivals up to ``now`` visible and rejects expired requests;
        returns the range of rejected requests."""
        self.visible = int(np.searchsorted(self.arrival, now, side="right"))
        r0 = self.head
        if self.max_wait is not None and self.head < self.visible:
            # requests that arrived before now - max_wait
            cut = int(np.searchsorted(self.arrival, now - self.max_wait, side="left"))
            cut = min(cut, self.visible)
            if cut > self.head:
                self.status[self.head:cut] = REJECTED
                self.head = cut
        return r0, self.head

    def take(self, max_bytes: int, max_bits: int, max_items: int):
        """Admits the longest run from the head whose bytes, bits and count
        fit; returns (i0, i1) (empty when the head does not fit)."""
        i0 = self.head
        i1 = min(self.visible, i0 + max_items)
        if i1 <= i0:
            return i0, i0
        cb = np.cumsum(self.nbytes[i0:i1])
        cbits = np.cumsum(self.bits[i0:i1])
        m = int(min(np.searchsorted(cb, max_bytes, side="right"), np.searchsorted(cbits, max_bits, side="right")))
        if m == 0 and cbits[0] > max_bits and cb[0] <= max_bytes:
            m = 1              # a single request larger than the bit cap still goes alone
        self.status[i0:i0 + m] = ADMITTED
        self.head = i0 + m
        return i0, i0 + m


class RingArena:
    """Byte ring over a device buffer: contiguous allocations at the free end,
    released in allocation order."""

    def __init__(self, capacity: int):
        self.capacity = int(capacity)
        self.live = collections.deque()   # (offset, size) in allocation order

    def used(self) -> int:
        return sum(s for _, s in self.live)

    def largest_free(self) -> int:
        if not self.live:
            return self.capacity
        s0 = self.live[0][0]
        o, s = self.live[-1]
        e = o + s
        if o < s0:             # wrapped: the free space lies between the ends
            return s0 - e
        return max(self.capacity - e, s0)

    def alloc(self, n: int) -> Optional[int]:
        n = int(align_up(n))
        if n <= 0 or n > self.capacity:
            return None
        if not self.live:
            off = 0
        else:
            s0 = self.live[0][0]
            o, s = self.live[-1]
            e = o + s
            wrapped = o < s0
            if wrapped:
                if n > s0 - e:
                    return None
                off = e
            elif n <= self.capacity - e:
                off = e
            elif n <= s0:
                off = 0
            else:
                return None
        self.live.append((off, n))
        return off

    def release(self):
        self.live.popleft()


def percentiles_us(x: np.ndarray) -> Dict[str, float]:
    if x.size == 0:
        return {"p50": None, "p99": None, "mean": None, "max": None}
    x = x * 1e6
    return {"p50": round(float(np.percentile(x, 50)), 1), "p99": round(float(np.percentile(x, 99)), 1),
            "mean": round(float(x.mean()), 1), "max": round(float(x.max()), 1)}


# ---------------------------------------------------------------- server ---

@dataclasses.dataclass
class ServeConfig:
    arena_bytes: int = 256 << 20       # device memory for admitted requests
    inflight: int = 3                  # batches in flight (CUDA streams)
    max_batch_bits: int = 16 << 20     # information bits per batch
    max_batch_items: int = 4096
    max_wait_ms: Optional[float] = 50.0
    reserve_sms: int = 0               # SMs the batch grid leaves to stream pushes
    geometry: Dict[str, tuple] = dataclasses.field(default_factory=lambda: {
        "K7_r1/2": (512, 42), "K7_r3/4": (512, 42), "K9_r1/3": (1024, 64)})
    # threads per pair of blocks per K, selecting the batch kernel's dense shape
    dense_threads: Dict[int, int] = dataclasses.field(default_factory=lambda: {7: 2, 9: 8})


class _Slot:
    def __init__(self, torch):
        self.stream = torch.cuda.Stream()
        self.event = torch.cuda.Event()
        self.batch = 0
        self.rng = (0, 0)
        self.done = False
        self.t_done = 0.0


class StreamFeeder:
    """S continuous streams of one code, each receiving a chunk of ``chunk``
    stages every ``period`` seconds; the chunks due are pushed to all streams
    in one launch on a high-priority CUDA stream.  Chunk c of stream s is the
    soft values pool[c mod pool_chunks, s]."""

    def __init__(self, decoder: "pbvd.Decoder", spec: synth.CodeSpec, n_streams: int, chunk: int, period: float,
                 n_chunks: int, seed: int, pool_chunks: int = 8, ebn0_db: float = 3.0):
        import torch
        self.torch = torch
        self.spec, self.S, self.chunk, self.period, self.n_chunks = spec, n_streams, chunk, period, n_chunks
        R = spec.R
        self.pool_chunks = min(pool_chunks, n_chunks)
        host = np.zeros((self.pool_chunks, n_streams, chunk * R), np.int8)
        for s in range(n_streams):
            f = synth.make_frame(spec, self.pool_chunks * chunk - spec.K + 1, ebn0_db,
                                 seed=np.random.SeedSequence([seed, 7, s]))
            host[:, s, :] = f.llr.reshape(self.pool_chunks, chunk * R)
        self.host = torch.from_numpy(host).pin_memory()
        self.stage = torch.empty((n_streams, chunk * R), dtype=torch.int8, device="cuda")
        self.streams = [pbvd.Stream(decoder, n_chunks * chunk, chunk) for _ in range(n_streams)]
        self.handles = [st.handle for st in self.streams]
        self.stage_ptrs = [self.stage[s].data_ptr() for s in range(n_streams)]
        self.cuda_stream = torch.cuda.Stream(priority=-1)
        self.inflight = collections.deque()     # (event, chunk index)
        self.next_chunk = 0
        self.arrive = np.arange(n_chunks) * period
        self.done_t = np.full(n_chunks, np.nan)
        self.closed = False

    def fed_llr(self, s: int) -> np.ndarray:
        """Soft values pushed to stream s (R per stage)."""
        h = self.host.numpy()
        return np.concatenate([h[c % self.pool_chunks, s] for c in range(self.n_chunks)])

    def poll(self, now: float, clock):
        torch = self.torch
        while self.inflight and self.inflight[0][0].query():
            _, c = self.inflight.popleft()
            self.done_t[c] = clock()
        while self.next_chunk < self.n_chunks and self.arrive[self.next_chunk] <= now:
            c = self.next_chunk
            with torch.cuda.stream(self.cuda_stream):
                self.stage.copy_(self.host[c % self.pool_chunks], non_blocking=True)
                pbvd.pbvd_stream_push_many(self.handles, self.stage_ptrs, [self.chunk] * self.S, close=False,
                                           stream=self.cuda_stream.cuda_stream)
                ev = torch.cuda.Event()
                ev.record(self.cuda_stream)
            self.inflight.append((ev, c))
            self.next_chunk += 1

    def finished(self) -> bool:
        return self.next_chunk >= self.n_chunks and not self.inflight

    def close(self):
        if not self.closed:
            pbvd.pbvd_stream_push_many(self.handles, [0] * self.S, [0] * self.S, close=True,
                                       stream=self.cuda_stream.cuda_stream)
            self.cuda_stream.synchronize()
            self.closed = True

    def bits(self, s: int) -> np.ndarray:
        n = self.n_chunks * self.chunk
        return np.unpackbits(self.streams[s].out.cpu().numpy(), bitorder="little")[:n]

    def destroy(self):
        for st in self.streams:
            st.destroy()


class Server:
    """Continuous-batching decode server on the current CUDA device."""

    def __init__(self, pool: RequestPool, cfg: ServeConfig = ServeConfig()):
        import torch
        self.torch = torch
        self.pool, self.cfg = pool, cfg
        specs = {c.name: c for c in (synth.K7_R12, synth.K7_R34, synth.K9_R13, synth.K3_R12)}
        self.decoders = {}
        for name in pool.code_names:
            s = specs[name]
            self.decoders[name] = pbvd.Decoder(s.K, s.gens, s.puncture, *cfg.geometry[name])
            # the dense shape of the mixed-code batch kernel (two threads per
            # pair for K=7, eight for K=9): several long-frame batches in
            # flight fill the GPU between them
            self.decoders[name].set_config(threads_per_pair=cfg.dense_threads[s.K])
        self.ctx_of_code = np.array([self.decoders[nm].ctx for nm in pool.code_names], np.uint64)
        self.host_in = torch.from_numpy(pool.host_in).pin_memory()
        self.host_out = torch.zeros(pool.out_bytes, dtype=torch.uint8).pin_memory()
        self.arena = torch.empty(cfg.arena_bytes, dtype=torch.uint8, device="cuda")
        self.arena_ptr = self.arena.data_ptr()
        self.slots = [_Slot(torch) for _ in range(cfg.inflight)]
        self._reserve()

    def _reserve(self):
        """Sizes every slot's batch buffers for the largest batch the limits
        allow, so that no device allocation happens while serving."""
        p = self.pool
        order = np.argsort(-p.info_bits)
        sel, bits, nbytes = [], 0, 0
        for j in order:
            if len(sel) >= self.cfg.max_batch_items or bits + p.info_bits[j] > 2 * self.cfg.max_batch_bits:
                continue
            sel.append(int(j))
            bits += int(p.info_bits[j])
        items = [(int(self.ctx_of_code[p.code[j]]), self.arena_ptr, int(p.n_stages[j]), self.arena_ptr)
                 for j in sel]
        for sl in self.slots:
            sl.batch = pbvd.pbvd_batch_prepare(items, sl.stream.cuda_stream)
        self.torch.cuda.synchronize()

    def close(self):
        for sl in self.slots:
            if sl.batch:
                pbvd.pbvd_batch_destroy(sl.batch)
                sl.batch = 0
        for d in self.decoders.values():
            d.close()

    def _runs(self, entries: np.ndarray):
        """Splits pool entries into runs that are consecutive in the pool."""
        brk = np.nonzero(np.diff(entries) != 1)[0] + 1
        return np.split(np.arange(entries.shape[0]), brk)

    def _launch(self, sl: _Slot, i0: int, i1: int, off: int):
        torch, p = self.torch, self.pool
        e = np.arange(i0, i1) % p.n
        in_len, out_len = p.in_len[e], p.out_len[e]
        a_in = off + np.concatenate([[0], np.cumsum(in_len)[:-1]])
        in_total = int(in_len.sum())
        a_out = off + in_total + np.concatenate([[0], np.cumsum(out_len)[:-1]])
        items = np.empty((i1 - i0, 4), np.uint64)
        items[:, 0] = self.ctx_of_code[p.code[e]]
        items[:, 1] = self.arena_ptr + a_in
        items[:, 2] = p.n_stages[e]
        items[:, 3] = self.arena_ptr + a_out
        runs = self._runs(e)
        with torch.cuda.stream(sl.stream):
            for r in runs:
                j0, j1 = e[r[0]], e[r[-1]]
                h0, h1 = int(p.in_off[j0]), int(p.in_off[j1] + p.in_len[j1])
                d0 = int(a_in[r[0]])
                self.arena[d0:d0 + h1 - h0].copy_(self.host_in[h0:h1], non_blocking=True)
            pbvd.pbvd_batch_update(sl.batch, items, self.cfg.reserve_sms, sl.stream.cuda_stream)
            pbvd.pbvd_batch_run(sl.batch, sl.stream.cuda_stream)
            for r in runs:
                j0, j1 = e[r[0]], e[r[-1]]
                h0, h1 = int(p.out_off[j0]), int(p.out_off[j1] + p.out_len[j1])
                d0 = int(a_out[r[0]])
                self.host_out[h0:h1].copy_(self.arena[d0:d0 + h1 - h0], non_blocking=True)
            sl.event.record(sl.stream)
        sl.rng = (i0, i1)
        sl.done = False

    def run(self, arrivals: np.ndarray, feeder: Optional[StreamFeeder] = None, time_limit: float = 60.0) -> dict:
        """Serves requests arriving at ``arrivals`` (s from start; request i
        uses pool entry i mod n) and, if given, the feeder's streams; returns
        the statistics."""
        torch, p, cfg = self.torch, self.pool, self.cfg
        n = arrivals.shape[0]
        e_all = np.arange(n) % p.n
        need = p.in_len[e_all] + p.out_len[e_all]
        q = AdmissionQueue(arrivals, need, p.info_bits[e_all],
                           None if cfg.max_wait_ms is None else cfg.max_wait_ms * 1e-3)
        arena = RingArena(cfg.arena_bytes)
        t_admit = np.full(n, np.nan)
        t_done = np.full(n, np.nan)
        free = collections.deque(self.slots)
        busy = collections.deque()
        batches, batch_items = 0, 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()

        def clock():
            return time.perf_counter() - t0

        while True:
            now = clock()
            # completions (space is released in allocation order)
            for sl in busy:
                if not sl.done and sl.event.query():
                    sl.done, sl.t_done = True, clock()
            while busy and busy[0].done:
                sl = busy.popleft()
                t_done[sl.rng[0]:sl.rng[1]] = sl.t_done
                arena.release()
                free.append(sl)
            if feeder is not None:
                feeder.poll(now, clock)
            q.advance(now)
            if free and q.queued():
                i0, i1 = q.take(arena.largest_free(), cfg.max_batch_bits, cfg.max_batch_items)
                if i1 > i0:
                    off = arena.alloc(int(need[i0:i1].sum()))
                    assert off is not None
                    sl = free.popleft()
                    t_admit[i0:i1] = clock()
                    self._launch(sl, i0, i1, off)
                    busy.append(sl)
                    batches += 1
                    batch_items += i1 - i0
            if q.finished() and not busy and (feeder is None or feeder.finished()):
                break
            if now > time_limit:
                raise RuntimeError("serving run exceeded its time limit")
        elapsed = clock()
        done = q.status == ADMITTED
        q.status[done] = DONE
        info = p.info_bits[e_all]
        first = float(arrivals[0]) if n else 0.0
        span = float(np.nanmax(t_done) - first) if done.any() else 0.0
        res = {
            "requests": int(n),
            "admitted": int(done.sum()),
            "rejected": int((q.status == REJECTED).sum()),
            "offered_rate_fps": round(n / float(arrivals[-1]), 1) if n > 1 else None,
            "offered_gbps": round(float(info.sum()) / float(arrivals[-1]) / 1e9, 3) if n > 1 else None,
            "admitted_gbps": round(float(info[done].sum()) / span / 1e9, 3) if span > 0 else None,
            "latency_us": percentiles_us(t_done[done] - arrivals[done]),
            "queue_us": percentiles_us(t_admit[done] - arrivals[done]),
            "service_us": percentiles_us(t_done[done] - t_admit[done]),
            "batches": batches,
            "mean_batch_frames": round(batch_items / batches, 1) if batches else 0,
            "elapsed_s": round(elapsed, 4),
        }
        if feeder is not None:
            feeder.close()
            lat = feeder.done_t - feeder.arrive
            res["streams"] = {
                "n": feeder.S, "code": feeder.spec.name, "chunk_stages": feeder.chunk,
                "period_us": round(feeder.period * 1e6, 1),
                "gbps": round(feeder.S * feeder.chunk * feeder.n_chunks / max(np.nanmax(feeder.done_t), 1e-9) / 1e9,
                              3),
                "latency_us": percentiles_us(lat[~np.isnan(lat)]),
            }
        self.t_admit, self.t_done, self.status = t_admit, t_done, q.status
        return res

    def output_bits(self, j: int) -> np.ndarray:
        """Decoded bits of pool entry j (from the host output buffer)."""
        p = self.pool
        o = int(p.out_off[j])
        b = self.host_out[o:o + int((p.n_stages[j] + 7) // 8)].numpy()
        return np.unpackbits(b, bitorder="little")[:int(p.n_stages[j])]
