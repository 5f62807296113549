"""Runs one decoder kernel on one workload a few times, with a fixed kernel
configuration and no tuning launches before it, so that a profiler can be
pointed at a known launch (skip the warm-up launches, capture the next).

    python -m paper_1608_00066_gb300.prof k7     [--tune JSON] [--warmup W] [--reps N]
    python -m paper_1608_00066_gb300.prof k9     [--tune JSON] ...
    python -m paper_1608_00066_gb300.prof batch  ...
    python -m paper_1608_00066_gb300.prof stream ...
    python -m paper_1608_00066_gb300.prof frame  [--tune JSON] ...
    python -m paper_1608_00066_gb300.prof two    ...
    python -m paper_1608_00066_gb300.prof pm8    [--q Q] [--D D] ...

Workloads (the benchmark's):
  k7     K=7 r1/2 (171,133) terminated stream, 2^24 info bits, 3 dB, D=512 L=42
  k9     K=9 r1/3 (557,663,711) terminated stream, 2^24 info bits, 2 dB, D=1024 L=64
  batch  10,000 mixed-code frames (K7 r1/2, K7 r3/4, K9 r1/3), one persistent launch
  stream 64 continuous K7 r1/2 streams, 4096 stages per push, one launch per push
  frame  one K7 r1/2 frame of 4096 info bits, 3 dB, D=512 L=42 (latency case)
  two    the k7 stream with the paper's two-kernel design (K1 then K2 per call)
  pm8    the k7 stream as packed q-bit words (default q = 3), 8-bit path
         metrics (gather kernel, then one thread per four blocks); D = 512
         unless --D is given

Prints one line per launch set: the workload, the configuration and the mean
device time per launch (CUDA events; L2 not flushed, so do not use it as a
benchmark number).
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import build, pbvd, synth


def _events(torch, fn, warmup: int, reps: int) -> float:
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / max(reps, 1)


def run_stream_decode(torch, spec, k, ebn0, seed, D, L, tune, warmup, reps):
    f = synth.make_frame(spec, k, ebn0, seed=seed)
    dec = pbvd.Decoder(spec.K, spec.gens, spec.puncture, D, L)
    if tune:
        dec.set_config(**tune)
    d_llr = torch.from_numpy(f.llr).cuda()
    d_out = torch.empty((f.n_stages + 7) // 8, dtype=torch.uint8, device="cuda")
    ms = _events(torch, lambda: dec.decode(d_llr, f.n_stages, d_out), warmup, reps)
    cfg = dec.get_config(f.n_stages)
    dec.close()
    return ms, cfg


def run_two_kernel(torch, warmup, reps):
    spec = synth.K7_R12
    f = synth.make_frame(spec, 1 << 24, 3.0, seed=2003)
    dec = pbvd.Decoder(spec.K, spec.gens, None, 512, 42)
    d_llr = torch.from_numpy(f.llr).cuda()
    d_out = torch.empty((f.n_stages + 7) // 8, dtype=torch.uint8, device="cuda")
    ms = _events(torch, lambda: pbvd.pbvd_decode_two_kernel(dec.ctx, d_llr.data_ptr(), f.n_stages, d_out.data_ptr()),
                 warmup, reps)
    dec.close()
    return ms, {"design": "two-kernel (K1 + K2)"}


def run_pm8(torch, q, D, warmup, reps):
    spec = synth.K7_R12
    f = synth.make_packed_frame(spec, 1 << 24, 3.0, q, seed=2003)
    dec = pbvd.Decoder(spec.K, spec.gens, None, D, 42)
    w = torch.from_numpy(f.words.view(np.int32).copy()).cuda()
    out = torch.empty((f.n_stages + 7) // 8, dtype=torch.uint8, device="cuda")
    ms = _events(torch, lambda: dec.decode_packed_pm8(w, q, f.n_stages, out), warmup, reps)
    dec.close()
    return ms, {"q": q, "D": D, "L": 42, "path_metrics": "8-bit, four blocks per register"}


def run_batch(torch, warmup, reps):
    from . import tune as tn
    frames = synth.batch_frames(10000, seed=4001)
    flat = np.concatenate([f.llr for f in frames])
    d_all = torch.from_numpy(flat).cuda()
    outs = torch.zeros(sum((f.n_stages + 7) // 8 for f in frames), dtype=torch.uint8, device="cuda")
    lp, op, off, ooff = [], [], 0, 0
    for f in frames:
        lp.append(d_all.data_ptr() + off)
        op.append(outs.data_ptr() + ooff)
        off += len(f.llr)
        ooff += (f.n_stages + 7) // 8
    geometry = {"K7_r1/2": (1024, 42), "K7_r3/4": (512, 42), "K9_r1/3": (2048, 64)}
    decs = {nm: pbvd.Decoder(synth.CODES[nm].K, synth.CODES[nm].gens, synth.CODES[nm].puncture, *geometry[nm])
            for nm in geometry}
    items = tn.make_items(frames, decs, lp, op)
    b = pbvd.pbvd_batch_prepare(items)
    ms = _events(torch, lambda: pbvd.pbvd_batch_run(b), warmup, reps)
    pbvd.pbvd_batch_destroy(b)
    return ms, {"geometry": geometry}


def run_streams(torch, warmup, reps, n_streams=64, chunk=4096):
    spec = synth.K7_R12
    dec = pbvd.Decoder(spec.K, spec.gens, None, 512, 42)
    pushes = warmup + reps
    cap = pushes * chunk + 64
    rng = np.random.default_rng(5003)
    llr = torch.from_numpy(rng.integers(-127, 128, size=chunk * 2 * n_streams, dtype=np.int8)).cuda()
    streams = [pbvd.Stream(dec, cap, chunk) for _ in range(n_streams)]
    handles = [s.handle for s in streams]
    ptrs = [llr.data_ptr() + i * chunk * 2 for i in range(n_streams)]
    counts = [chunk] * n_streams
    ms = _events(torch, lambda: pbvd.pbvd_stream_push_many(handles, ptrs, counts), warmup, reps)
    for s in streams:
        s.destroy()
    dec.close()
    return ms, {"streams": n_streams, "chunk": chunk}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("target", choices=["k7", "k9", "batch", "stream", "frame", "two", "pm8"])
    ap.add_argument("--tune", default="", help="JSON kernel configuration for k7 / k9")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--q", type=int, default=3, help="bits per soft value (pm8)")
    ap.add_argument("--D", type=int, default=512, help="block length (pm8)")
    args = ap.parse_args(argv)
    import torch
    build.build()
    tune = json.loads(args.tune) if args.tune else None
    if args.target == "k7":
        ms, cfg = run_stream_decode(torch, synth.K7_R12, 1 << 24, 3.0, 2003, 512, 42, tune, args.warmup, args.reps)
    elif args.target == "k9":
        ms, cfg = run_stream_decode(torch, synth.K9_R13, 1 << 24, 2.0, 3001, 1024, 64, tune, args.warmup, args.reps)
    elif args.target == "frame":
        ms, cfg = run_stream_decode(torch, synth.K7_R12, 4096, 3.0, 1001, 512, 42, tune, args.warmup, args.reps)
    elif args.target == "two":
        ms, cfg = run_two_kernel(torch, args.warmup, args.reps)
    elif args.target == "pm8":
        ms, cfg = run_pm8(torch, args.q, args.D, args.warmup, args.reps)
    elif args.target == "batch":
        ms, cfg = run_batch(torch, args.warmup, args.reps)
    else:
        ms, cfg = run_streams(torch, args.warmup, args.reps)
    print(json.dumps({"target": args.target, "config": cfg, "ms_per_launch": round(ms, 4)}))


if __name__ == "__main__":
    main()
