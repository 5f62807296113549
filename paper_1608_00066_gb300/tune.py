"""Autotuning of the decoder's free parameters.

Two layers:
  * kernel configuration (threads per pair of blocks = states per lane, CTA
    size, survivor placement): ``pbvd_autotune`` in the C library times every
    built configuration on the caller's data; the decoded bits do not depend
    on it;
  * block geometry for batches: D changes the decoded bits (Sec. III-A: each
    block restarts from zero metrics L stages before it), so the tuner only
    picks D from a candidate set with L held at each code's decoding depth
    (the paper settles on L = 42, about 6K, for K = 7); callers that check
    results must decode their reference with the chosen (D, L).
"""
from __future__ import annotations

import itertools
from typing import Dict, Sequence, Tuple

from . import pbvd

# decoding depth L per code (about 6K, Sec. V)
DEPTH = {"K7_r1/2": 42, "K7_r3/4": 42, "K9_r1/3": 64, "K3_r1/2": 18}
D_CANDIDATES = (512, 1024, 2048, 4096, 8192)


def make_items(frames, decoders, d_llr_ptrs, d_out_ptrs):
    return [(decoders[f.spec.name].ctx, p, f.n_stages, o) for f, p, o in zip(frames, d_llr_ptrs, d_out_ptrs)]


def time_batch(items, reps: int = 5) -> float:
    """Median device time (ms) of one prepared batch launch."""
    import torch
    b = pbvd.pbvd_batch_prepare(items)
    try:
        s = torch.cuda.current_stream()
        pbvd.pbvd_batch_run(b, s.cuda_stream)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            pbvd.pbvd_batch_run(b, s.cuda_stream)
            e1.record(s)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ts.sort()
        return ts[len(ts) // 2]
    finally:
        pbvd.pbvd_batch_destroy(b)


def tune_batch_geometry(frames, d_llr_ptrs: Sequence[int], d_out_ptrs: Sequence[int],
                        candidates: Sequence[int] = D_CANDIDATES, reps: int = 3
                        ) -> Tuple[Dict[str, Tuple[int, int]], float, list]:
    """Chooses D per code (L = DEPTH[code]) minimising the batch decode time.

    Returns ({code: (D, L)}, best ms, [(choice, ms) ...]).  Every candidate
    decodes into d_out_ptrs, so their contents afterwards are those of the last
    candidate tried; decode again with the chosen geometry.
    """
    names = sorted({f.spec.name for f in frames})
    trials = []
    best = None
    for combo in itertools.product(candidates, repeat=len(names)):
        choice = {n: (d, DEPTH[n]) for n, d in zip(names, combo)}
        decs = {n: pbvd.Decoder(frames_spec(frames, n).K, frames_spec(frames, n).gens,
                                frames_spec(frames, n).puncture, *choice[n]) for n in names}
        ms = time_batch(make_items(frames, decs, d_llr_ptrs, d_out_ptrs), reps)
        trials.append((choice, ms))
        if best is None or ms < best[1]:
            best = (choice, ms)
        for d in decs.values():
            d.close()
    return best[0], best[1], trials


def frames_spec(frames, name):
    for f in frames:
        if f.spec.name == name:
            return f.spec
    raise KeyError(name)
