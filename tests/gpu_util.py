"""Helpers shared by the GPU tests: run the CUDA decoder through the C ABI on
seeded synthetic inputs and compute the oracle's answer for the same bytes."""
import numpy as np

import oracle
from paper_1608_00066_gb300 import pbvd, synth

# (code, T values built for it)
T_VALUES = {
    "K3_r1/2": (1, 2),
    "K7_r1/2": (1, 2, 4, 8, 16, 32),
    "K7_r3/4": (1, 2, 4, 8, 16, 32),
    "K9_r1/3": (4, 8, 16, 32),
}


def make_decoder(spec, D, L):
    return pbvd.Decoder(spec.K, spec.gens, spec.puncture, D, L)


def mother_llr(spec, frame_llr, n):
    if spec.puncture is None:
        return np.asarray(frame_llr, np.int8).reshape(n, spec.R)
    return oracle.depuncture(spec.pattern_array(), frame_llr, n)


def gpu_bits(dec, llr, n, **cfg):
    import torch
    if cfg:
        dec.set_config(**cfg)
    d = torch.from_numpy(np.ascontiguousarray(llr)).cuda()
    out = dec.decode(d, n)
    torch.cuda.synchronize()
    return np.unpackbits(out.cpu().numpy(), bitorder="little")[:n]


def oracle_bits(spec, frame_llr, n, D, L, blocks=None):
    return oracle.viterbi_block(spec.K, spec.gens, mother_llr(spec, frame_llr, n), D, L, blocks)


def _oracle_range(args):
    """Child process: blocks [b0, b1) of a stream saved as an (n, R) .npy."""
    path, K, gens, D, L, b0, b1 = args
    llr = np.load(path, mmap_mode="r")
    n = llr.shape[0]
    out = oracle.viterbi_block(K, gens, np.ascontiguousarray(llr), D, L, blocks=(b0, b1))
    return b0, out[b0 * D:min(b1 * D, n)].copy()


def oracle_bits_parallel(spec, frame_llr, n, D, L, procs=None):
    """Every block of the stream with the CPU oracle, the blocks spread over
    the host cores (spawned processes, so no forked copy of a CUDA context)."""
    import multiprocessing as mp
    import os
    import tempfile
    mother = np.ascontiguousarray(mother_llr(spec, frame_llr, n))
    nb = (n + D - 1) // D
    procs = procs or os.cpu_count() or 1
    chunk = max(1, (nb + 4 * procs - 1) // (4 * procs))
    tmp = tempfile.NamedTemporaryFile(suffix=".npy", delete=False)
    tmp.close()
    try:
        np.save(tmp.name, mother)
        jobs = [(tmp.name, spec.K, tuple(spec.gens), D, L, b, min(nb, b + chunk)) for b in range(0, nb, chunk)]
        out = np.zeros(n, dtype=np.uint8)
        with mp.get_context("spawn").Pool(procs) as pool:
            for b0, bits in pool.imap_unordered(_oracle_range, jobs):
                out[b0 * D:b0 * D + len(bits)] = bits
        return out
    finally:
        os.unlink(tmp.name)


def batch_oracle_job(args):
    """Child process: oracle bits of frames [f_lo, f_hi) of the mixed-code
    batch drawn with the given seed, each at its code's (D, L)."""
    f_lo, f_hi, seed, geometry = args
    out = []
    for i in range(f_lo, f_hi):
        f = synth.batch_frame(i, seed)
        D, L = geometry[f.spec.name]
        out.append((i, oracle_bits(f.spec, f.llr, f.n_stages, D, L)))
    return out
