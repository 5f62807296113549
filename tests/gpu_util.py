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
