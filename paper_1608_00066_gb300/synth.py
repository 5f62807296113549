"""Seeded synthetic transmitter: the inputs both the decoder and its checks read.

This module is the channel side only.  It draws message bits, encodes them as
polynomial products over GF(2), punctures, maps to BPSK, adds white Gaussian
noise and quantises to int8 soft values.  It contains no decoding arithmetic
(no branch metric, no add-compare-select, no traceback), so the decoder and
the CPU oracle can both read its output without sharing any of the method.

Workload recipe (the paper's experiments use the (2,1,7) CCSDS code over
AWGN with 8-bit soft inputs, Sec. V):
  * message bits ~ Bernoulli(1/2) from ``numpy.random.default_rng(seed)``;
  * zero tail of K-1 bits (frames and streams are terminated);
  * code bit 0 -> +1, 1 -> -1; noise variance sigma^2 = 1 / (2 Rc 10^(EbN0/10))
    with Rc the rate actually sent (after puncturing);
  * soft value = clamp(rint(32 y), -127, 127) as int8, positive favouring 0.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional, Sequence, Tuple

import numpy as np

LLR_SCALE = 32.0


@dataclass(frozen=True)
class CodeSpec:
    """An (R,1,K) convolutional code, optionally punctured.

    ``gens`` are octal-style integers whose bit K-1 is the tap on the new input
    bit and bit 0 the tap on the oldest memory cell.  ``puncture`` is an R x P
    0/1 pattern: code bit r of stage s is sent iff ``puncture[r][s % P]``.
    """

    name: str
    K: int
    gens: Tuple[int, ...]
    puncture: Optional[Tuple[Tuple[int, ...], ...]] = None

    @property
    def R(self) -> int:
        return len(self.gens)

    @property
    def v(self) -> int:
        return self.K - 1

    @property
    def rate(self) -> float:
        """Information bits per sent code bit."""
        if self.puncture is None:
            return 1.0 / self.R
        P = len(self.puncture[0])
        return P / float(sum(sum(row) for row in self.puncture))

    def pattern_array(self) -> Optional[np.ndarray]:
        if self.puncture is None:
            return None
        return np.asarray(self.puncture, dtype=np.uint8)

    def sent_per_stage_prefix(self, n_stages: int) -> int:
        """Number of soft values sent for the first n_stages stages."""
        if self.puncture is None:
            return n_stages * self.R
        pat = self.pattern_array()
        P = pat.shape[1]
        per_col = pat.sum(axis=0)
        full, rem = divmod(n_stages, P)
        return int(full * per_col.sum() + per_col[:rem].sum())


K7_R12 = CodeSpec("K7_r1/2", 7, (0o171, 0o133))
K7_R34 = CodeSpec("K7_r3/4", 7, (0o171, 0o133), ((1, 1, 0), (1, 0, 1)))
K9_R13 = CodeSpec("K9_r1/3", 9, (0o557, 0o663, 0o711))
K3_R12 = CodeSpec("K3_r1/2", 3, (0o7, 0o5))
CODES = {c.name: c for c in (K7_R12, K7_R34, K9_R13, K3_R12)}


def taps(g: int, K: int) -> np.ndarray:
    """Impulse response h[i] = g_{K-1-i}: h[0] multiplies the newest input."""
    return np.array([(g >> (K - 1 - i)) & 1 for i in range(K)], dtype=np.uint8)


def conv_encode(spec: CodeSpec, msg: np.ndarray) -> np.ndarray:
    """Zero-terminated encoding as c^(r)(D) = m(D) g^(r)(D) over GF(2).

    Returns an (n, R) uint8 array with n = len(msg) + K - 1.
    """
    m = np.concatenate([np.asarray(msg, dtype=np.uint8),
                        np.zeros(spec.v, dtype=np.uint8)])
    n = len(m)
    out = np.empty((n, spec.R), dtype=np.uint8)
    for r, g in enumerate(spec.gens):
        out[:, r] = (np.convolve(m.astype(np.int32), taps(g, spec.K).astype(np.int32))[:n] & 1)
    return out


def conv_encode_tailbiting(spec: CodeSpec, msg: np.ndarray) -> np.ndarray:
    """Tail-biting encoding as a circular convolution over GF(2): code bit r
    of stage s is sum_i h_i m[(s - i) mod k] (the encoder starts in the state
    its last K-1 message bits leave it in, and ends there).  (k, R) uint8."""
    m = np.asarray(msg, dtype=np.int64)
    k = len(m)
    out = np.zeros((k, spec.R), dtype=np.uint8)
    for r, g in enumerate(spec.gens):
        h = taps(g, spec.K).astype(np.int64)
        acc = np.zeros(k, dtype=np.int64)
        for i in range(spec.K):
            if h[i]:
                acc ^= np.roll(m, i)
        out[:, r] = acc & 1
    return out


def puncture_bits(spec: CodeSpec, coded: np.ndarray) -> np.ndarray:
    """(n, R) code bits -> 1-D sent bits in stage-major, r-ascending order."""
    if spec.puncture is None:
        return np.ascontiguousarray(coded).reshape(-1)
    pat = spec.pattern_array()
    P = pat.shape[1]
    n = coded.shape[0]
    keep = pat.T[np.arange(n) % P].astype(bool)  # (n, R)
    return np.ascontiguousarray(coded[keep])


def noise_sigma(ebn0_db: float, rate: float) -> float:
    return float(np.sqrt(1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0))))


def bpsk_awgn_int8(rng: np.random.Generator, bits: np.ndarray, ebn0_db: float,
                   rate: float) -> np.ndarray:
    """BPSK over AWGN, quantised to int8 soft values (positive favours 0)."""
    s = 1.0 - 2.0 * bits.astype(np.float64)
    y = s + noise_sigma(ebn0_db, rate) * rng.standard_normal(len(bits))
    return np.clip(np.rint(LLR_SCALE * y), -127, 127).astype(np.int8)


def quantise_q(y: np.ndarray, q: int) -> np.ndarray:
    """q-bit soft values of channel outputs y (Sec. IV-C): for q >= 2,
    clamp(rint(2^(q-2) y), -Q, Q) with Q = 2^(q-1) - 1 (steps of 1/2^(q-2)
    of the BPSK amplitude); for q = 1 (hard decision) -1 where y < 0, else +1."""
    if q == 1:
        return np.where(y < 0, -1, 1).astype(np.int8)
    Q = (1 << (q - 1)) - 1
    return np.clip(np.rint(float(1 << (q - 2)) * y), -Q, Q).astype(np.int8)


def pack_q(values: np.ndarray, q: int) -> np.ndarray:
    """Packs q-bit values floor(32/q) to a uint32 word (Sec. IV-C): value i
    at bits [q (i mod m), q (i mod m) + q) of word i // m, two's complement;
    for q = 1 the bit is 1 for a negative value (code bit 1)."""
    v = np.asarray(values, dtype=np.int64)
    m = 32 // q
    if q == 1:
        codes = (v < 0).astype(np.uint64)
    else:
        codes = (v & ((1 << q) - 1)).astype(np.uint64)
    nw = (len(v) + m - 1) // m
    padded = np.zeros(nw * m, dtype=np.uint64)
    padded[:len(v)] = codes
    shifts = (np.arange(m, dtype=np.uint64) * np.uint64(q))
    words = (padded.reshape(nw, m) << shifts).sum(axis=1, dtype=np.uint64)
    return words.astype(np.uint32)


@dataclass
class PackedFrame:
    spec: CodeSpec
    msg: np.ndarray         # uint8[k]
    q: int                  # bits per soft value (1 = hard decision)
    values: np.ndarray      # int8 q-bit soft values, stage major (n * R)
    words: np.ndarray       # uint32, floor(32/q) values per word
    n_stages: int


def make_packed_frame(spec: CodeSpec, k: int, ebn0_db: float, q: int, seed) -> PackedFrame:
    """A terminated frame quantised to q bits per sent soft value and packed
    (punctured codes: the sent values only)."""
    rng = np.random.default_rng(seed)
    msg = rng.integers(0, 2, size=k, dtype=np.uint8)
    bits = puncture_bits(spec, conv_encode(spec, msg))
    s = 1.0 - 2.0 * bits.astype(np.float64)
    y = s + noise_sigma(ebn0_db, spec.rate) * rng.standard_normal(len(bits))
    vals = quantise_q(y, q)
    return PackedFrame(spec, msg, q, vals, pack_q(vals, q), k + spec.v)


def noiseless_int8(bits: np.ndarray) -> np.ndarray:
    """Error-free soft values: +127 for 0, -127 for 1."""
    return (127 - 254 * bits.astype(np.int16)).astype(np.int8)


@dataclass
class Frame:
    spec: CodeSpec
    msg: np.ndarray         # uint8[k]
    llr: np.ndarray         # int8, sent soft values (punctured if the code is)
    n_stages: int           # k + K - 1
    ebn0_db: float


def make_frame(spec: CodeSpec, k: int, ebn0_db: Optional[float], seed) -> Frame:
    """A terminated frame of k random message bits; ``ebn0_db=None`` gives
    error-free soft values."""
    rng = np.random.default_rng(seed)
    msg = rng.integers(0, 2, size=k, dtype=np.uint8)
    coded = conv_encode(spec, msg)
    sent = puncture_bits(spec, coded)
    if ebn0_db is None:
        llr = noiseless_int8(sent)
    else:
        llr = bpsk_awgn_int8(rng, sent, ebn0_db, spec.rate)
    return Frame(spec, msg, llr, k + spec.v, float("inf") if ebn0_db is None else ebn0_db)


def make_tailbiting_frame(spec: CodeSpec, k: int, ebn0_db: Optional[float], seed) -> Frame:
    """A tail-biting frame of k random message bits (k stages, no tail);
    ``ebn0_db=None`` gives error-free soft values.  Unpunctured codes only."""
    if spec.puncture is not None:
        raise ValueError("tail-biting frames are built for unpunctured codes")
    rng = np.random.default_rng(seed)
    msg = rng.integers(0, 2, size=k, dtype=np.uint8)
    sent = conv_encode_tailbiting(spec, msg).reshape(-1)
    if ebn0_db is None:
        llr = noiseless_int8(sent)
    else:
        llr = bpsk_awgn_int8(rng, sent, ebn0_db, spec.rate)
    return Frame(spec, msg, llr, k, float("inf") if ebn0_db is None else ebn0_db)


def batch_frame(f: int, seed: int, k_range=(40, 6144), ebn0_range=(1.0, 5.0),
                codes: Sequence[CodeSpec] = (K7_R12, K7_R34, K9_R13)) -> Frame:
    """Frame f of a mixed-code batch: info length ~ U{k_lo..k_hi}, code uniform
    over ``codes``, Eb/N0 ~ U[lo, hi] dB, all drawn from SeedSequence([seed, f])."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, f]))
    k = int(rng.integers(k_range[0], k_range[1] + 1))
    spec = codes[int(rng.integers(0, len(codes)))]
    eb = float(rng.uniform(ebn0_range[0], ebn0_range[1]))
    sub = int(rng.integers(0, 2 ** 63 - 1))
    return make_frame(spec, k, eb, sub)


def batch_frames(n_frames: int, seed: int, k_range=(40, 6144), ebn0_range=(1.0, 5.0),
                 codes: Sequence[CodeSpec] = (K7_R12, K7_R34, K9_R13)):
    """Mixed-code batch of n_frames frames (see batch_frame)."""
    return [batch_frame(f, seed, k_range, ebn0_range, codes) for f in range(n_frames)]
