"""Plain CPU oracle for the parallel block-based Viterbi decoder.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the decoder library
and its Python binding never do.  The arithmetic lives in ``pbvd_oracle.c``
(plain C, 64-bit path metrics); this module only builds it with gcc and
marshals numpy arrays.  It shares no code with the CUDA path.

Conventions (from the paper, Sec. III-B and Table 2):
  * state d = (D_{v-1} ... D_0)_2, v = K - 1, N = 2^v states;
  * generator integers hold g_m in bit m, the leftmost octal digit is g_{K-1};
  * codewords are integers with c^(1) as the most significant bit;
  * LLRs are int8, positive favours code bit 0, -128 is read as -127.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pbvd_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

BIG = 8192


def build(force: bool = False) -> str:
    """Compile ``pbvd_oracle.c`` into ``_liboracle.so`` (gcc, -O2)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                           "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I = ctypes.c_int
        I64 = ctypes.c_int64
        U32 = ctypes.c_uint32
        sigs = {
            "orc_codeword": (U32, [I, I, P, U32, I]),
            "orc_next_state": (U32, [I, U32, I]),
            "orc_output_table": (None, [I, I, P, P]),
            "orc_encode": (I64, [I, I, P, P, I64, P]),
            "orc_puncture": (I64, [I, P, I, P, I64, P]),
            "orc_depuncture": (I64, [I, P, I, P, I64, P]),
            "orc_branch_metric": (I64, [I, P, U32]),
            "orc_acs_stage": (None, [I, I, P, P, P, P, P]),
            "orc_viterbi_full": (I, [I, I, P, P, I64, P, P, P, P]),
            "orc_block_geometry": (None, [I64, I64, I64, I64, P, P, P, P]),
            "orc_viterbi_block_range": (I, [I, I, P, P, I64, I64, I64, I64, I64, P]),
            "orc_viterbi_block": (I, [I, I, P, P, I64, I64, I64, P]),
            "orc_viterbi_block_metrics": (I, [I, I, P, P, I64, I64, I64, I64, I64, P, P]),
            "orc_viterbi_block_variant": (I, [I, I, P, P, I64, I64, I64, I64, I64, I, P, P]),
            "orc_encode_tailbiting": (I64, [I, I, P, P, I64, P]),
            "orc_unpack_soft": (I, [I, P, I64, P]),
            "orc_branch_metric_q": (I64, [I, P, U32, I]),
            "orc_acs_stage_q": (None, [I, I, P, P, I, P, P, P]),
            "orc_viterbi_block_q": (I, [I, I, P, P, I64, I64, I64, I, P]),
            "orc_viterbi_window": (I, [I, I, P, P, I64, I64, I64, P]),
            "orc_brute_force": (I, [I, I, P, P, I, P, P, P]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _gens(gens) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(gens, dtype=np.uint32))


def _i8(llr) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(llr, dtype=np.int8))


def codeword(K: int, gens, d: int, x: int) -> int:
    """c(S_d, x) of Eq. (2) as an R-bit integer, c^(1) most significant."""
    g = _gens(gens)
    return int(_load().orc_codeword(K, len(g), _ptr(g), d, x))


def next_state(K: int, d: int, x: int) -> int:
    return int(_load().orc_next_state(K, d, x))


def output_table(K: int, gens) -> np.ndarray:
    """table[d, x] = c(S_d, x) for all states."""
    g = _gens(gens)
    N = 1 << (K - 1)
    t = np.zeros(N * 2, dtype=np.uint32)
    _load().orc_output_table(K, len(g), _ptr(g), _ptr(t))
    return t.reshape(N, 2)


def encode(K: int, gens, msg) -> np.ndarray:
    """Zero-terminated encoding; returns an (n, R) uint8 array, n = k + K - 1."""
    g = _gens(gens)
    m = np.ascontiguousarray(np.asarray(msg, dtype=np.uint8))
    R = len(g)
    n = len(m) + K - 1
    out = np.zeros(n * R, dtype=np.uint8)
    _load().orc_encode(K, R, _ptr(g), _ptr(m), len(m), _ptr(out))
    return out.reshape(n, R)


def puncture(pattern, bits) -> np.ndarray:
    """Keeps code bit r of stage s iff pattern[r, s % P]; bits is (n, R)."""
    pat = np.ascontiguousarray(np.asarray(pattern, dtype=np.uint8))
    R, P = pat.shape
    b = np.ascontiguousarray(np.asarray(bits, dtype=np.uint8))
    n = b.shape[0]
    out = np.zeros(n * R, dtype=np.uint8)
    k = _load().orc_puncture(R, _ptr(pat), P, _ptr(b), n, _ptr(out))
    return out[:k].copy()


def depuncture(pattern, llr_tx, n: int) -> np.ndarray:
    """Soft values of the sent positions -> (n, R) int8 with zeros elsewhere."""
    pat = np.ascontiguousarray(np.asarray(pattern, dtype=np.uint8))
    R, P = pat.shape
    tx = _i8(llr_tx)
    out = np.zeros(n * R, dtype=np.int8)
    used = _load().orc_depuncture(R, _ptr(pat), P, _ptr(tx), n, _ptr(out))
    if used != len(tx):
        raise ValueError("depuncture consumed %d of %d soft values" % (used, len(tx)))
    return out.reshape(n, R)


def branch_metric(lam, c: int) -> int:
    l = _i8(lam)
    return int(_load().orc_branch_metric(len(l), _ptr(l), c))


def acs_stage(K: int, gens, lam, pm_prev):
    """One stage of Eq. (1); returns (pm_next int64[N], dec uint8[N])."""
    g = _gens(gens)
    l = _i8(lam)
    N = 1 << (K - 1)
    pp = np.ascontiguousarray(np.asarray(pm_prev, dtype=np.int64))
    pn = np.zeros(N, dtype=np.int64)
    dec = np.zeros(N, dtype=np.uint8)
    _load().orc_acs_stage(K, len(g), _ptr(g), _ptr(l), _ptr(pp), _ptr(pn), _ptr(dec))
    return pn, dec


def viterbi_full(K: int, gens, llr, want_trace: bool = False):
    """Full-frame VA on (n, R) mother-code soft values.

    Returns bits (uint8[n]) and final metrics (int64[N]); with want_trace also
    survivor bits (uint8[n, N]) and metrics after every stage (int64[n, N]).
    """
    g = _gens(gens)
    R = len(g)
    l = _i8(llr).reshape(-1)
    n = len(l) // R
    N = 1 << (K - 1)
    out = np.zeros(n, dtype=np.uint8)
    fpm = np.zeros(N, dtype=np.int64)
    dec = np.zeros(n * N, dtype=np.uint8) if want_trace else None
    tr = np.zeros(n * N, dtype=np.int64) if want_trace else None
    rc = _load().orc_viterbi_full(K, R, _ptr(g), _ptr(l), n, _ptr(out), _ptr(fpm),
                                  _ptr(dec) if want_trace else None,
                                  _ptr(tr) if want_trace else None)
    if rc != 0:
        raise MemoryError("orc_viterbi_full failed")
    if want_trace:
        return out, fpm, dec.reshape(n, N), tr.reshape(n, N)
    return out, fpm


def block_geometry(n: int, D: int, L: int, b: int):
    """(f0, f1, o0, o1) of block b."""
    v = [ctypes.c_int64() for _ in range(4)]
    _load().orc_block_geometry(n, D, L, b, *[ctypes.byref(x) for x in v])
    return tuple(int(x.value) for x in v)


def viterbi_block(K: int, gens, llr, D: int, L: int, blocks=None) -> np.ndarray:
    """Block-based VA on (n, R) mother-code soft values; uint8[n] bits.

    With ``blocks=(b0, b1)`` only blocks b0..b1-1 are decoded and the other
    entries of the result stay 0.
    """
    g = _gens(gens)
    R = len(g)
    l = _i8(llr).reshape(-1)
    n = len(l) // R
    out = np.zeros(n, dtype=np.uint8)
    if blocks is None:
        rc = _load().orc_viterbi_block(K, R, _ptr(g), _ptr(l), n, D, L, _ptr(out))
    else:
        rc = _load().orc_viterbi_block_range(K, R, _ptr(g), _ptr(l), n, D, L,
                                             blocks[0], blocks[1], _ptr(out))
    if rc != 0:
        raise ValueError("orc_viterbi_block failed (D=%d, L=%d)" % (D, L))
    return out


def viterbi_block_metrics(K: int, gens, llr, D: int, L: int, blocks):
    """Blocks b0..b1-1 of the block-based VA: (bits uint8[n], pm_end int64[b1-b0]).

    pm_end[i] is PM(S_0) after the last forward stage of block b0 + i, the
    metric of the path its traceback follows."""
    g = _gens(gens)
    R = len(g)
    l = _i8(llr).reshape(-1)
    n = len(l) // R
    out = np.zeros(n, dtype=np.uint8)
    b0, b1 = blocks
    pm = np.zeros(max(b1 - b0, 1), dtype=np.int64)
    rc = _load().orc_viterbi_block_metrics(K, R, _ptr(g), _ptr(l), n, D, L, b0, b1,
                                           _ptr(out), _ptr(pm))
    if rc != 0:
        raise ValueError("orc_viterbi_block_metrics failed (D=%d, L=%d)" % (D, L))
    return out, pm[:b1 - b0].copy()


TB_ARGMIN = 1
CIRCULAR = 2


def viterbi_block_variant(K: int, gens, llr, D: int, L: int, argmin: bool = False,
                          circular: bool = False, blocks=None):
    """Block form with the argmin traceback start (Sec. II's S_E) and/or
    circular (tail-biting) windows; returns (bits uint8[n], pm_end int64[])."""
    g = _gens(gens)
    R = len(g)
    l = _i8(llr).reshape(-1)
    n = len(l) // R
    nb = (n + D - 1) // D
    b0, b1 = blocks if blocks is not None else (0, nb)
    out = np.zeros(n, dtype=np.uint8)
    pm = np.zeros(max(b1 - b0, 1), dtype=np.int64)
    flags = (TB_ARGMIN if argmin else 0) | (CIRCULAR if circular else 0)
    rc = _load().orc_viterbi_block_variant(K, R, _ptr(g), _ptr(l), n, D, L, b0, b1, flags,
                                           _ptr(out), _ptr(pm))
    if rc != 0:
        raise ValueError("orc_viterbi_block_variant failed (D=%d, L=%d)" % (D, L))
    return out, pm[:b1 - b0].copy()


def encode_tailbiting(K: int, gens, msg) -> np.ndarray:
    """Tail-biting encoding (start state = end state); (k, R) uint8, k >= K-1."""
    g = _gens(gens)
    m = np.ascontiguousarray(np.asarray(msg, dtype=np.uint8))
    R = len(g)
    out = np.zeros(len(m) * R, dtype=np.uint8)
    if _load().orc_encode_tailbiting(K, R, _ptr(g), _ptr(m), len(m), _ptr(out)) < 0:
        raise ValueError("tail-biting frames need k >= K - 1")
    return out.reshape(len(m), R)


def q_max(q: int) -> int:
    """Largest magnitude Q of a q-bit soft value (1 for hard decisions)."""
    return 1 if q == 1 else (1 << (q - 1)) - 1


def unpack_soft(q: int, words, count: int) -> np.ndarray:
    """Sec. IV-C packing: count q-bit soft values from uint32 words."""
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint32))
    out = np.zeros(max(count, 1), dtype=np.int8)
    if _load().orc_unpack_soft(q, _ptr(w), count, _ptr(out)) != 0:
        raise ValueError("q must be 1..8")
    return out[:count].copy()


def branch_metric_q(lam, c: int, Q: int) -> int:
    l = _i8(lam)
    return int(_load().orc_branch_metric_q(len(l), _ptr(l), c, Q))


def acs_stage_q(K: int, gens, lam, Q: int, pm_prev):
    g = _gens(gens)
    l = _i8(lam)
    N = 1 << (K - 1)
    pp = np.ascontiguousarray(np.asarray(pm_prev, dtype=np.int64))
    pn = np.zeros(N, dtype=np.int64)
    dec = np.zeros(N, dtype=np.uint8)
    _load().orc_acs_stage_q(K, len(g), _ptr(g), _ptr(l), Q, _ptr(pp), _ptr(pn), _ptr(dec))
    return pn, dec


def viterbi_block_q(K: int, gens, llr_q, D: int, L: int, Q: int) -> np.ndarray:
    """Block form on unpacked q-bit values (n, R) with mu = +-Q."""
    g = _gens(gens)
    R = len(g)
    l = _i8(llr_q).reshape(-1)
    n = len(l) // R
    out = np.zeros(n, dtype=np.uint8)
    if _load().orc_viterbi_block_q(K, R, _ptr(g), _ptr(l), n, D, L, Q, _ptr(out)) != 0:
        raise ValueError("orc_viterbi_block_q failed")
    return out


def viterbi_window(K: int, gens, llr, D: int, L: int) -> np.ndarray:
    """Carried-metric stream form (see pbvd_oracle.c); uint8[n] bits."""
    g = _gens(gens)
    R = len(g)
    l = _i8(llr).reshape(-1)
    n = len(l) // R
    out = np.zeros(n, dtype=np.uint8)
    rc = _load().orc_viterbi_window(K, R, _ptr(g), _ptr(l), n, D, L, _ptr(out))
    if rc != 0:
        raise ValueError("orc_viterbi_window failed")
    return out


def brute_force(K: int, gens, llr, k: int):
    """ML over all 2^k messages: (first best message, best metric, #best)."""
    g = _gens(gens)
    R = len(g)
    l = _i8(llr).reshape(-1)
    if len(l) != (k + K - 1) * R:
        raise ValueError("llr length does not match k")
    msg = np.zeros(max(k, 1), dtype=np.uint8)
    bm = ctypes.c_int64()
    nb = ctypes.c_int64()
    rc = _load().orc_brute_force(K, R, _ptr(g), _ptr(l), k, _ptr(msg),
                                 ctypes.byref(bm), ctypes.byref(nb))
    if rc != 0:
        raise ValueError("brute force supports k <= 24")
    return msg[:k].copy(), int(bm.value), int(nb.value)


def pack_bits(bits) -> np.ndarray:
    """Bit s -> byte s >> 3, bit s & 7 (LSB first), as the decoder writes."""
    return np.packbits(np.asarray(bits, dtype=np.uint8), bitorder="little")
