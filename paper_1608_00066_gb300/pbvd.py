"""Python binding of the C ABI in include/pbvd.h (argument marshalling only).

Every decoding step runs in the CUDA library ``libpbvd.so`` built in-tree by
``paper_1608_00066_gb300.build``.  There is no CPU fallback: if the library
cannot be loaded, every call raises ``PbvdError``.

The functions keep the C names: ``pbvd_create``, ``pbvd_decode``,
``pbvd_decode_batch``, ``pbvd_destroy`` ...  Device buffers are passed as
integer addresses (e.g. ``tensor.data_ptr()``) and streams as raw
``cudaStream_t`` handles (e.g. ``torch.cuda.current_stream().cuda_stream``).
``Decoder`` wraps a context for use with torch tensors.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpbvd.so")

PBVD_OK = 0
PBVD_EINVAL = -1
PBVD_ENOMEM = -2
PBVD_ECUDA = -3
PBVD_EUNSUPPORTED = -4
PBVD_ETIMEOUT = -5
PBVD_EBUSY = -6

# Exported symbols of include/pbvd.h (checked by the tests).
EXPORTS = (
    "pbvd_create", "pbvd_destroy", "pbvd_decode", "pbvd_llr_count", "pbvd_decode_batch",
    "pbvd_set_config", "pbvd_get_config", "pbvd_strerror", "pbvd_last_cuda_error",
    "pbvd_decode_noalloc", "pbvd_noalloc_max_survivor_bytes",
    "pbvd_batch_prepare", "pbvd_batch_run", "pbvd_batch_destroy", "pbvd_autotune",
    "pbvd_stream_open", "pbvd_stream_push", "pbvd_stream_push_many", "pbvd_stream_close",
    "pbvd_stream_released", "pbvd_stream_destroy", "pbvd_batch_update", "pbvd_decode_host",
    "pbvd_decode_packed", "pbvd_decode_host_packed", "pbvd_set_mode", "pbvd_get_mode",
    "pbvd_decode_two_kernel", "pbvd_decode_packed_pm8", "pbvd_measure_int_rate", "pbvd_stream_metrics",
)

PBVD_MODE_ARGMIN = 1
PBVD_MODE_TAILBITING = 2


class PbvdError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = "%s failed: %s (%d)" % (where, _strerror(code), code)
        if code == PBVD_ECUDA and _lib is not None:
            msg += " [%s]" % _lib.pbvd_last_cuda_error().decode()
        super().__init__(msg)


class pbvd_config(ctypes.Structure):
    _fields_ = [("threads_per_pair", ctypes.c_int), ("cta_threads", ctypes.c_int),
                ("survivors_in_smem", ctypes.c_int)]


class pbvd_batch_item(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("d_llr", ctypes.c_void_p),
                ("n_stages", ctypes.c_size_t), ("d_out", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()


def _strerror(code: int) -> str:
    if _lib is None:
        return "error %d" % code
    return _lib.pbvd_strerror(code).decode()


def load(path: Optional[str] = None):
    """Loads libpbvd.so (raises PbvdError if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise PbvdError(PBVD_EUNSUPPORTED, "load %s (run paper_1608_00066_gb300.build)" % p)
        lib = ctypes.CDLL(p)
        V, I, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        lib.pbvd_create.argtypes = [ctypes.POINTER(V), I, I, V, V, I, I, I]
        lib.pbvd_create.restype = I
        lib.pbvd_destroy.argtypes = [V]
        lib.pbvd_destroy.restype = None
        lib.pbvd_decode.argtypes = [V, V, SZ, V, V]
        lib.pbvd_decode.restype = I
        lib.pbvd_decode_host.argtypes = [V, V, SZ, V, I, V]
        lib.pbvd_decode_host.restype = I
        lib.pbvd_decode_two_kernel.argtypes = [V, V, SZ, V, V]
        lib.pbvd_decode_two_kernel.restype = I
        lib.pbvd_set_mode.argtypes = [V, I]
        lib.pbvd_set_mode.restype = I
        lib.pbvd_get_mode.argtypes = [V, ctypes.POINTER(I)]
        lib.pbvd_get_mode.restype = I
        lib.pbvd_decode_packed.argtypes = [V, V, I, SZ, V, V]
        lib.pbvd_decode_packed.restype = I
        lib.pbvd_decode_packed_pm8.argtypes = [V, V, I, SZ, V, V]
        lib.pbvd_decode_packed_pm8.restype = I
        lib.pbvd_measure_int_rate.argtypes = [I, ctypes.POINTER(ctypes.c_double)]
        lib.pbvd_measure_int_rate.restype = I
        lib.pbvd_decode_host_packed.argtypes = [V, V, I, SZ, V, I, V]
        lib.pbvd_decode_host_packed.restype = I
        lib.pbvd_llr_count.argtypes = [V, SZ, ctypes.POINTER(SZ)]
        lib.pbvd_llr_count.restype = I
        lib.pbvd_decode_batch.argtypes = [V, SZ, V]
        lib.pbvd_decode_batch.restype = I
        lib.pbvd_set_config.argtypes = [V, ctypes.POINTER(pbvd_config)]
        lib.pbvd_set_config.restype = I
        lib.pbvd_get_config.argtypes = [V, SZ, ctypes.POINTER(pbvd_config)]
        lib.pbvd_get_config.restype = I
        lib.pbvd_strerror.argtypes = [I]
        lib.pbvd_strerror.restype = ctypes.c_char_p
        lib.pbvd_last_cuda_error.argtypes = []
        lib.pbvd_last_cuda_error.restype = ctypes.c_char_p
        lib.pbvd_decode_noalloc.argtypes = [V, V, SZ, V, V]
        lib.pbvd_decode_noalloc.restype = I
        lib.pbvd_noalloc_max_survivor_bytes.argtypes = []
        lib.pbvd_noalloc_max_survivor_bytes.restype = SZ
        lib.pbvd_batch_prepare.argtypes = [ctypes.POINTER(V), V, SZ, V]
        lib.pbvd_batch_prepare.restype = I
        lib.pbvd_batch_update.argtypes = [V, V, SZ, I, V]
        lib.pbvd_batch_update.restype = I
        lib.pbvd_batch_run.argtypes = [V, V]
        lib.pbvd_batch_run.restype = I
        lib.pbvd_batch_destroy.argtypes = [V]
        lib.pbvd_batch_destroy.restype = None
        lib.pbvd_autotune.argtypes = [V, V, SZ, V, V, I, ctypes.POINTER(pbvd_config),
                                      ctypes.POINTER(ctypes.c_float)]
        lib.pbvd_autotune.restype = I
        lib.pbvd_stream_open.argtypes = [ctypes.POINTER(V), V, SZ, V, SZ]
        lib.pbvd_stream_open.restype = I
        lib.pbvd_stream_push.argtypes = [V, V, SZ, V]
        lib.pbvd_stream_push.restype = I
        lib.pbvd_stream_push_many.argtypes = [V, V, V, SZ, I, V]
        lib.pbvd_stream_push_many.restype = I
        lib.pbvd_stream_close.argtypes = [V, V]
        lib.pbvd_stream_close.restype = I
        lib.pbvd_stream_released.argtypes = [V]
        lib.pbvd_stream_released.restype = ctypes.c_int64
        lib.pbvd_stream_metrics.argtypes = [V, ctypes.POINTER(ctypes.c_int64), V, V]
        lib.pbvd_stream_metrics.restype = I
        lib.pbvd_stream_destroy.argtypes = [V]
        lib.pbvd_stream_destroy.restype = None
        _lib = lib
        return lib


def _check(rc: int, where: str):
    if rc != PBVD_OK:
        raise PbvdError(rc, where)


# ------------------------------------------------------------ C-named calls

def pbvd_create(K: int, gens: Sequence[int], puncture=None, D: int = 512, L: int = 42) -> int:
    """Returns a context handle (int).  ``puncture`` is an R x P 0/1 nested
    sequence or None."""
    lib = load()
    R = len(gens)
    g = (ctypes.c_uint32 * R)(*gens)
    if puncture is not None:
        rows = [list(r) for r in puncture]
        P = len(rows[0])
        flat = [int(x) for r in rows for x in r]
        pat = (ctypes.c_uint8 * len(flat))(*flat)
        pat_p = ctypes.cast(pat, ctypes.c_void_p)
    else:
        P, pat_p = 0, None
    h = ctypes.c_void_p()
    _check(lib.pbvd_create(ctypes.byref(h), K, R, ctypes.cast(g, ctypes.c_void_p), pat_p, P, D, L),
           "pbvd_create")
    return h.value


def pbvd_destroy(ctx: int) -> None:
    load().pbvd_destroy(ctx)


def pbvd_decode(ctx: int, d_llr: int, n_stages: int, d_out: int, stream: int = 0) -> None:
    _check(load().pbvd_decode(ctx, d_llr, n_stages, d_out, stream or None), "pbvd_decode")


def pbvd_decode_host(ctx: int, h_llr: int, n_stages: int, h_out: int, segments: int = 0, stream: int = 0) -> None:
    """Host-memory decode (host pointers).  segments: 0 = copy pipeline with
    an automatic number of runs of blocks, > 0 = that many runs, -1 = direct
    access by the kernel (both buffers mapped page-locked memory)."""
    _check(load().pbvd_decode_host(ctx, h_llr, n_stages, h_out, segments, stream), "pbvd_decode_host")


def pbvd_decode_two_kernel(ctx: int, d_llr: int, n_stages: int, d_out: int, stream: int = 0) -> None:
    """The paper's two-kernel design (K1 forward, K2 traceback) as an ablation;
    the same bits as pbvd_decode."""
    _check(load().pbvd_decode_two_kernel(ctx, d_llr, n_stages, d_out, stream or None), "pbvd_decode_two_kernel")


def pbvd_set_mode(ctx: int, flags: int) -> None:
    """Decoding variants: PBVD_MODE_ARGMIN | PBVD_MODE_TAILBITING (0 = plain)."""
    _check(load().pbvd_set_mode(ctx, flags), "pbvd_set_mode")


def pbvd_get_mode(ctx: int) -> int:
    f = ctypes.c_int()
    _check(load().pbvd_get_mode(ctx, ctypes.byref(f)), "pbvd_get_mode")
    return int(f.value)


def pbvd_decode_packed(ctx: int, d_words: int, q: int, n_stages: int, d_out: int, stream: int = 0) -> None:
    """Decode of q-bit soft values packed floor(32/q) to a 32-bit word
    (device pointers; q = 1 is hard decision)."""
    _check(load().pbvd_decode_packed(ctx, d_words, q, n_stages, d_out, stream or None), "pbvd_decode_packed")


def pbvd_decode_packed_pm8(ctx: int, d_words: int, q: int, n_stages: int, d_out: int, stream: int = 0) -> None:
    """pbvd_decode_packed with 8-bit path metrics, four blocks per register
    (device pointers; small q only, PBVD_EUNSUPPORTED otherwise)."""
    _check(load().pbvd_decode_packed_pm8(ctx, d_words, q, n_stages, d_out, stream or None),
           "pbvd_decode_packed_pm8")


INT_RATE_OPS = {0: "viaddmnmx_s16x2", 1: "add3", 2: "lop3", 3: "prmt", 4: "imad", 5: "lop3+imad",
                6: "viaddmnmx+imad"}


def pbvd_measure_int_rate(op: int) -> float:
    """Thread-level operations per clock per SM of one instruction kind on the
    current device (see INT_RATE_OPS); a measurement helper."""
    r = ctypes.c_double()
    _check(load().pbvd_measure_int_rate(op, ctypes.byref(r)), "pbvd_measure_int_rate")
    return float(r.value)


def pbvd_decode_host_packed(ctx: int, h_words: int, q: int, n_stages: int, h_out: int, segments: int = 0,
                            stream: int = 0) -> None:
    """pbvd_decode_host with packed q-bit input (host pointers)."""
    _check(load().pbvd_decode_host_packed(ctx, h_words, q, n_stages, h_out, segments, stream or None),
           "pbvd_decode_host_packed")


def pbvd_decode_noalloc(ctx: int, d_llr: int, n_stages: int, d_out: int, stream: int = 0) -> None:
    """pbvd_decode without any device allocation: the survivor bits live in a
    fixed array inside the library (see include/pbvd.h)."""
    _check(load().pbvd_decode_noalloc(ctx, d_llr, n_stages, d_out, stream or None), "pbvd_decode_noalloc")


def pbvd_noalloc_max_survivor_bytes() -> int:
    return int(load().pbvd_noalloc_max_survivor_bytes())


def pbvd_llr_count(ctx: int, n_stages: int) -> int:
    c = ctypes.c_size_t()
    _check(load().pbvd_llr_count(ctx, n_stages, ctypes.byref(c)), "pbvd_llr_count")
    return int(c.value)


def pbvd_decode_batch(items: Sequence[tuple], stream: int = 0) -> None:
    """items: sequence of (ctx, d_llr, n_stages, d_out)."""
    arr = _items(items)
    _check(load().pbvd_decode_batch(ctypes.cast(arr, ctypes.c_void_p), len(items), stream or None),
           "pbvd_decode_batch")


def _items(items):
    arr = (pbvd_batch_item * max(len(items), 1))()
    for i, (ctx, llr, n, out) in enumerate(items):
        arr[i].ctx, arr[i].d_llr, arr[i].n_stages, arr[i].d_out = ctx, llr, n, out
    return arr


def pbvd_batch_update(batch: int, items, reserve_sms: int = 0, stream: int = 0) -> None:
    """Replaces the items of a prepared batch.  ``items`` is a sequence of
    (ctx, d_llr, n_stages, d_out) or a C-contiguous uint64 numpy array of
    shape (n, 4) in that column order (the layout of pbvd_batch_item)."""
    import numpy as np
    if isinstance(items, np.ndarray):
        if items.dtype != np.uint64 or items.ndim != 2 or items.shape[1] != 4 or not items.flags.c_contiguous:
            raise ValueError("items must be a C-contiguous uint64 array of shape (n, 4)")
        ptr, n = items.ctypes.data, items.shape[0]
    else:
        arr = _items(items)
        ptr, n = ctypes.cast(arr, ctypes.c_void_p).value, len(items)
    _check(load().pbvd_batch_update(batch, ptr, n, reserve_sms, stream or None), "pbvd_batch_update")


def pbvd_batch_prepare(items: Sequence[tuple], stream: int = 0) -> int:
    """Builds the work list of items (ctx, d_llr, n_stages, d_out); returns a
    batch handle for pbvd_batch_run / pbvd_batch_destroy."""
    arr = _items(items)
    h = ctypes.c_void_p()
    _check(load().pbvd_batch_prepare(ctypes.byref(h), ctypes.cast(arr, ctypes.c_void_p), len(items),
                                     stream or None), "pbvd_batch_prepare")
    return h.value


def pbvd_batch_run(batch: int, stream: int = 0) -> None:
    _check(load().pbvd_batch_run(batch, stream or None), "pbvd_batch_run")


def pbvd_batch_destroy(batch: int) -> None:
    load().pbvd_batch_destroy(batch)


def pbvd_set_config(ctx: int, threads_per_pair: int = 0, cta_threads: int = 0,
                    survivors_in_smem: int = -1) -> None:
    cfg = pbvd_config(threads_per_pair, cta_threads, survivors_in_smem)
    _check(load().pbvd_set_config(ctx, ctypes.byref(cfg)), "pbvd_set_config")


def pbvd_get_config(ctx: int, n_stages: int) -> dict:
    cfg = pbvd_config()
    _check(load().pbvd_get_config(ctx, n_stages, ctypes.byref(cfg)), "pbvd_get_config")
    return {"threads_per_pair": cfg.threads_per_pair, "cta_threads": cfg.cta_threads,
            "survivors_in_smem": cfg.survivors_in_smem}


def pbvd_autotune(ctx: int, d_llr: int, n_stages: int, d_out: int, stream: int = 0, reps: int = 3):
    """Times the built kernel configurations on this data and keeps the
    fastest in ctx; returns (config dict, milliseconds)."""
    cfg = pbvd_config()
    ms = ctypes.c_float()
    _check(load().pbvd_autotune(ctx, d_llr, n_stages, d_out, stream or None, reps, ctypes.byref(cfg),
                                ctypes.byref(ms)), "pbvd_autotune")
    return ({"threads_per_pair": cfg.threads_per_pair, "cta_threads": cfg.cta_threads,
             "survivors_in_smem": cfg.survivors_in_smem}, float(ms.value))


def pbvd_strerror(code: int) -> str:
    return load().pbvd_strerror(code).decode()


def pbvd_stream_open(ctx: int, max_push: int, d_out: int, out_capacity: int) -> int:
    h = ctypes.c_void_p()
    _check(load().pbvd_stream_open(ctypes.byref(h), ctx, max_push, d_out, out_capacity), "pbvd_stream_open")
    return h.value


def pbvd_stream_push(s: int, d_llr: int, n_stages: int, stream: int = 0) -> None:
    _check(load().pbvd_stream_push(s, d_llr, n_stages, stream), "pbvd_stream_push")


def pbvd_stream_push_many(handles: Sequence[int], d_llrs: Sequence[int], n_stages: Sequence[int],
                          close: bool = False, stream: int = 0) -> None:
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*handles)
    ps = (ctypes.c_void_p * n)(*[p or None for p in d_llrs])
    ns = (ctypes.c_size_t * n)(*n_stages)
    _check(load().pbvd_stream_push_many(hs, ps, ns, n, 1 if close else 0, stream), "pbvd_stream_push_many")


def pbvd_stream_close(s: int, stream: int = 0) -> None:
    _check(load().pbvd_stream_close(s, stream), "pbvd_stream_close")


def pbvd_stream_released(s: int) -> int:
    return int(load().pbvd_stream_released(s))


def pbvd_stream_metrics(s: int, n_states: int, stream: int = 0):
    """(stages decoded, int32 array of the carried path metrics in state
    order) of a stream; waits for the work queued on `stream`."""
    import numpy as np
    out = np.zeros(n_states, dtype=np.int32)
    t = ctypes.c_int64()
    _check(load().pbvd_stream_metrics(s, ctypes.byref(t), out.ctypes.data, stream or None), "pbvd_stream_metrics")
    return int(t.value), out


def pbvd_stream_destroy(s: int) -> None:
    load().pbvd_stream_destroy(s)


# ------------------------------------------------------------- convenience

class Decoder:
    """Owns one context.  ``decode`` takes torch tensors on the GPU."""

    def __init__(self, K: int, gens: Sequence[int], puncture=None, D: int = 512, L: int = 42):
        self.K, self.gens, self.puncture, self.D, self.L = K, tuple(gens), puncture, D, L
        self.ctx = pbvd_create(K, gens, puncture, D, L)

    def close(self):
        if self.ctx:
            pbvd_destroy(self.ctx)
            self.ctx = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def llr_count(self, n_stages: int) -> int:
        return pbvd_llr_count(self.ctx, n_stages)

    def set_config(self, **kw):
        pbvd_set_config(self.ctx, **kw)

    def get_config(self, n_stages: int) -> dict:
        return pbvd_get_config(self.ctx, n_stages)

    def autotune(self, llr, n_stages: int, out=None, reps: int = 3):
        """Tunes the kernel configuration on this input (torch tensors)."""
        import torch
        nbytes = (n_stages + 7) // 8
        if out is None:
            out = torch.empty(nbytes, dtype=torch.uint8, device=llr.device)
        s = torch.cuda.current_stream(llr.device)
        return pbvd_autotune(self.ctx, llr.data_ptr(), n_stages, out.data_ptr(), s.cuda_stream, reps)

    def decode(self, llr, n_stages: int, out=None, stream=None):
        """llr: int8 CUDA tensor of the sent soft values; returns (or fills) a
        uint8 CUDA tensor of ceil(n_stages / 8) packed bytes."""
        import torch
        if llr.dtype != torch.int8 or not llr.is_cuda or not llr.is_contiguous():
            raise ValueError("llr must be a contiguous int8 CUDA tensor")
        if llr.numel() < self.llr_count(n_stages):
            raise ValueError("llr holds %d values, %d needed" % (llr.numel(), self.llr_count(n_stages)))
        nbytes = (n_stages + 7) // 8
        if out is None:
            out = torch.empty(nbytes, dtype=torch.uint8, device=llr.device)
        elif out.numel() < nbytes or out.dtype != torch.uint8 or not out.is_cuda:
            raise ValueError("out must be a uint8 CUDA tensor of %d bytes" % nbytes)
        s = stream if stream is not None else torch.cuda.current_stream(llr.device)
        pbvd_decode(self.ctx, llr.data_ptr(), n_stages, out.data_ptr(), s.cuda_stream)
        return out


    def decode_host(self, llr, n_stages: int, out=None, segments: int = 0, stream=None):
        """llr: int8 CPU tensor of the sent soft values; returns (or fills) a
        uint8 CPU tensor of ceil(n_stages / 8) packed bytes, complete once
        ``stream`` has passed this call.  Page-locked tensors (the default
        ``out`` is one) let the copies overlap the decoding; ``segments`` > 0
        sets the number of runs of blocks, -1 selects direct access by the
        kernel (page-locked tensors only)."""
        import torch
        if llr.dtype != torch.int8 or llr.is_cuda or not llr.is_contiguous():
            raise ValueError("llr must be a contiguous int8 CPU tensor")
        if llr.numel() < self.llr_count(n_stages):
            raise ValueError("llr holds %d values, %d needed" % (llr.numel(), self.llr_count(n_stages)))
        nbytes = (n_stages + 7) // 8
        if out is None:
            out = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
        elif out.numel() < nbytes or out.dtype != torch.uint8 or out.is_cuda or not out.is_contiguous():
            raise ValueError("out must be a contiguous uint8 CPU tensor of %d bytes" % nbytes)
        s = stream if stream is not None else torch.cuda.current_stream()
        pbvd_decode_host(self.ctx, llr.data_ptr(), n_stages, out.data_ptr(), segments, s.cuda_stream)
        return out


    def set_mode(self, argmin: bool = False, tailbiting: bool = False):
        pbvd_set_mode(self.ctx, (PBVD_MODE_ARGMIN if argmin else 0) | (PBVD_MODE_TAILBITING if tailbiting else 0))

    def decode_packed(self, words, q: int, n_stages: int, out=None, stream=None):
        """words: int32 tensor of packed q-bit soft values, on the GPU (device
        decode) or in CPU memory (host pipeline, result in CPU memory)."""
        import torch
        if words.dtype not in (torch.int32, torch.uint32) or not words.is_contiguous():
            raise ValueError("words must be a contiguous 32-bit tensor")
        m = 32 // q
        need = (self.llr_count(n_stages) + m - 1) // m
        if words.numel() < need:
            raise ValueError("words holds %d words, %d needed" % (words.numel(), need))
        nbytes = (n_stages + 7) // 8
        if out is None:
            out = (torch.empty(nbytes, dtype=torch.uint8, device=words.device) if words.is_cuda
                   else torch.empty(nbytes, dtype=torch.uint8).pin_memory())
        if out.numel() < nbytes or out.dtype != torch.uint8 or out.is_cuda != words.is_cuda:
            raise ValueError("out must be a uint8 tensor of %d bytes beside words" % nbytes)
        if words.is_cuda:
            s = stream if stream is not None else torch.cuda.current_stream(words.device)
            pbvd_decode_packed(self.ctx, words.data_ptr(), q, n_stages, out.data_ptr(), s.cuda_stream)
        else:
            s = stream if stream is not None else torch.cuda.current_stream()
            pbvd_decode_host_packed(self.ctx, words.data_ptr(), q, n_stages, out.data_ptr(), 0, s.cuda_stream)
        return out

    def decode_packed_pm8(self, words, q: int, n_stages: int, out=None, stream=None):
        """decode_packed on the GPU with 8-bit path metrics (same bits)."""
        import torch
        if words.dtype not in (torch.int32, torch.uint32) or not words.is_contiguous() or not words.is_cuda:
            raise ValueError("words must be a contiguous 32-bit CUDA tensor")
        m = 32 // q
        need = (self.llr_count(n_stages) + m - 1) // m
        if words.numel() < need:
            raise ValueError("words holds %d words, %d needed" % (words.numel(), need))
        nbytes = (n_stages + 7) // 8
        if out is None:
            out = torch.empty(nbytes, dtype=torch.uint8, device=words.device)
        if out.numel() < nbytes or out.dtype != torch.uint8 or not out.is_cuda:
            raise ValueError("out must be a uint8 CUDA tensor of %d bytes" % nbytes)
        s = stream if stream is not None else torch.cuda.current_stream(words.device)
        pbvd_decode_packed_pm8(self.ctx, words.data_ptr(), q, n_stages, out.data_ptr(), s.cuda_stream)
        return out


class Stream:
    """A continuous stream decoded with carried path metrics (torch tensors).

    ``out`` is a uint8 CUDA tensor of ceil(capacity / 8) bytes that receives
    the decoded bits; ``released`` is the number of leading stages whose bits
    are final once the pushes so far have completed on their CUDA stream."""

    def __init__(self, decoder: Decoder, capacity: int, max_push: int, device=None):
        import torch
        self.decoder = decoder
        self.capacity = capacity
        self.out = torch.zeros((capacity + 7) // 8, dtype=torch.uint8, device=device or "cuda")
        self.handle = pbvd_stream_open(decoder.ctx, max_push, self.out.data_ptr(), capacity)

    @property
    def released(self) -> int:
        return pbvd_stream_released(self.handle)

    def push(self, llr, n_stages: int, stream=None):
        import torch
        if n_stages and (llr.dtype != torch.int8 or not llr.is_cuda or llr.dim() != 1 or not llr.is_contiguous()
                         or llr.numel() < n_stages * len(self.decoder.gens)):
            raise ValueError("llr must be a 1-D contiguous int8 CUDA tensor of R * n_stages values")
        s = stream if stream is not None else torch.cuda.current_stream(self.out.device)
        pbvd_stream_push(self.handle, llr.data_ptr() if n_stages else 0, n_stages, s.cuda_stream)

    def close(self, stream=None):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream(self.out.device)
        pbvd_stream_close(self.handle, s.cuda_stream)

    def metrics(self, stream=None):
        """(stages decoded, carried path metrics in state order)."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream(self.out.device)
        return pbvd_stream_metrics(self.handle, 1 << (self.decoder.K - 1), s.cuda_stream)

    def destroy(self):
        if self.handle:
            pbvd_stream_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
