"""Builds libpbvd.so in-tree with nvcc for sm_103a (GB300).

The translation units are compiled in parallel and linked into one shared
library with the CUDA runtime linked statically, so the library exports only
the C ABI of include/pbvd.h.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpbvd.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC,-fvisibility=hidden",
              "-I" + INCLUDE, "-I" + CSRC]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _deps() + [__file__])


# Headers the run-time compiled kernels need (pbvd_jit.cu embeds them).
JIT_HEADERS = ("pbvd_device.cuh", "pbvd_internal.h", "pbvd_rtc_types.h")


def write_jit_sources() -> str:
    """Writes _build/pbvd_jit_src.inc: the kernel headers as string literals,
    so that the library compiles kernels for new codes without reading any
    file at run time."""
    path = os.path.join(BUILD, "pbvd_jit_src.inc")
    parts = ["// Generated by build.py from csrc/: the headers of run-time compiled kernels.",
             "constexpr int kJitNumHeaders = %d;" % len(JIT_HEADERS),
             "const char* const kJitHeaderNames[] = {%s};" % ", ".join('"%s"' % h for h in JIT_HEADERS),
             "const char* const kJitHeaders[] = {"]
    for h in JIT_HEADERS:
        text = open(os.path.join(CSRC, h)).read()
        if ")PBVDJIT\"" in text:
            raise RuntimeError("%s contains the raw-string delimiter" % h)
        parts.append('R"PBVDJIT(' + text + ')PBVDJIT",')
    parts.append("};")
    data = "\n".join(parts) + "\n"
    if not os.path.exists(path) or open(path).read() != data:
        with open(path, "w") as f:
            f.write(data)
    return path


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    if not force and not extra_flags and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    write_jit_sources()
    cc = nvcc()
    srcs = _sources()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        cmd = [cc] + ARCH + NVCC_FLAGS + ["-I" + BUILD] + list(extra_flags) + ["-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=max(1, min(os.cpu_count() or 1, len(srcs)))) as ex:
        results = list(ex.map(compile_one, srcs))
    if verbose:
        for obj, log in results:
            sys.stderr.write(log)
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = [cc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + [o for o, _ in results] + ["-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
