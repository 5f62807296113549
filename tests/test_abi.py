"""CPU-side checks of the C-ABI library: it builds, loads, exports every
symbol include/*.h declares, and rejects bad arguments before touching the
GPU.  No decoding runs here."""
import ctypes
import glob
import os
import re

import pytest

from paper_1608_00066_gb300 import build as pbuild
from paper_1608_00066_gb300 import pbvd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pbuild.build()
    return pbvd.load()


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names += re.findall(r"PBVD_API\s+[\w\s\*]*?\b(pbvd_\w+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "pbvd_create" in names and "pbvd_decode_batch" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(pbvd.EXPORTS)


def test_strerror(lib):
    assert pbvd.pbvd_strerror(0) == "ok"
    assert "invalid" in pbvd.pbvd_strerror(pbvd.PBVD_EINVAL)


@pytest.mark.parametrize("K,gens,punct,D,L", [
    (2, (3, 1), None, 512, 42),            # K too small
    (10, (0o1171, 0o1133), None, 512, 42), # K too large
    (7, (0o171,), None, 512, 42),          # R = 1
    (7, (0o171, 0o533), None, 512, 42),    # generator wider than K
    (7, (0o171, 0o076), None, 512, 42),    # neither end tap set
    (7, (0o171, 0o133), None, 500, 42),    # D not a multiple of 8
    (7, (0o171, 0o133), None, 0, 42),      # D = 0
    (7, (0o171, 0o133), None, 512, -1),    # L < 0
    (7, (0o171, 0o133), ((1, 0), (0, 0)), 512, 42),  # a column sends nothing
    (7, (0o171, 0o133), ((1, 2), (1, 1)), 512, 42),  # pattern entry not 0/1
])
def test_create_rejects_bad_arguments(lib, K, gens, punct, D, L):
    with pytest.raises(pbvd.PbvdError) as ei:
        pbvd.pbvd_create(K, gens, punct, D, L)
    assert ei.value.code == pbvd.PBVD_EINVAL


def _nvrtc_loadable():
    for name in ("libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13"):
        try:
            ctypes.CDLL(name)
            return True
        except OSError:
            pass
    return False


def test_code_without_built_in_kernels_passes_the_code_checks(lib):
    """A valid code the library has no compiled kernel for is compiled at run
    time, so pbvd_create accepts it (with libnvrtc present) and goes on to the
    device; without a GPU that last step is what fails."""
    with pytest.raises(pbvd.PbvdError) as ei:
        ctx = pbvd.pbvd_create(7, (0o171, 0o165), None, 512, 42)
        pbvd.pbvd_destroy(ctx)
        raise pbvd.PbvdError(pbvd.PBVD_OK, "pbvd_create succeeded")
    assert ei.value.code != pbvd.PBVD_EINVAL
    if _nvrtc_loadable():
        assert ei.value.code != pbvd.PBVD_EUNSUPPORTED


def test_null_arguments(lib):
    assert lib.pbvd_create(None, 7, 2, None, None, 0, 512, 42) == pbvd.PBVD_EINVAL
    assert lib.pbvd_decode(None, None, 0, None, None) == pbvd.PBVD_EINVAL
    assert lib.pbvd_decode_batch(None, 1, None) == pbvd.PBVD_EINVAL
    lib.pbvd_destroy(None)
