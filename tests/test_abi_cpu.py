"""The C-ABI library builds, loads on a machine without a GPU, and exports
every function that include/ras.h declares (no compute calls)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s*([a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2007_13966_gb300 import build_lib, ras
    if not os.path.exists(ras.LIB_PATH):
        build_lib.build()
    return ras.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("ras_setup", "ras_factor", "ras_apply", "gmres_solve", "residual_eval", "newton_step"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib):
    from paper_2007_13966_gb300 import ras
    assert set(declared_functions()) <= set(ras.EXPORTED)


def test_status_strings_without_gpu(lib):
    assert lib.ras_status_string(0) == b"ok"
    assert b"pivot" in lib.ras_status_string(-5)


def test_noalloc_rejects_out_of_range_sizes_on_the_host(lib):
    """ras_norm2_noalloc refuses n < 0 and n > 2^31 - 1 before any CUDA call
    (its reduction loop has a 64-bit index, so sizes up to the limit cannot
    overflow a stride step); nothing is launched, so this runs without a GPU."""
    import ctypes as C
    from paper_2007_13966_gb300 import ras
    fake = C.c_void_p(0x1000)   # never dereferenced: the size check comes first
    for n in (2 ** 31, 2 ** 40, -1):
        assert lib.ras_norm2_noalloc(fake, C.c_longlong(n), fake, None) == ras.RAS_EINVAL
    assert lib.ras_norm2_noalloc(fake, C.c_longlong(8), None, None) == ras.RAS_EINVAL
