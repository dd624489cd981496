"""The C-ABI library builds, loads without a GPU and exports every symbol the
public header declares (no compute calls: this file runs on CPU-only hosts)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"EO_API\s+[\w\s\*]+?\b(eo_\w+)\s*\(", text)
    return names


@pytest.fixture(scope="module")
def libeo():
    from paper_1806_01036_gb300 import build
    path = build.build()
    return C.CDLL(path)


def test_header_declares_the_four_operations():
    names = declared_symbols()
    for op in ("eo_gram", "eo_project", "eo_cholqr", "eo_svqb", "eo_create", "eo_destroy", "eo_set_stream",
               "eo_last_error", "eo_version"):
        assert op in names


def test_library_exports_every_declared_symbol(libeo):
    for name in declared_symbols():
        assert hasattr(libeo, name), name


def test_only_declared_symbols_are_exported():
    from paper_1806_01036_gb300 import build
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", build.build()], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l and l.split()[-1].startswith("eo_")}
    assert exported == set(declared_symbols())


def test_null_context_is_rejected_without_touching_a_gpu(libeo):
    libeo.eo_gram.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_int64, C.c_int, C.c_void_p,
                              C.c_int64, C.c_void_p, C.c_void_p, C.c_int, C.c_int]
    assert libeo.eo_gram(None, 10, 2, None, 10, 2, None, 10, None, None, 2, 1) == 1  # EO_EINVAL
    libeo.eo_last_error.restype = C.c_char_p
    libeo.eo_last_error.argtypes = [C.c_void_p]
    assert libeo.eo_last_error(None) == b"null context"
    assert libeo.eo_version() == 1


def test_batch_calls_reject_null_handles_without_touching_a_gpu(libeo):
    libeo.eo_batch_run.argtypes = [C.c_void_p]
    libeo.eo_batch_destroy.argtypes = [C.c_void_p]
    libeo.eo_tune_cache.argtypes = [C.c_void_p, C.c_char_p]
    libeo.eo_batch_kernels.argtypes = [C.c_void_p]
    libeo.eo_batch_kernels.restype = C.c_int64
    libeo.eo_batch_create.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_int,
                                      C.c_void_p, C.c_int, C.c_int, C.c_void_p]
    assert libeo.eo_batch_run(None) == 1
    assert libeo.eo_batch_destroy(None) == 1
    assert libeo.eo_tune_cache(None, b"/nonexistent") == 1
    assert libeo.eo_batch_kernels(None) == -1
    assert libeo.eo_batch_create(None, 1, None, 0, -1.0, 0, 1, None, 0, 0, None) == 1
