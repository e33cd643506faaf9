"""The C-ABI library loads and exports every entry point its headers declare
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(ipc_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def libipc():
    from paper_2502_04093_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_core_calls():
    d = declared()
    for name in ("ipc_compress", "ipc_retrieve", "ipc_refine", "ipc_free", "ipc_selection",
                 "ipc_compressed_size", "ipc_export", "ipc_import"):
        assert name in d


def test_every_declared_symbol_is_exported(libipc):
    missing = [n for n in declared() if not hasattr(libipc, n)]
    assert not missing, missing


def test_last_error_without_gpu(libipc):
    libipc.ipc_last_error.restype = ctypes.c_char_p
    assert libipc.ipc_last_error() is not None
    # argument validation happens before any CUDA call
    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 1)(4)
    rc = libipc.ipc_compress(None, 0, 1, dims, 0, ctypes.c_double(1e-3), 1, 0, None,
                             ctypes.byref(h))
    assert rc == -1
    assert libipc.ipc_free(None) == 0


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2502_04093_gb300.ipc as ipc
    monkeypatch.setattr(ipc, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(ipc, "_lib", None)
    with pytest.raises(ipc.LibraryMissing):
        ipc.lib()


def test_autotune_table_without_gpu(libipc):
    """The shape table's host API: empty after a clear, out-of-range entries
    rejected, and a tuning call with bad arguments refused before any CUDA
    work."""
    assert libipc.ipc_autotune_clear() == 0
    ns = ctypes.c_int(-7)
    assert libipc.ipc_autotune_entry(0, None, None, None, ctypes.byref(ns), None) == -1
    assert libipc.ipc_autotune_entry(-1, None, None, None, None, None) == -1
    assert ns.value == -7  # untouched on failure

    class Target(ctypes.Structure):
        _fields_ = [("kind", ctypes.c_int), ("value", ctypes.c_double)]
    n = ctypes.c_int()
    rc = libipc.ipc_autotune_retrieve(None, Target(0, 1e-3), None, None, 3, ctypes.byref(n))
    assert rc == -1
