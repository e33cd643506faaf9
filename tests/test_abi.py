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


def test_autotune_table_save_and_restore(tmp_path):
    """The shape table round-trips through a file (host only): the shapes
    the tuner can record are accepted and listed back in key order, others
    are refused, and a restored table equals the saved one."""
    from paper_2502_04093_gb300 import build, ipc
    build.build()
    ipc.ipc_autotune_clear()
    good = [(0, 1, (257, 257, 129), 2, 4), (0, 0, (129, 129, 65), 4, 4),
            (1, 0, (513, 513, 513), 1, 3), (1, 1, (65, 65, 33), 0, 0)]
    for d, w, M, ns, ps in good:
        ipc.ipc_autotune_set(d, w, M, ns, ps)
    ipc.ipc_autotune_set(0, 1, (257, 257, 129), 1, 2)  # same key: replaced
    want = sorted([(0, 1, (257, 257, 129), 1, 2)] + good[1:])
    assert ipc.ipc_autotune_entries() == want
    bad = [(2, 0, (9, 9, 9), 1, 1),       # element type
           (0, 2, (9, 9, 9), 1, 1),       # code width
           (0, 0, (0, 9, 9), 1, 1),       # extents
           (0, 0, (9, 9, 300), 2, 1),     # two planes need rows of at most 256
           (0, 0, (9, 9, 200), 4, 1),     # four need at most 128
           (0, 0, (9, 9, 9), 3, 1),       # planes per tile
           (1, 0, (9, 9, 9), 1, 4),       # f64, 32-bit codes: at most 3 per SM
           (0, 0, (9, 9, 9), 1, 0),       # a tuned shape has CTAs per SM
           (0, 0, (9, 9, 9), 0, 2)]
    for d, w, M, ns, ps in bad:
        with pytest.raises(ipc.IpcError) as e:
            ipc.ipc_autotune_set(d, w, M, ns, ps)
        assert e.value.rc == ipc.IPC_EINVAL
    assert ipc.ipc_autotune_entries() == want
    p = str(tmp_path / "shapes.json")
    assert ipc.ipc_autotune_save(p) == 4
    ipc.ipc_autotune_clear()
    assert ipc.ipc_autotune_entries() == []
    assert ipc.ipc_autotune_load(p) == 4
    assert ipc.ipc_autotune_entries() == want
    ipc.ipc_autotune_clear()
