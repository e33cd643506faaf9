"""Byte-level pins of the oracle's container: an independent pure-Python
restatement (tests/pyref.py) must produce the same bytes on tiny grids, the
plane streams must round-trip losslessly, and damaged containers must be
rejected."""
import numpy as np
import pytest

import pyref
from paper_2502_04093_gb300 import synth

CASES = [((7,), np.float32, "smooth", 1e-2, 1), ((40,), np.float64, "noise", 1e-3, 1),
         ((6, 9), np.float32, "smooth", 1e-4, 1), ((5, 4, 3), np.float32, "spiky", 1e-3, 1),
         ((9, 9), np.float64, "ramp", 1e-5, 0), ((3, 5, 7), np.float32, "noise", 1e-1, 0),
         ((2, 1, 33), np.float32, "smooth", 1e-6, 1), ((1,), np.float32, "smooth", 1e-3, 1),
         ((66,), np.float32, "smooth", 1e-7, 1), ((40,), np.float64, "noise", 1e-3, 2),
         ((6, 9), np.float32, "smooth", 1e-4, 2), ((5, 4, 7), np.float32, "spiky", 1e-3, 2),
         ((17, 3, 11), np.float64, "smooth", 1e-6, 2)]


@pytest.mark.parametrize("shape,dtype,kind,eb,cubic", CASES)
def test_bytes_equal_independent_restatement(oracle, shape, dtype, kind, eb, cubic):
    x = synth.random_field(shape, seed=len(shape) * 13 + int(-np.log10(eb)), dtype=dtype, kind=kind)
    for mode in (oracle.ABS, oracle.REL):
        f = oracle.compress(x, eb, mode, cubic)
        ref, codes = pyref.compress(x, eb, mode, cubic)
        got = f.export()
        assert got == ref
        for t in range(f.info()["S"]):
            assert f.codes(t).tolist() == codes[t]


@pytest.mark.parametrize("shape,dtype,kind,eb,cubic", CASES[:6] + CASES[-3:])
def test_reconstruction_equals_restatement(oracle, shape, dtype, kind, eb, cubic):
    x = synth.random_field(shape, seed=3, dtype=dtype, kind=kind)
    f = oracle.compress(x, eb, oracle.REL, cubic)
    _, codes = pyref.compress(x, eb, oracle.REL, cubic)
    info = f.info()
    K = info["K"]
    st, _ = pyref.stages(shape)
    # outliers as (code index, value) per stage, read back through the oracle
    outl = []
    raw = f.export()
    import struct
    S = info["S"]
    off = 112 + 32 * S + 8 * 32 * S
    for t in range(S):
        no = f.stage(t)["noutliers"]
        ol = []
        for i in range(no):
            ci, v = struct.unpack_from("<Qd", raw, off)
            off += 16
            ol.append((ci, v))
        outl.append(ol)
    rng = np.random.default_rng(1)
    for b in [[0] * K, [32] * K] + [list(rng.integers(0, 33, size=K)) for _ in range(6)]:
        mine = f.reconstruct(b)
        ref = pyref.reconstruct(shape, dtype, codes, outl, float(x.reshape(-1)[0]),
                                info["eb"], b, cubic, info["xmaxabs"])
        assert np.array_equal(mine, ref, equal_nan=True), b


def test_import_export_roundtrip(oracle):
    x = synth.gaussians3d((20, 21, 22), seed=77)
    f = oracle.compress(x, 1e-4, oracle.REL)
    raw = f.export()
    g = oracle.import_bytes(raw, x.shape, x.dtype)
    assert g.export() == raw
    for E in (1e-1, 1e-3, 1e-4):
        a, va = f.retrieve(oracle.EB, E)
        b, vb = g.retrieve(oracle.EB, E)
        assert np.array_equal(a, b) and va.selection() == vb.selection()
    for t in range(f.info()["S"]):
        assert np.array_equal(f.codes(t), g.codes(t))


def test_stream_modes_and_sizes(oracle):
    # a field whose codes are all zero: every stream is the 4-byte empty form
    x = np.zeros((16, 16), dtype=np.float32)
    f = oracle.compress(x, 1e-3)
    for t in range(f.info()["S"]):
        for k in range(32):
            assert f.stream_size(t, k) == 4
    # white noise at a tiny eb fills the low planes densely
    x = synth.random_field((64, 64), seed=4, kind="noise")
    f = oracle.compress(x, 1e-6, oracle.REL)
    t = f.info()["S"] - 1
    st = f.stage(t)
    W = st["ncodes"] // 64 * 2  # 64 codes per row, 2 words per row (2-D last stage)
    sizes = [f.stream_size(t, k) for k in range(32)]
    assert 4 + 4 * W in sizes                  # some dense plane
    assert 4 in sizes                          # some empty high plane


@pytest.mark.parametrize("where", ["magic", "version", "dtype", "truncate", "size", "extra",
                                   "stage", "empty"])
def test_corrupt_containers_rejected(oracle, where):
    x = synth.random_field((10, 12), seed=9)
    raw = bytearray(oracle.compress(x, 1e-3, oracle.REL).export())
    S = oracle.import_bytes(bytes(raw), x.shape, x.dtype).info()["S"]
    if where == "magic":
        raw[0] ^= 0xFF
    elif where == "version":
        raw[4] = 9
    elif where == "dtype":
        raw[8] = 7
    elif where == "truncate":
        raw = raw[:-5]
    elif where == "size":
        off = 112 + 32 * S
        raw[off] ^= 0x04
    elif where == "extra":
        raw += b"\0\0\0\0"
    elif where == "stage":
        raw[112] ^= 0x01  # level of stage 0
    elif where == "empty":
        raw = bytearray()
    assert oracle.import_rc(bytes(raw)) == oracle.ECORRUPT if raw else \
        oracle.import_rc(b"") in (oracle.ECORRUPT, oracle.EINVAL)
