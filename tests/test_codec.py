"""The lossless stage (the entropy coder after predictive coding, Sec. 6.2.1;
this build's rANS in place of the paper's zstd), on the CPU: the library's
coder against the plain-Python restatement in oracle/rans_oracle.py (same
bytes both ways), the defining identity decode(encode(x)) == x, the order-0
entropy bound every such coder approaches, and rejection of corrupt input."""
import math

import numpy as np
import pytest

from oracle import oracle
from oracle import rans_oracle as ro
from paper_2502_04093_gb300 import ipc, synth


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2502_04093_gb300 import build
    build.build()
    oracle.build()


def inputs():
    rng = np.random.default_rng(11)
    yield "empty", b""
    yield "one byte", b"\x07"
    yield "one symbol, 3 blocks", b"\x00" * 9000
    yield "uniform", rng.integers(0, 256, 5000, dtype=np.uint8).tobytes()
    yield "geometric", rng.geometric(0.2, 12000).clip(0, 255).astype(np.uint8).tobytes()
    yield "two symbols", rng.choice([3, 250], 7000, p=[0.99, 0.01]).astype(np.uint8).tobytes()
    yield "all 256 + tail", bytes(range(256)) * 3 + b"\x01" * 5000
    yield "block boundary", rng.geometric(0.5, 8192).astype(np.uint8).tobytes()
    # odd block lengths: the last symbol of a coded block falls to state 0 alone
    yield "odd last block", rng.geometric(0.3, 4096 + 1001).clip(0, 255).astype(np.uint8).tobytes()
    yield "odd short block", rng.geometric(0.6, 4096 + 1023).clip(0, 255).astype(np.uint8).tobytes()


@pytest.mark.parametrize("name,raw", list(inputs()), ids=[n for n, _ in inputs()])
def test_library_equals_oracle_bytes(name, raw):
    lib = ipc.ipc_encode_container(raw, block_log2=12)
    assert lib == ro.encode(raw, block_log2=12)
    assert ro.decode(lib) == raw
    assert ipc.ipc_decode_container(lib) == raw


def test_round_trip_large_and_threads():
    rng = np.random.default_rng(3)
    raw = rng.geometric(0.05, (5 << 20) + 123).clip(0, 255).astype(np.uint8).tobytes()
    c1 = ipc.ipc_encode_container(raw, nthreads=1)
    c8 = ipc.ipc_encode_container(raw, nthreads=8)
    assert c1 == c8  # blocks are independent: the thread count changes nothing
    assert ipc.ipc_decode_container(c1, nthreads=3) == raw


def test_order0_entropy_bound():
    """An i.i.d. block codes to within 1 % of n H / 8 bytes (H the empirical
    order-0 entropy, the least any memoryless coder can reach) plus the
    record's 517 fixed bytes."""
    rng = np.random.default_rng(5)
    raw = rng.geometric(0.3, 1 << 20).clip(0, 255).astype(np.uint8).tobytes()
    c = ipc.ipc_encode_container(raw)
    p = np.bincount(np.frombuffer(raw, np.uint8), minlength=256) / len(raw)
    H = -(p[p > 0] * np.log2(p[p > 0])).sum()
    rec = len(c) - 24 - 4
    assert len(raw) * H / 8 <= rec - 517 + 8  # cannot beat the entropy (a few bytes of state)
    assert rec <= 1.01 * len(raw) * H / 8 + 517


def test_stored_and_single_symbol_records():
    rng = np.random.default_rng(9)
    raw = rng.integers(0, 256, 4096, dtype=np.uint8).tobytes()  # incompressible
    c = ipc.ipc_encode_container(raw, block_log2=12)
    assert len(c) == 24 + 4 + 1 + 4096 and c[28] == 0
    c = ipc.ipc_encode_container(b"\x42" * 4096, block_log2=12)
    # one symbol of frequency 4096: the states never move, no byte is
    # emitted; the record holds the two final states
    assert len(c) == 24 + 4 + 1 + 512 + 8 and c[28] == 2


def test_corrupt_inputs_rejected():
    raw = np.random.default_rng(2).geometric(0.3, 10000).astype(np.uint8).tobytes()
    c = ipc.ipc_encode_container(raw, block_log2=12)
    bad = [b"XPCZ" + c[4:], c[:4] + b"\x03" + c[5:], c[:-1], c + b"\x00", c[:20]]
    tab = bytearray(c)
    off = 24 + 4 * 3 + 1  # first record's frequency table (3 blocks)
    tab[off] ^= 1  # frequencies no longer sum to 4096
    bad.append(bytes(tab))
    for k in (2, 6):  # the first record's final states 0 and 1
        st = bytearray(c)
        st[off + 512 + k] ^= 0x40
        bad.append(bytes(st))
    md = bytearray(c)
    md[off - 1] = 3  # the first record's mode
    bad.append(bytes(md))
    for b in bad:
        with pytest.raises(ipc.IpcError) as e:
            ipc.ipc_decode_container(b)
        assert e.value.rc == ipc.IPC_ECORRUPT
        with pytest.raises(ro.CodecError):
            ro.decode(b)


def test_oracle_container_shrinks():
    """An oracle container of a smooth field: the coder keeps it exact and
    shrinks it (plane streams of the low planes are nearly random, the high
    ones and the tables are not)."""
    x = synth.grf_k53((64, 64, 64), seed=4).numpy()
    raw = oracle.compress(x, 1e-6, oracle.ABS).export()
    c = ipc.ipc_encode_container(raw)
    assert ipc.ipc_decode_container(c) == raw
    assert len(c) < len(raw)
    assert math.isfinite(len(raw) / len(c))


def test_version_1_containers_still_decode():
    """Containers of version 1 (one rANS state per record), as the
    restatement still writes them, decode in the library and in the
    restatement; version 2 records are one state pair per record."""
    rng = np.random.default_rng(8)
    for raw in (rng.geometric(0.2, 20000).clip(0, 255).astype(np.uint8).tobytes(), b"\x05" * 5000,
                bytes(range(256)) * 40):
        v1 = ro.encode(raw, block_log2=12, version=1)
        assert v1[4] == 1 and ro.decode(v1) == raw
        assert ipc.ipc_decode_container(v1) == raw
        v2 = ro.encode(raw, block_log2=12)
        assert v2[4] == 2 and v2 == ipc.ipc_encode_container(raw, block_log2=12)


@pytest.mark.parametrize("n", [4097, 4099, 6001, 8191])
def test_odd_length_coded_blocks(n):
    """One coded block of odd length (block size 2^13): both states finish
    in their initial value only if the odd symbol was coded by state 0."""
    raw = np.random.default_rng(n).geometric(0.4, n).clip(0, 255).astype(np.uint8).tobytes()
    c = ipc.ipc_encode_container(raw, block_log2=13)
    assert c[28] == 2  # coded, not stored
    assert c == ro.encode(raw, block_log2=13)
    assert ipc.ipc_decode_container(c) == raw and ro.decode(c) == raw
