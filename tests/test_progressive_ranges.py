"""Progressive loading (Sec. 5: a retrieval reads only the bitplanes its
selection needs), host side: the byte ranges of a container that hold a
selection's planes, computed from the leading tables, on containers written
by the oracle. Their total is the oracle's count of loaded bytes for that
selection, and a selection's ranges plus the complement's tile the
container exactly. Runs on the CPU."""
import numpy as np
import pytest

from oracle import oracle
from paper_2502_04093_gb300 import ipc, synth


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2502_04093_gb300 import build
    build.build()
    oracle.build()


def covered(ranges):
    return sum(n for _, n in ranges)


@pytest.mark.parametrize("shape,dtype,eb,mode", [((40, 48, 56), np.float32, 1e-6, oracle.ABS),
                                                 ((300, 170), np.float32, 1e-5, oracle.REL),
                                                 ((30, 20, 25), np.float64, 1e-9, oracle.REL)])
def test_ranges_hold_the_selected_bytes(shape, dtype, eb, mode):
    x = synth.random_field(shape, seed=sum(shape), dtype=dtype, kind="smooth")
    o = oracle.compress(x, eb, mode)
    raw = o.export()
    info = o.info()
    head = raw[:112 + 288 * info["S"]]  # the tables alone are enough (no outliers here)
    K = info["K"]
    prev = None
    for E in (1e-1, 1e-2, 1e-3, 1e-4):
        _, v = o.retrieve(oracle.EB, E)
        b, nbytes, _ = v.selection()
        r = ipc.ipc_container_ranges(raw, b)
        assert r == ipc.ipc_container_ranges(head, b)
        assert r[0][0] == 0 and r[0][1] >= info["mandatory"]  # the tables (and adjacent streams)
        assert covered(r) == nbytes  # exactly what the selection loads
        rest = ipc.ipc_container_ranges(raw, [0] * K, b)
        spans = sorted(r + rest)
        assert spans[0][0] == 0 and sum(n for _, n in spans) == len(raw)
        for (a, n), (c, _) in zip(spans, spans[1:]):
            assert a + n == c  # disjoint and without gaps
        # per stage, the run is the streams of planes >= b_l (oracle sizes)
        want = sum(o.stream_size(t, k) for t in range(info["S"])
                   for k in range(b[o.stage(t)["level"] - 1], 32))
        assert covered(r) - info["mandatory"] == want
        if prev is not None and all(bp >= bn for bp, bn in zip(prev, b)):
            more = ipc.ipc_container_ranges(raw, b, prev)
            assert covered(more) == covered(r) - covered(ipc.ipc_container_ranges(raw, prev))
        prev = b


def test_range_arguments():
    x = synth.random_field((20, 21, 22), seed=3)
    raw = oracle.compress(x, 1e-4).export()
    K = oracle.compress(x, 1e-4).info()["K"]
    with pytest.raises(ipc.IpcError) as e:
        ipc.ipc_container_ranges(raw, [0] * (K + 1))
    assert e.value.rc == ipc.IPC_EINVAL
    with pytest.raises(ipc.IpcError) as e:
        ipc.ipc_container_ranges(raw, [5] * K, [4] * K)  # b_new above b_old
    assert e.value.rc == ipc.IPC_EINVAL
    with pytest.raises(ipc.IpcError) as e:
        ipc.ipc_container_ranges(raw[:60], [0] * K)
    assert e.value.rc == ipc.IPC_ECORRUPT
    assert ipc.ipc_container_ranges(raw, [32] * K) == [(0, len(raw) - sum(
        n for _, n in ipc.ipc_container_ranges(raw, [0] * K, [32] * K)))]
