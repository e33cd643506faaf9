"""Host selection of the library (ipc_select_container, Sec. 5.2 / 5.3) on
containers written by the oracle: the per-level plane choice, the loaded
bytes and the guaranteed bound must equal the oracle's, from the whole
container and from its leading tables alone. Runs on the CPU."""
import numpy as np
import pytest

from oracle import oracle
from paper_2502_04093_gb300 import ipc, synth


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2502_04093_gb300 import build
    build.build()
    oracle.build()


def prefix_len(o):
    """Header (112 bytes) + 32-byte stage records + 256-byte size tables."""
    return 112 + 288 * o.info()["S"]


CASES = [
    ((48, 40, 36), np.float32, "grf", 1e-6, oracle.ABS, oracle.CUBIC, oracle.STRICT),
    ((40, 33, 27), np.float32, "smooth", 1e-4, oracle.REL, oracle.CUBIC, oracle.STRICT),
    ((30, 31, 32), np.float64, "smooth", 1e-8, oracle.REL, oracle.CUBIC, oracle.PAPER),
    ((90, 180), np.float32, "zonal", 1e-4, oracle.REL, oracle.LINEAR, oracle.STRICT),
    ((1000,), np.float32, "noise", 1e-3, oracle.ABS, oracle.CUBIC, oracle.STRICT),
    ((20, 30, 40), np.float32, "spiky", 1e-4, oracle.ABS, oracle.CUBIC, oracle.STRICT),
    ((33, 50, 70), np.float32, "smooth", 1e-6, oracle.ABS, oracle.CUBIC_QUAD, oracle.STRICT),
    ((400, 700), np.float32, "zonal", 1e-5, oracle.REL, oracle.CUBIC, oracle.STRICT),
    # the per-field choice: the container carries the chosen mode
    ((24, 26, 28), np.float64, "spiky", 1e-7, oracle.REL, oracle.AUTO, oracle.STRICT),
    ((30, 29, 31), np.float32, "smooth", 1e-5, oracle.ABS, oracle.AUTO, oracle.PAPER),
]


def make(shape, dtype, kind, seed):
    if kind == "grf":
        return synth.grf_k53(shape, seed=seed).numpy().astype(dtype)
    if kind == "zonal":
        return synth.zonal2d(shape, seed=seed).astype(dtype)
    return synth.random_field(shape, seed=seed, dtype=dtype, kind=kind)


@pytest.mark.parametrize("case", CASES, ids=[str(c[0]) + c[2] for c in CASES])
def test_selection_equals_oracle(case):
    shape, dtype, kind, eb, mode, interp, bound = case
    x = make(shape, dtype, kind, seed=len(shape) * 7 + shape[0])
    o = oracle.compress(x, eb, mode, interp, bound)
    raw = o.export()
    head = raw[:prefix_len(o)]
    rng = np.random.default_rng(5)
    eb_targets = [eb, eb * 1.5, eb * 10, eb * 1e3, 0.3] + list(eb * 10 ** rng.uniform(0, 5, 12))
    br_targets = [0.25, 0.5, 1, 2, 4, 8, 16, 32] + list(rng.uniform(0.1, 24, 12))
    for k, targets in ((oracle.EB, eb_targets), (oracle.BITRATE, br_targets)):
        for t in targets:
            try:
                _, ov = o.retrieve(k, t)
                want = ov.selection()
            except oracle.OracleError as e:
                for buf in (raw, head):
                    with pytest.raises(ipc.IpcError) as ge:
                        ipc.ipc_select_container(buf, k, t)
                    assert ge.value.rc == e.rc
                continue
            assert ipc.ipc_select_container(raw, k, t) == want, (k, t)
            assert ipc.ipc_select_container(head, k, t) == want, (k, t)


def test_rejects_bad_headers():
    x = synth.random_field((20, 21, 22), seed=3)
    raw = oracle.compress(x, 1e-3).export()
    for buf in (raw[:50], b"\0" * 200, raw[:111]):
        with pytest.raises(ipc.IpcError) as e:
            ipc.ipc_select_container(buf, oracle.EB, 1e-2)
        assert e.value.rc == ipc.IPC_ECORRUPT
    o = oracle.compress(x, 1e-3)
    S = o.info()["S"]
    bad = bytearray(raw)
    off = 112 + 32 * S  # first size-table entry: plane 31 of stage 0
    bad[off] ^= 0x01  # a plane size no stream of the stage can have
    with pytest.raises(ipc.IpcError) as e:
        ipc.ipc_select_container(bytes(bad), oracle.EB, 1e-2)
    assert e.value.rc == ipc.IPC_ECORRUPT
