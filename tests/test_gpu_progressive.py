"""Progressive loading on the device (Sec. 5: a retrieval reads only the
bitplanes it selects): a field imported from the byte ranges of one
selection, planes added later from the ranges of a finer one. Every
retrieval selects among the resident planes and reconstructs bit for bit
what the oracle reconstructs from the same planes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle  # noqa: E402
from paper_2502_04093_gb300 import ipc, synth  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_04093_gb300 import build
    build.build()
    oracle.build()


def gather(raw, ranges):
    return b"".join(raw[a:a + n] for a, n in ranges)


def same(y, ref):
    return np.array_equal(y.cpu().numpy().view(np.uint8), ref.view(np.uint8))


def retrieve(h, shape, dtype, kind, value):
    out = torch.empty(shape, dtype=dtype, device="cuda")
    v = ipc.ipc_retrieve(h, kind, value, out)
    torch.cuda.synchronize()
    sel = ipc.ipc_selection(v)
    ipc.ipc_free(v)
    return out, sel


@pytest.mark.parametrize("shape,dtype,eb,mode", [((70, 45, 130), np.float32, 1e-6, oracle.ABS),
                                                 ((33, 40, 60), np.float64, 1e-9, oracle.REL),
                                                 ((300, 500), np.float32, 1e-5, oracle.REL)])
def test_partial_import_then_more_planes(shape, dtype, eb, mode):
    x = synth.random_field(shape, seed=sum(shape) + 1, dtype=dtype, kind="smooth")
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    o = oracle.compress(x, eb, mode)
    raw = o.export()
    K = o.info()["K"]
    y1, v1 = o.retrieve(oracle.EB, 1e-2)
    b1, bytes1, bound1 = v1.selection()
    h = ipc.ipc_import_partial(gather(raw, ipc.ipc_container_ranges(raw, b1)), b1)
    try:
        assert ipc.ipc_field_resident(h) == b1
        # the selection that loaded the planes: the oracle's retrieval exactly
        out, sel = retrieve(h, shape, tdt, ipc.IPC_TARGET_EB, 1e-2)
        assert sel[0] == b1 and sel[1] == bytes1 and sel[2] == bound1
        assert same(out, y1)
        # a looser target selects among the resident planes (b >= b1)
        out, sel = retrieve(h, shape, tdt, ipc.IPC_TARGET_EB, 1e-1)
        assert all(b >= r for b, r in zip(sel[0], b1))
        assert same(out, o.reconstruct(sel[0]))
        # a bitrate: the budget of the resident planes selects among them
        out, sel = retrieve(h, shape, tdt, ipc.IPC_TARGET_BITRATE, bytes1 * 8.0 / x.size)
        assert all(b >= r for b, r in zip(sel[0], b1)) and sel[1] <= bytes1
        assert same(out, o.reconstruct(sel[0]))
        # a tighter target than those planes allow, and the export, are refused
        with pytest.raises(ipc.IpcError) as e:
            retrieve(h, shape, tdt, ipc.IPC_TARGET_EB, 1e-4)
        assert e.value.rc == ipc.IPC_EBOUND
        with pytest.raises(ipc.IpcError) as e:
            ipc.ipc_export(h)
        assert e.value.rc == ipc.IPC_EINVAL
        # a view retrieved now, refined after loading more planes
        out_v = torch.empty(shape, dtype=tdt, device="cuda")
        view = ipc.ipc_retrieve(h, ipc.IPC_TARGET_EB, 1e-2, out_v)
        y3, v3 = o.retrieve(oracle.EB, 1e-4)
        b3 = v3.selection()[0]
        lo = [min(a, c) for a, c in zip(b1, b3)]
        more = gather(raw, ipc.ipc_container_ranges(raw, lo, b1))
        ipc.ipc_field_load_planes(h, more, lo)
        assert ipc.ipc_field_resident(h) == lo
        out, sel = retrieve(h, shape, tdt, ipc.IPC_TARGET_EB, 1e-4)
        assert sel[0] == b3 and same(out, y3)
        ipc.ipc_refine(view, ipc.IPC_TARGET_EB, 1e-4, out_v)
        torch.cuda.synchronize()
        assert same(out_v, o.reconstruct(ipc.ipc_selection(view)[0]))
        ipc.ipc_free(view)
        # the rest: every plane resident, the container exports whole
        ipc.ipc_field_load_planes(h, gather(raw, ipc.ipc_container_ranges(raw, [0] * K, lo)),
                                  [0] * K)
        assert ipc.ipc_field_resident(h) == [0] * K
        assert ipc.ipc_export(h) == raw
        out, _ = retrieve(h, shape, tdt, ipc.IPC_TARGET_EB, eb)
        assert same(out, o.retrieve(oracle.EB, eb)[0])
    finally:
        ipc.ipc_free(h)


def test_partial_fields_in_a_batch():
    """Partial fields in one batched retrieval: each selects among its own
    resident planes and reconstructs what the oracle does from them."""
    xs = [synth.random_field((40, 50, 60), seed=s, kind="smooth") for s in (1, 2, 3)]
    os_ = [oracle.compress(x, 1e-6, oracle.ABS) for x in xs]
    hs = []
    try:
        for o in os_:
            raw = o.export()
            b = o.retrieve(oracle.EB, 1e-3)[1].selection()[0]
            hs.append(ipc.ipc_import_partial(gather(raw, ipc.ipc_container_ranges(raw, b)), b))
        outs = [torch.empty((40, 50, 60), dtype=torch.float32, device="cuda") for _ in xs]
        views = ipc.ipc_retrieve_batch(hs, [(ipc.IPC_TARGET_EB, 1e-3), (ipc.IPC_TARGET_EB, 1e-2),
                                            (ipc.IPC_TARGET_EB, 1e-1)], outs, want_views=True)
        torch.cuda.synchronize()
        for h, o, out, v in zip(hs, os_, outs, views):
            b = ipc.ipc_selection(v)[0]
            assert all(a >= r for a, r in zip(b, ipc.ipc_field_resident(h)))
            assert same(out, o.reconstruct(b))
            ipc.ipc_free(v)
        assert same(outs[0], os_[0].retrieve(oracle.EB, 1e-3)[0])
    finally:
        for h in hs:
            ipc.ipc_free(h)


def test_bad_parts_refused():
    x = synth.random_field((30, 40, 50), seed=9, kind="smooth")
    o = oracle.compress(x, 1e-6, oracle.ABS)
    raw = o.export()
    b = o.retrieve(oracle.EB, 1e-2)[1].selection()[0]
    parts = gather(raw, ipc.ipc_container_ranges(raw, b))
    for bad, bb in ((parts[:-4], b), (parts + b"\0" * 4, b), (parts, [x + 1 for x in b])):
        with pytest.raises(ipc.IpcError) as e:
            ipc.ipc_import_partial(bad, bb)
        assert e.value.rc in (ipc.IPC_ECORRUPT, ipc.IPC_EINVAL)
    h = ipc.ipc_import_partial(parts, b)
    try:
        with pytest.raises(ipc.IpcError) as e:
            ipc.ipc_field_load_planes(h, b"\0" * 16, [0] * len(b))
        assert e.value.rc == ipc.IPC_ECORRUPT
        assert ipc.ipc_field_resident(h) == b  # unchanged
    finally:
        ipc.ipc_free(h)
