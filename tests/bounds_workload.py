"""Workload run under the bounds-checking build (IPC_BOUNDS_CHECK=1) by
test_gpu_bounds.py: every kind of level launch on ragged shapes -- f32 and
f64, the three interpolation modes, 16- and 32-bit code rows, tiles of 1, 2
and 4 planes, batches, incremental refinements, partial fields -- checked
against the oracle, with no access outside its array recorded."""
import os
import sys

import numpy as np
import torch

assert os.environ.get("IPC_BOUNDS_CHECK") == "1"
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from oracle import oracle  # noqa: E402
from paper_2502_04093_gb300 import ipc, synth  # noqa: E402


def clean(what):
    rec = ipc.ipc_debug_bounds(reset=True)
    assert rec[0] == 0, "%s: %d accesses out of bounds, first at site %d index %d limit %d" % (
        (what,) + tuple(rec))


def same(y, ref):
    return np.array_equal(y.cpu().numpy().view(np.uint8), ref.view(np.uint8))


oracle.build()
clean("start")
cases = [((67, 130, 259), np.float32, oracle.CUBIC), ((5, 2049, 7), np.float32, oracle.LINEAR),
         ((33, 40, 61), np.float64, oracle.CUBIC_QUAD), ((200, 300), np.float32, oracle.CUBIC_QUAD),
         ((1030,), np.float64, oracle.CUBIC), ((70, 45, 100), np.float32, oracle.CUBIC)]
for shape, dtype, interp in cases:
    x = synth.random_field(shape, seed=sum(shape), dtype=dtype, kind="spiky")
    eb = 1e-6 if dtype == np.float32 else 1e-10
    o = oracle.compress(x, eb, oracle.REL, interp)
    g = ipc.Field.compress(torch.from_numpy(x).cuda(), eb, ipc.IPC_EB_REL, interp)
    assert g.export() == o.export(), shape
    clean("compress %s" % (shape,))
    for E in (1e-1, 1e-3, eb):
        y, _ = g.retrieve(ipc.IPC_TARGET_EB, E)
        torch.cuda.synchronize()
        assert same(y, o.retrieve(oracle.EB, E)[0]), (shape, E)
    br = o.info()["mandatory"] * 8.0 / x.size + 2.0  # two bits per value above the tables
    y, _ = g.retrieve(ipc.IPC_TARGET_BITRATE, br)
    torch.cuda.synchronize()
    assert same(y, o.retrieve(oracle.BITRATE, br)[0]), shape
    clean("retrieve %s" % (shape,))
    # incremental chain
    yo, vo = o.retrieve(oracle.EB, 1e-2)
    yg, vg = g.retrieve(ipc.IPC_TARGET_EB, 1e-2, refine_mode=ipc.IPC_REFINE_INCREMENTAL)
    for E in (1e-3, 1e-5):
        vo.refine_delta(oracle.EB, E)
        vg.refine(ipc.IPC_TARGET_EB, E)
        torch.cuda.synchronize()
        assert same(yg, yo), (shape, E)
    clean("refine %s" % (shape,))
    # a partial field and more planes
    raw = o.export()
    b = o.retrieve(oracle.EB, 1e-2)[1].selection()[0]
    parts = b"".join(raw[a:a + n] for a, n in ipc.ipc_container_ranges(raw, b))
    h = ipc.ipc_import_partial(parts, b)
    K = len(b)
    more = b"".join(raw[a:a + n] for a, n in ipc.ipc_container_ranges(raw, [0] * K, b))
    ipc.ipc_field_load_planes(h, more, [0] * K)
    assert ipc.ipc_export(h) == raw
    ipc.ipc_free(h)
    clean("partial %s" % (shape,))
# batches: uneven 2-D and 3-D fields, compressed and retrieved together
xs = [synth.random_field(s, seed=i, kind="smooth") for i, s in
      enumerate([(90, 180), (300, 77), (40, 33, 70), (9, 9, 9), (2, 3000)])]
dev = [torch.from_numpy(x).cuda() for x in xs]
hs = ipc.ipc_compress_batch(dev, 1e-5, ipc.IPC_EB_REL)
outs = [torch.empty_like(d) for d in dev]
ipc.ipc_retrieve_batch(hs, [(ipc.IPC_TARGET_EB, E) for E in (1e-1, 1e-2, 1e-3, 1e-4, 1e-5)], outs)
torch.cuda.synchronize()
for x, h, out, E in zip(xs, hs, outs, (1e-1, 1e-2, 1e-3, 1e-4, 1e-5)):
    o = oracle.compress(x, 1e-5, oracle.REL)
    assert ipc.ipc_export(h) == o.export()
    assert same(out, o.retrieve(oracle.EB, E)[0])
    ipc.ipc_free(h)
clean("batches")
print("bounds workload: no access out of bounds")
