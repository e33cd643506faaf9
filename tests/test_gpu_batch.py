"""Batched compression / retrieval (one launch per level over all fields):
every field's result must equal its single-field result and the oracle's."""
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


def uneven_fields(scale=8, n=12, seed=1300):
    shapes, seeds = synth.zonal_batch(seed=seed, scale=scale)
    return [synth.zonal2d(shapes[i], seed=seeds[i]) for i in range(n)]


def test_batch_compress_equals_single_and_oracle():
    xs = uneven_fields()
    xs.append(synth.gaussians3d((20, 21, 22), seed=5))  # mixed rank, different K
    xs.append(synth.random_field((100,), seed=2))
    dev = [torch.from_numpy(x).cuda() for x in xs]
    hs = ipc.ipc_compress_batch(dev, 1e-4, ipc.IPC_EB_REL)
    try:
        for x, d, h in zip(xs, dev, hs):
            single = ipc.Field.compress(d, 1e-4, ipc.IPC_EB_REL)
            blob = ipc.ipc_export(h)
            assert blob == single.export()
            assert blob == oracle.compress(x, 1e-4, oracle.REL).export()
    finally:
        for h in hs:
            ipc.ipc_free(h)


def test_batch_mixed_dtypes_and_modes():
    xs = [synth.random_field((33, 40), seed=1), synth.sinusoids3d((16, 12, 20), seed=3),
          synth.random_field((9, 9, 9), seed=4, dtype=np.float64, kind="spiky")]
    dev = [torch.from_numpy(x).cuda() for x in xs]
    hs = ipc.ipc_compress_batch(dev, [1e-3, 1e-7, 1e-5], [ipc.IPC_EB_ABS, ipc.IPC_EB_REL,
                                                         ipc.IPC_EB_REL])
    try:
        for x, h, eb, m in zip(xs, hs, [1e-3, 1e-7, 1e-5], [0, 1, 1]):
            assert ipc.ipc_export(h) == oracle.compress(x, eb, m).export()
    finally:
        for h in hs:
            ipc.ipc_free(h)


def test_batch_mixed_interpolation():
    """One batch whose fields use the three interpolation modes: each field's
    container and reconstruction are the oracle's for its own mode."""
    xs = [synth.random_field((40, 33, 70), seed=11), synth.random_field((300, 77), seed=12),
          synth.random_field((21, 50, 130), seed=13, dtype=np.float64)]
    modes = [ipc.IPC_CUBIC_QUAD, ipc.IPC_LINEAR, ipc.IPC_CUBIC_QUAD]
    dev = [torch.from_numpy(x).cuda() for x in xs]
    hs = ipc.ipc_compress_batch(dev, 1e-5, ipc.IPC_EB_REL, modes)
    try:
        ofs = [oracle.compress(x, 1e-5, oracle.REL, m) for x, m in zip(xs, modes)]
        for h, of in zip(hs, ofs):
            assert ipc.ipc_export(h) == of.export()
        outs = [torch.empty_like(d) for d in dev]
        ipc.ipc_retrieve_batch(hs, [(ipc.IPC_TARGET_EB, 1e-3)] * 3, outs)
        torch.cuda.synchronize()
        for out, of in zip(outs, ofs):
            y, _ = of.retrieve(oracle.EB, 1e-3)
            assert np.array_equal(out.cpu().numpy().view(np.uint8), y.view(np.uint8))
    finally:
        for h in hs:
            ipc.ipc_free(h)


def test_batch_retrieve_and_plan_equal_single():
    xs = uneven_fields(n=10)
    dev = [torch.from_numpy(x).cuda() for x in xs]
    fields = [ipc.Field.compress(d, 1e-5, ipc.IPC_EB_REL) for d in dev]
    rng = np.random.default_rng(0)
    targets = []
    for i in range(len(xs)):
        if i % 3 == 2:
            targets.append((ipc.IPC_TARGET_BITRATE, float(rng.uniform(1, 12))))
        else:
            targets.append((ipc.IPC_TARGET_EB, float(10 ** rng.uniform(-5, -1))))
    outs = [torch.empty_like(d) for d in dev]
    views = ipc.ipc_retrieve_batch([f.h for f in fields], targets, outs, want_views=True)
    torch.cuda.synchronize()
    for f, t, o, v, x in zip(fields, targets, outs, views, xs):
        y, sv = f.retrieve(*t)
        torch.cuda.synchronize()
        assert torch.equal(o, y)
        assert ipc.ipc_selection(v) == sv.selection()
        of = oracle.compress(x, 1e-5, oracle.REL)
        oy, ov = of.retrieve(*t)
        assert np.array_equal(o.cpu().numpy(), oy) and ipc.ipc_selection(v) == ov.selection()
        ipc.ipc_free(v)
    # captured plan: replays give the same bits
    outs2 = [torch.full_like(d, float("nan")) for d in dev]
    plan = ipc.ipc_plan_retrieve_batch([f.h for f in fields], targets, outs2)
    try:
        for _ in range(3):
            ipc.ipc_plan_launch(plan)
        torch.cuda.synchronize()
        for o, o2 in zip(outs, outs2):
            assert torch.equal(o, o2)
    finally:
        ipc.ipc_free(plan)


def test_autotuned_shapes_keep_results():
    """ipc_autotune_retrieve times every launch shape of each level and
    records the fastest; reconstructions with the recorded shapes (single,
    batched, planned) stay bitwise equal to the oracle's."""
    x = synth.random_field((24, 70, 300), seed=88)  # rows 300/150/75/38/..: 1, 2, 4 planes per tile
    o = oracle.compress(x, 1e-5)
    g = ipc.Field.compress(torch.from_numpy(x).cuda(), 1e-5)
    try:
        ipc.ipc_autotune_clear()
        out = torch.empty(x.shape, dtype=torch.float32, device="cuda")
        n = ipc.ipc_autotune_retrieve(g.h, ipc.IPC_TARGET_EB, 1e-4, out, reps=1)
        ents = ipc.ipc_autotune_entries()
        assert n == len(ents) >= 1
        for dt, w16, M, ns, psm in ents:
            assert dt == 0 and w16 in (0, 1) and ns in (0, 1, 2, 4) and 0 <= psm <= 4
            assert ns == 0 or ns == 1 or M[2] <= 512 // ns
        oy, _ = o.retrieve(oracle.EB, 1e-4)
        assert np.array_equal(out.cpu().numpy().view(np.uint8), oy.view(np.uint8))
        for E in (1e-4, 1e-3):
            oy, _ = o.retrieve(oracle.EB, E)
            y, _ = g.retrieve(ipc.IPC_TARGET_EB, E)
            torch.cuda.synchronize()
            assert np.array_equal(y.cpu().numpy().view(np.uint8), oy.view(np.uint8)), E
        outs = [torch.empty_like(out) for _ in range(3)]
        tg = [(ipc.IPC_TARGET_EB, 1e-4)] * 3
        ipc.ipc_retrieve_batch([g.h] * 3, tg, outs)
        plan = ipc.ipc_plan_retrieve_batch([g.h] * 3, tg, outs)
        try:
            ipc.ipc_plan_launch(plan)
        finally:
            torch.cuda.synchronize()
            ipc.ipc_free(plan)
        oy, _ = o.retrieve(oracle.EB, 1e-4)
        for y in outs:
            assert np.array_equal(y.cpu().numpy().view(np.uint8), oy.view(np.uint8))
        with pytest.raises(ipc.IpcError):
            ipc.ipc_autotune_retrieve(g.h, ipc.IPC_TARGET_EB, 1e-4, out, reps=0)
    finally:
        ipc.ipc_autotune_clear()
