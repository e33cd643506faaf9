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
