"""The per-field interpolation choice (IPC_INTERP_AUTO) through the C ABI:
single and batched compressions give the oracle's container for the same
choice (the oracle's rule: the smallest container on the centred sample,
compressed with the whole field's absolute bound, the lower mode on a tie),
on fields whose choices differ and on fields larger than the sample."""
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


def fields():
    x = synth.random_field((12, 200, 16), 9, kind="smooth")
    x[:, :20, :] += 50.0  # the whole field's range is outside the sample
    rng = np.random.default_rng(7)
    return [
        ("spiky 3-D (linear)", synth.random_field((40, 36, 44), 3, kind="spiky"), 1e-4, 1),
        ("gaussians 3-D (quadratic boundaries)", synth.gaussians3d((48, 40, 36), seed=1001), 1e-3, 1),
        ("zonal 2-D (cubic)", synth.zonal2d((120, 260), seed=1301), 1e-4, 1),
        ("sinusoids f64", synth.sinusoids3d((40, 40, 30), seed=1401), 1e-8, 1),
        ("3-D wider than the sample", synth.random_field((20, 150, 30), 5, kind="smooth"), 1e-5, 1),
        ("2-D wider than the sample", synth.zonal2d((40, 1500), seed=1302), 1e-4, 1),
        ("range outside the sample", x.astype(np.float32), 1e-4, 1),
        ("1-D absolute", np.cumsum(rng.normal(size=3000)).astype(np.float32), 1e-3, 0),
    ]


@pytest.mark.parametrize("i", range(8), ids=[f[0] for f in fields()])
def test_single_field_choice_equals_oracle(i):
    name, x, eb, mode = fields()[i]
    h = ipc.ipc_compress(torch.from_numpy(x).cuda(), eb, mode, interp=ipc.IPC_INTERP_AUTO)
    try:
        m = oracle.auto_interp(x, eb, mode)
        blob = ipc.ipc_export(h)
        assert blob == oracle.compress(x, eb, mode, interp=oracle.AUTO).export()
        assert blob == oracle.compress(x, eb, mode, interp=m).export()
    finally:
        ipc.ipc_free(h)


def test_batch_with_chosen_and_fixed_modes():
    fs = fields()
    xs = [f[1] for f in fs]
    ebs = [f[2] for f in fs]
    modes = [f[3] for f in fs]
    interp = [ipc.IPC_INTERP_AUTO if i % 3 else ipc.IPC_CUBIC for i in range(len(xs))]
    hs = ipc.ipc_compress_batch([torch.from_numpy(x).cuda() for x in xs], ebs, modes, interp=interp)
    try:
        for x, h, eb, m, it in zip(xs, hs, ebs, modes, interp):
            assert ipc.ipc_export(h) == oracle.compress(x, eb, m, interp=it).export()
    finally:
        for h in hs:
            ipc.ipc_free(h)


def test_refused_without_finite_values():
    x = torch.full((16, 16), float("nan"), device="cuda")
    with pytest.raises(ipc.IpcError) as e:
        ipc.ipc_compress(x, 1e-3, ipc.IPC_EB_REL, interp=ipc.IPC_INTERP_AUTO)
    assert e.value.rc == ipc.IPC_EINVAL
    with pytest.raises(ipc.IpcError) as e:
        ipc.ipc_compress(x, 1e-3, ipc.IPC_EB_ABS, interp=4)
    assert e.value.rc == ipc.IPC_EINVAL
