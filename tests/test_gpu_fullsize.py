"""Parity at the full size of the bench workload, in the launch configuration
the bench times: the 512^3 f32 field with the k^-5/3 power spectrum,
compressed at eb 1e-6 (absolute, cubic, strict). The whole container and
whole reconstructions are compared with the oracle's, bit for bit; the
oracle takes about a minute on one core."""
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


def test_bench_workload_512_cubed():
    x = synth.grf_k53((512, 512, 512), seed=1002, device="cuda")
    torch.cuda.synchronize()
    xh = x.cpu().numpy()  # the oracle gets the GPU's input exactly
    g = ipc.Field.compress(x, 1e-6)
    o = oracle.compress(xh, 1e-6)
    assert g.export() == o.export(), "512^3 container differs"
    del xh
    # eb 1e-1: 16-bit code rows at level 1; eb 1e-5: every plane, 32-bit rows;
    # 4 bits/value: a bitrate selection
    cases = [(ipc.IPC_TARGET_EB, 1e-1), (ipc.IPC_TARGET_EB, 1e-5), (ipc.IPC_TARGET_BITRATE, 4.0)]
    want = []
    for kind, v in cases:
        y, view = g.retrieve(kind, v)
        oy, ov = o.retrieve(oracle.EB if kind == ipc.IPC_TARGET_EB else oracle.BITRATE, v)
        torch.cuda.synchronize()
        assert view.selection() == ov.selection(), (kind, v)
        assert np.array_equal(y.cpu().numpy().view(np.uint32), oy.view(np.uint32)), (kind, v)
        bound = view.selection()[2]  # Theorem 1 (strict form): max error <= the guaranteed bound
        assert float((y.double() - x.double()).abs().max()) <= bound
        want.append(oy)
        del y, view
    # the same retrievals in one batched call (the bench's bitrate path)
    outs = [torch.empty_like(x) for _ in cases]
    ipc.ipc_retrieve_batch([g.h] * len(cases), cases, outs)
    torch.cuda.synchronize()
    for y, oy in zip(outs, want):
        assert np.array_equal(y.cpu().numpy().view(np.uint32), oy.view(np.uint32))
