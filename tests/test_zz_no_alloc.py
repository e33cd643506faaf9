"""ipc_range_noalloc: the range reduction for callers that cannot allocate
device memory (a process whose memory is owned by another pool or allocator,
a loop with a fixed footprint). Through the C ABI, on two calls in a row, its
results must equal what the allocating path computes (ipc_compress's range,
read back with ipc_field_info) and the exact numpy values; a warm call must
leave the device's free memory unchanged. This file is collected last."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_04093_gb300 import build
    build.build()
    from paper_2502_04093_gb300 import ipc
    L = ipc.lib()
    L.ipc_range_noalloc.argtypes = [C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_uint64),
                                    C.c_int, C.c_void_p, C.POINTER(C.c_double)]
    return L


def call(L, tensors, dtype_code):
    n = len(tensors)
    ptrs = (C.c_void_p * max(n, 1))(*[t.data_ptr() for t in tensors])
    sizes = (C.c_uint64 * max(n, 1))(*[t.numel() for t in tensors])
    out = (C.c_double * (4 * max(n, 1)))()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.ipc_range_noalloc(n, ptrs, sizes, dtype_code, stream, out)
    return rc, np.array(out[:4 * n]).reshape(n, 4)


def reference(L, t):
    """The allocating path: ipc_compress computes the same range."""
    from paper_2502_04093_gb300 import ipc
    h = ipc.ipc_compress(t, 1e-3, ipc.IPC_EB_ABS)
    try:
        info = ipc.ipc_field_info(h)
    finally:
        ipc.ipc_free(h)
    return info["xmin"], info["xmax"]


def make_batch(seed, dtype):
    from paper_2502_04093_gb300 import synth
    rng = np.random.default_rng(seed)
    xs = []
    for i in range(5):
        shape = tuple(int(v) for v in rng.integers(3, 60, size=int(rng.integers(1, 4))))
        x = synth.random_field(shape, seed=seed * 10 + i, dtype=dtype,
                               kind=["smooth", "noise", "spiky"][i % 3])
        if i == 1:
            x.reshape(-1)[::7] = np.nan
        xs.append(x)
    return xs


@pytest.mark.parametrize("dtype,code", [(np.float32, 0), (np.float64, 1)])
def test_two_calls_match_the_allocating_path(lib, dtype, code):
    for seed in (1, 2):  # two calls in a row reuse the same device array
        xs = make_batch(seed, dtype)
        ts = [torch.from_numpy(x).cuda() for x in xs]
        rc, got = call(lib, ts, code)
        assert rc == 0
        for x, t, row in zip(xs, ts, got):
            fin = x[np.isfinite(x)].astype(np.float64)
            mn, mx = reference(lib, t)
            assert row[0] == mn and row[1] == mx
            assert row[0] == fin.min() and row[1] == fin.max()
            assert row[2] == np.abs(fin).max() and row[3] == fin.size


def test_rejects_more_arrays_than_the_scratch_holds(lib):
    t = torch.ones(4, device="cuda")
    from paper_2502_04093_gb300 import ipc
    rc, _ = call(lib, [t] * 1025, 0)
    assert rc == ipc.IPC_EINVAL
    rc, got = call(lib, [t] * 3, 0)
    assert rc == 0 and (got[:, :3] == 1.0).all() and (got[:, 3] == 4).all()


def test_signed_zeros(lib):
    """max|x| of signed zeros is +0 (an all -0.0 array, and a mixed one)."""
    for dt, code in ((np.float32, 0), (np.float64, 1)):
        neg = np.full(3000, -0.0, dtype=dt)
        mixed = np.zeros(5000, dtype=dt)
        mixed[::3] = -0.0
        mixed[1::7] = dt(-2.5)
        mixed[2::11] = dt(1.25)
        ts = [torch.from_numpy(neg).cuda(), torch.from_numpy(mixed).cuda()]
        rc, got = call(lib, ts, code)
        assert rc == 0
        assert got[0, 2] == 0.0 and not np.signbit(got[0, 2])
        assert got[0, 0] == 0.0 and got[0, 1] == 0.0 and got[0, 3] == 3000
        fin = mixed.astype(np.float64)
        assert got[1, 0] == fin.min() and got[1, 1] == fin.max()
        assert got[1, 2] == np.abs(fin).max() == 2.5 and got[1, 3] == 5000


def test_warm_call_allocates_nothing(lib):
    xs = make_batch(3, np.float32)
    ts = [torch.from_numpy(x).cuda() for x in xs]
    rc, first = call(lib, ts, 0)
    assert rc == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        rc, again = call(lib, ts, 0)
        assert rc == 0 and np.array_equal(first, again)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_capturing_stream_is_refused_and_capture_survives(lib):
    from paper_2502_04093_gb300 import ipc
    a = torch.arange(64, device="cuda", dtype=torch.float32)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        b = a * 2.0  # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b = a * 2.0
        rc, _ = call(lib, [a], 0)
    assert rc == ipc.IPC_EINVAL
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(b, a * 2.0)
    rc, got = call(lib, [a], 0)  # usable again outside the capture
    assert rc == 0 and got[0, 1] == 63.0 and got[0, 3] == 64
