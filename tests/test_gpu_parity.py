"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer and byte results (quantization codes, plane streams, statistics,
outliers, selections) must be bit-exact; reconstructed floats must be bitwise
equal too, because both sides evaluate the same IEEE operations in the same
order without FMA contraction."""
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


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def both(x, eb, mode=ipc.IPC_EB_REL, interp=ipc.IPC_CUBIC, bound=ipc.IPC_BOUND_STRICT):
    g = ipc.Field.compress(to_dev(x), eb, mode, interp, bound)
    o = oracle.compress(x, eb, mode, interp, bound)
    return g, o


def check_retrieve(g, o, kind, value):
    try:
        oy, ov = o.retrieve(kind, value)
    except oracle.OracleError as e:
        with pytest.raises(ipc.IpcError) as ge:
            g.retrieve(kind, value)
        assert ge.value.rc == e.rc
        return None
    y, v = g.retrieve(kind, value)
    torch.cuda.synchronize()
    assert v.selection() == ov.selection()
    got = y.cpu().numpy()
    assert np.array_equal(got.view(np.uint8), oy.view(np.uint8)), "reconstruction bits differ"
    return v, y


SMALL = [
    ((1,), np.float32, "smooth"), ((2,), np.float32, "smooth"), ((37,), np.float64, "noise"),
    ((1000,), np.float32, "smooth"), ((5, 9), np.float32, "smooth"), ((64, 63), np.float32, "noise"),
    ((33, 1, 17), np.float32, "smooth"), ((3, 5, 7), np.float64, "spiky"),
    ((40, 33, 27), np.float32, "smooth"), ((17, 70, 129), np.float32, "smooth"),
    ((9, 9, 9), np.float64, "ramp"), ((16, 16, 16), np.float32, "const"),
    ((2, 300, 5), np.float32, "noise"), ((100, 1, 1), np.float32, "smooth"),
]


@pytest.mark.parametrize("shape,dtype,kind", SMALL)
@pytest.mark.parametrize("interp", [ipc.IPC_CUBIC, ipc.IPC_LINEAR, ipc.IPC_CUBIC_QUAD])
def test_compress_bytes_and_retrieve_bits(shape, dtype, kind, interp):
    x = synth.random_field(shape, seed=sum(shape) + (7 if kind == "noise" else 0), dtype=dtype,
                           kind=kind)
    for eb in (1e-2, 1e-5):
        g, o = both(x, eb, interp=interp)
        assert g.export() == o.export(), "compressed container differs"
        assert g.size() == len(o.export())
        for E in (eb, eb * 3, eb * 100, 0.5):
            check_retrieve(g, o, oracle.EB, E)
        for br in (1.0, 4.0, 16.0):
            check_retrieve(g, o, oracle.BITRATE, br)


@pytest.mark.parametrize("mode,bound", [(ipc.IPC_EB_ABS, ipc.IPC_BOUND_STRICT),
                                        (ipc.IPC_EB_REL, ipc.IPC_BOUND_PAPER)])
def test_modes(mode, bound):
    x = synth.gaussians3d((30, 31, 32), seed=12)
    g, o = both(x, 1e-4, mode, ipc.IPC_CUBIC, bound)
    assert g.export() == o.export()
    for E in (1e-4, 1e-3, 1e-2):
        check_retrieve(g, o, oracle.EB, E)


def test_config1_gaussians_64cubed():
    """64^3 f32, 8 Gaussians + 1e-3 noise, eb = 1e-3 * range, cubic; retrieve
    at 1e-1, 1e-2, 1e-3."""
    x = synth.gaussians3d((64, 64, 64), seed=1001)
    g, o = both(x, 1e-3, ipc.IPC_EB_REL)
    assert g.export() == o.export()
    for E in (1e-1, 1e-2, 1e-3):
        v, y = check_retrieve(g, o, oracle.EB, E)
        _, _, bound = v.selection()
        err = np.abs(y.cpu().numpy().astype(np.float64) - x).max()
        assert err <= bound <= E * (x.max() - x.min()) * (1 + 1e-12)


def test_outliers_and_nonfinite():
    x = synth.random_field((20, 30, 40), seed=3, kind="spiky")
    x[1, 2, 3] = np.nan
    x[5, 5, 5] = np.inf
    g, o = both(x, 1e-4, ipc.IPC_EB_ABS)
    assert g.export() == o.export()
    for E in (1e-4, 1e-2, 10.0):
        check_retrieve(g, o, oracle.EB, E)


def test_many_outliers_grow_buffer():
    # every point is non-finite -> more outliers than the initial buffer
    x = np.full((300, 300), np.nan, dtype=np.float32)
    x[::7, ::3] = 1.0
    g, o = both(x, 1e-3, ipc.IPC_EB_ABS)
    assert g.export() == o.export()
    check_retrieve(g, o, oracle.EB, 1e-3)


def test_refine_chain_f64():
    """Sinusoid field, rel eb 1e-8; refine 1e-2 -> 1e-4 -> 1e-6 -> 1e-8 ends
    bitwise equal to full decompression, each step bitwise equal to the
    oracle's refine."""
    x = synth.sinusoids3d((48, 40, 32), seed=1401)
    g, o = both(x, 1e-8, ipc.IPC_EB_REL)
    assert g.export() == o.export()
    y, v = g.retrieve(ipc.IPC_TARGET_EB, 1e-2)
    oy, ov = o.retrieve(oracle.EB, 1e-2)
    for E in (1e-4, 1e-6, 1e-8):
        v.refine(ipc.IPC_TARGET_EB, E)
        oy = ov.refine(oracle.EB, E)
        torch.cuda.synchronize()
        assert v.selection() == ov.selection()
        assert np.array_equal(y.cpu().numpy(), oy)
    full, _ = g.retrieve(ipc.IPC_TARGET_EB, 1e-8)
    torch.cuda.synchronize()
    assert torch.equal(full, y)


def test_import_from_oracle_bytes():
    x = synth.zonal2d((90, 180), seed=1301)
    o = oracle.compress(x, 1e-4, oracle.REL)
    raw = o.export()
    g = ipc.Field.from_bytes(raw, x.shape, torch.float32)
    assert g.export() == raw
    for E in (1e-4, 1e-2):
        check_retrieve(g, o, oracle.EB, E)
    bad = bytearray(raw)
    bad[-3] ^= 0x10  # flips a payload/bitmap bit: population or size check fails
    bad2 = bytearray(raw)
    bad2[0] ^= 1
    for b in (bytes(bad2), raw[:-4], raw + b"\0\0\0\0"):
        with pytest.raises(ipc.IpcError) as e:
            ipc.ipc_import(b)
        assert e.value.rc == ipc.IPC_ECORRUPT


def test_import_coded_container():
    """ipc_import also takes the lossless stage's coded form (decoded on the
    host first): the same field, container and reconstructions; coded bytes
    that do not decode, or a coded container inside another, are refused."""
    from oracle import rans_oracle
    x = synth.random_field((40, 33, 70), seed=17)
    g, o = both(x, 1e-5, ipc.IPC_EB_ABS)
    raw = g.export()
    for coded in (ipc.ipc_encode_container(raw), rans_oracle.encode(raw, block_log2=14)):
        h = ipc.Field.from_bytes(coded, x.shape, torch.float32)
        assert h.export() == raw == o.export()
        for E in (1e-5, 1e-3):
            check_retrieve(h, o, oracle.EB, E)
    coded = ipc.ipc_encode_container(raw)
    for b in (coded[:-1], ipc.ipc_encode_container(coded)):
        with pytest.raises(ipc.IpcError) as e:
            ipc.ipc_import(b)
        assert e.value.rc == ipc.IPC_ECORRUPT


def test_errors():
    x = torch.ones(8, 8, device="cuda")
    with pytest.raises(ipc.IpcError) as e:
        ipc.ipc_compress(x, 0.0)
    assert e.value.rc == ipc.IPC_EINVAL
    # empty extents are rejected (every extent >= 1), as the oracle does
    for shape in [(0,), (3, 0, 5)]:
        with pytest.raises(ipc.IpcError) as e:
            ipc.ipc_compress(torch.empty(shape, device="cuda"), 1e-3)
        assert e.value.rc == ipc.IPC_EINVAL
        assert oracle.compress_rc(np.zeros(shape, np.float32), 1e-3) == e.value.rc
    f = ipc.Field.compress(x, 1e-3)
    with pytest.raises(ipc.IpcError) as e:
        f.retrieve(ipc.IPC_TARGET_EB, 1e-4)
    assert e.value.rc == ipc.IPC_EBOUND
    with pytest.raises(ipc.IpcError) as e:
        f.retrieve(ipc.IPC_TARGET_BITRATE, 0.01)
    assert e.value.rc == ipc.IPC_EBUDGET


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_large_ragged(dtype):
    """Several tiles per sweep with ragged rows in every dimension."""
    x = synth.random_field((67, 130, 259), seed=8, dtype=dtype)
    g, o = both(x, 1e-6)
    assert g.export() == o.export()
    for E in (1e-6, 1e-4, 1e-2):
        check_retrieve(g, o, oracle.EB, E)
    check_retrieve(g, o, oracle.BITRATE, 2.0)


@pytest.mark.parametrize("shape,dtype", [((67, 130, 259), np.float32), ((67, 130, 259), np.float64),
                                         ((5, 2049, 7), np.float32), ((2, 33, 1100), np.float32),
                                         ((1030,), np.float64), ((200, 1000), np.float32)])
def test_quadratic_boundaries_tiled(shape, dtype):
    """Cubic interpolation with the three-point quadratic at the boundaries:
    every sweep of the tiled level kernels and of the coarse-level kernel
    meets targets that miss one far neighbour (near both ends of every
    extent, at every level)."""
    x = synth.random_field(shape, seed=sum(shape) + 5, dtype=dtype)
    g, o = both(x, 1e-6, interp=ipc.IPC_CUBIC_QUAD)
    assert g.export() == o.export()
    for E in (1e-6, 1e-4, 1e-2):
        check_retrieve(g, o, oracle.EB, E)
    check_retrieve(g, o, oracle.BITRATE, 2.0)


def test_unaligned_output_view():
    """A reconstruction target that starts one element into its allocation
    takes the scalar-store path and gives the same bits."""
    x = synth.random_field((19, 40, 67), seed=13)
    g, o = both(x, 1e-4)
    buf = torch.empty(x.size + 1, dtype=torch.float32, device="cuda")
    out = buf[1:].view(x.shape)
    _, v = g.retrieve(ipc.IPC_TARGET_EB, 1e-3, out=out)
    torch.cuda.synchronize()
    oy, ov = o.retrieve(oracle.EB, 1e-3)
    assert v.selection() == ov.selection()
    assert np.array_equal(out.cpu().numpy(), oy)


@pytest.mark.parametrize("shape", [(1030,), (3, 1030), (2, 33, 1100), (1025, 3), (5, 2049, 7)])
def test_multi_tile_rows(shape):
    """Rows longer than one 512-column tile (halo across column tiles), odd
    extents at every level."""
    x = synth.random_field(shape, seed=len(shape))
    g, o = both(x, 1e-5)
    assert g.export() == o.export()
    for E in (1e-5, 1e-3):
        check_retrieve(g, o, oracle.EB, E)


def test_export_into_host_buffer():
    """ipc_export into a caller's (pinned) buffer gives the same container."""
    x = synth.random_field((33, 40, 50), seed=21)
    g, o = both(x, 1e-4)
    raw = o.export()
    n = ipc.ipc_export_size(g.h)
    assert n == len(raw)
    buf = torch.empty(n + 7, dtype=torch.uint8, pin_memory=True)
    mv = ipc.ipc_export(g.h, buf.numpy())
    assert bytes(mv) == raw
    with pytest.raises(ValueError):
        ipc.ipc_export(g.h, bytearray(n - 1))


@pytest.mark.parametrize("shape,dtype", [
    ((9, 257, 257), np.float32),   # level 1 one plane per tile, level 2 two, level 3 four
    ((5, 20, 513), np.float32),    # two column tiles at level 1
    ((17, 40, 129), np.float32),   # 129 / 65 / 33 columns: sub-tile edges
    ((12, 33, 256), np.float64),   # f64 tiles of 8 rows with two and four planes
    ((7, 64, 100), np.float64),
])
def test_planes_per_tile_and_dense_levels(shape, dtype):
    """Levels whose rows are narrow put two or four planes in a tile; levels
    above 1 read their known points from the next level's dense lattice."""
    x = synth.random_field(shape, seed=sum(shape), dtype=dtype)
    g, o = both(x, 1e-5)
    assert g.export() == o.export()
    for E in (1e-5, 1e-3, 1e-1):
        check_retrieve(g, o, oracle.EB, E)
    for br in (2.0, 8.0):
        check_retrieve(g, o, oracle.BITRATE, br)


def test_outliers_on_narrow_levels():
    x = synth.random_field((24, 100, 120), seed=31, kind="spiky")
    x[3, 50, 60] = np.inf
    g, o = both(x, 1e-4, ipc.IPC_EB_ABS)
    assert g.export() == o.export()
    for E in (1e-4, 1e-2, 1.0):
        check_retrieve(g, o, oracle.EB, E)


def test_batch_mixed_widths_and_repeats():
    """One batched retrieval over fields whose levels take different tile
    shapes (the launch uses the smallest planes-per-tile of the batch) and
    over the same field several times."""
    shapes = [(10, 40, 600), (12, 30, 100), (8, 64, 250)]
    xs = [synth.random_field(s, seed=40 + i) for i, s in enumerate(shapes)]
    gs = [ipc.Field.compress(to_dev(x), 1e-5) for x in xs]
    os_ = [oracle.compress(x, 1e-5) for x in xs]
    fields = [gs[0].h, gs[1].h, gs[2].h, gs[1].h, gs[1].h]
    srcs = [0, 1, 2, 1, 1]
    # (bitrates well above the small fields' mandatory tables)
    targets = [(ipc.IPC_TARGET_EB, 1e-3), (ipc.IPC_TARGET_BITRATE, 8.0), (ipc.IPC_TARGET_EB, 1e-5),
               (ipc.IPC_TARGET_EB, 1e-2), (ipc.IPC_TARGET_BITRATE, 16.0)]
    outs = [torch.empty(shapes[i], dtype=torch.float32, device="cuda") for i in srcs]
    ipc.ipc_retrieve_batch(fields, targets, outs)
    torch.cuda.synchronize()
    for j, (i, (k, v)) in enumerate(zip(srcs, targets)):
        oy, _ = os_[i].retrieve(oracle.EB if k == ipc.IPC_TARGET_EB else oracle.BITRATE, v)
        assert np.array_equal(outs[j].cpu().numpy().view(np.uint8), oy.view(np.uint8)), j


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_window_bases(dtype):
    """Codes up to ~2^21 (noise at eb 1e-6 of its scale): retrievals that drop
    0..21 low planes keep 16-plane windows at many bases, odd and even,
    across the levels (the code value is scaled by the window base)."""
    x = synth.random_field((20, 37, 140), seed=77, dtype=dtype, kind="noise")
    x = (x * np.linspace(0.2, 3.0, 140)).astype(dtype)  # code sizes vary along the rows
    g, o = both(x, 1e-6, ipc.IPC_EB_ABS)
    assert g.export() == o.export()
    for j in range(0, 22):
        check_retrieve(g, o, oracle.EB, 1e-6 * 2.0 ** j * 1.3)
    for br in (3.0, 6.0, 9.0, 12.0):
        check_retrieve(g, o, oracle.BITRATE, br)
