"""Pins of the oracle's per-field interpolation choice (interp 3): the
interpolation mode whose container is smallest on a centred sample of the
field, compressed with the whole field's absolute error bound, the lower
mode on a tie; the field's container is then that mode's container. The
sample and the bound are rebuilt here with numpy and each mode's container
size comes from a separate compression, so a wrong crop, a bound taken from
the sample instead of the whole field, or a wrong tie rule fails."""
import numpy as np
import pytest

from paper_2502_04093_gb300 import synth

CAP = {1: 1 << 20, 2: 1024, 3: 128}


def sample(x):
    sl = []
    for n in x.shape:
        e = min(n, CAP[x.ndim])
        o = (n - e) // 2
        sl.append(slice(o, o + e))
    return np.ascontiguousarray(x[tuple(sl)])


def abs_eb(x, eb, mode, oracle):
    if mode == oracle.ABS:
        return eb
    v = x[np.isfinite(x)].astype(np.float64)
    r = float(v.max() - v.min())
    return eb * r if r > 0 else eb


def expected_mode(oracle, x, eb, mode, bound=0):
    s = sample(x)
    e = abs_eb(x, eb, mode, oracle)
    sizes = [len(oracle.compress(s, e, oracle.ABS, interp=m, bound=bound).export())
             for m in (0, 1, 2)]
    return int(np.argmin(sizes)), sizes  # argmin takes the first minimum


def fields():
    rng = np.random.default_rng(7)
    yield "spiky 3-D", synth.random_field((40, 36, 44), 3, kind="spiky"), 1e-4, 1
    yield "gaussians 3-D", synth.gaussians3d((48, 40, 36), seed=1001), 1e-3, 1
    yield "sinusoids f64", synth.sinusoids3d((40, 40, 30), seed=1401), 1e-8, 1
    yield "zonal 2-D", synth.zonal2d((120, 260), seed=1301), 1e-4, 1
    # larger than the sample along some dimensions (the centred crop)
    x = synth.random_field((20, 150, 30), 5, kind="smooth")
    yield "3-D wider than the sample", x, 1e-5, 1
    yield "2-D wider than the sample", synth.zonal2d((40, 1500), seed=1302), 1e-4, 1
    # an offset field: the relative bound comes from the whole field's range
    x = synth.random_field((12, 200, 16), 9, kind="smooth")
    x[:, :20, :] += 50.0
    yield "range outside the sample", x.astype(np.float32), 1e-4, 1
    yield "1-D absolute", np.cumsum(rng.normal(size=3000)).astype(np.float32), 1e-3, 0


@pytest.mark.parametrize("name,x,eb,mode", list(fields()), ids=[f[0] for f in fields()])
def test_choice_is_the_smallest_sample_container(oracle, name, x, eb, mode):
    m, sizes = expected_mode(oracle, x, eb, mode)
    assert oracle.auto_interp(x, eb, mode) == m, sizes
    auto = oracle.compress(x, eb, mode, interp=oracle.AUTO).export()
    assert auto == oracle.compress(x, eb, mode, interp=m).export()


def test_range_of_the_whole_field_sets_the_sample_bound(oracle):
    """A field whose crop excludes the extreme values: with the crop's own
    range the sample bound would be ten times smaller."""
    x = synth.random_field((10, 300, 10), 2, kind="smooth").astype(np.float64)
    x[:, :40, :] *= 10.0
    s = sample(x)
    assert np.ptp(s) < 0.5 * np.ptp(x)
    m, sizes = expected_mode(oracle, x, 1e-6, oracle.REL)
    assert oracle.auto_interp(x, 1e-6, oracle.REL) == m, sizes


def test_spikes_take_linear_and_cubic_polynomials_do_not(oracle):
    """Two fields whose best mode is known without compressing: rare huge
    spikes spread through a cubic stencil's wider support (linear wins), and
    an integer cubic polynomial is predicted exactly by the cubic rule in the
    interior, where the linear rule leaves a residual at every target."""
    x = synth.random_field((48, 48, 48), 3, kind="spiky")
    assert oracle.auto_interp(x, 1e-4, oracle.REL) == oracle.LINEAR
    i, j, k = np.meshgrid(*(np.arange(n, dtype=np.float64) for n in (33, 34, 35)), indexing="ij")
    p = (i ** 3 - 2 * j ** 3 + 3 * k ** 2 * i + j * k).astype(np.float32)
    assert oracle.auto_interp(p, 0.25, oracle.ABS) in (oracle.CUBIC, oracle.CUBIC_QUAD)


def test_invalid_arguments(oracle):
    x = np.full((8, 8), np.nan, dtype=np.float32)
    with pytest.raises(oracle.OracleError):
        oracle.auto_interp(x, 1e-3, oracle.REL)
    assert oracle.compress_rc(np.zeros(8, np.float32), 1e-3, oracle.ABS, interp=4) != 0
    assert oracle.compress_rc(np.zeros(8, np.float32), 1e-3, oracle.ABS, interp=oracle.AUTO) == 0


def test_ties_take_the_lower_mode(oracle):
    """A constant field codes to the same container under every mode (every
    prediction is exact), and a field of two points has no interpolated
    target: both ties go to linear."""
    for x in (np.full((9, 10, 11), 3.5, dtype=np.float32), np.array([1.0, 2.0], dtype=np.float64)):
        m, sizes = expected_mode(oracle, x, 1e-3, oracle.ABS)
        assert sizes[0] == sizes[1] == sizes[2]
        assert m == 0 and oracle.auto_interp(x, 1e-3, oracle.ABS) == oracle.LINEAR
