"""Pins of the quantizer (Sec. 4.2.2, Eq. 4), the Theorem-1 style guarantee
(Sec. 5.1) and the two optimized loaders (Sec. 5.2, 5.3)."""
import itertools
import math

import numpy as np
import pytest

from helpers import eb_for_bin
from paper_2502_04093_gb300 import synth


def test_bin_width_two_eb(oracle):
    # 1-D N = 2: x[1] is predicted by copying the anchor, so q = (x1-x0)/bin,
    # the bin being 2eb less the element-type rounding allowance (here chosen
    # to be exactly 2^-7).
    for dt in (np.float32, np.float64):
        for k in range(-60, 61):
            x = np.array([0.75, 0.75 + k * 2.0 ** -7], dtype=dt)
            eb = eb_for_bin(float(np.abs(x).max()), dt == np.float32, 2.0 ** -8)
            f = oracle.compress(x, eb)
            assert f.codes(0)[0] == k
            assert f.stage(0)["noutliers"] == 0
    # residuals round to the nearest bin, exact half bins to the even one
    for k in range(-9, 10):
        for frac in (0.49, 0.5, 0.51):
            x = np.array([0.0, (k + frac) * 2.0 ** -7], dtype=np.float64)
            eb = eb_for_bin(float(np.abs(x).max()), False, 2.0 ** -8)
            f = oracle.compress(x, eb)
            assert f.codes(0)[0] == int(np.rint(k + frac))
            y, _ = f.retrieve(oracle.EB, eb)
            assert abs(y[1] - x[1]) <= eb


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("kind", ["smooth", "noise", "ramp", "const", "spiky"])
@pytest.mark.parametrize("shape", [(1,), (2,), (37,), (5, 9), (3, 5, 7), (12, 10, 9)])
def test_full_retrieval_within_eb(oracle, dtype, kind, shape):
    x = synth.random_field(shape, seed=hash((kind, shape)) % 1000, dtype=dtype, kind=kind)
    for eb in (1e-1, 1e-3, 1e-6):
        f = oracle.compress(x, eb, oracle.REL)
        ebabs = f.info()["eb"]
        y, v = f.retrieve(oracle.EB, eb)
        b, _, bound = v.selection()
        assert all(bb == 0 for bb in b)
        err = np.abs(y.astype(np.float64) - x.astype(np.float64)).max()
        assert err <= ebabs, (err, ebabs)
        assert bound == ebabs


def test_outliers_exact(oracle):
    x = synth.random_field((6, 7), seed=3, dtype=np.float32)
    x[2, 3] = np.nan
    x[4, 1] = np.inf
    x[1, 1] = -np.inf
    x[5, 6] = 3e30
    f = oracle.compress(x, 1e-3)
    assert sum(f.stage(t)["noutliers"] for t in range(f.info()["S"])) >= 4
    y, _ = f.retrieve(oracle.EB, 1e-3)
    assert np.isnan(y[2, 3]) and y[4, 1] == np.inf and y[1, 1] == -np.inf and y[5, 6] == x[5, 6]
    ok = np.isfinite(x)
    ok[5, 6] = False
    assert np.abs(y[ok].astype(np.float64) - x[ok]).max() <= 1e-3
    # dropping planes never touches outliers
    y2 = f.reconstruct([32] * f.info()["K"])
    assert np.isnan(y2[2, 3]) and y2[4, 1] == np.inf and y2[5, 6] == x[5, 6]


def consistent_bound(f, b, oracle):
    """Guaranteed bound of selection b, with the magnitude bound A made
    self-consistent (A = max|x| + bound)."""
    info = f.info()
    eb = info["eb"]
    E = eb
    for _ in range(50):
        cost, _ = f.option_tables(E)
        total = sum(int(cost[l, b[l]]) for l in range(len(b)))
        G = eb + total * eb / 65536.0
        if G <= E:
            return G
        E = G
    return G


@pytest.mark.parametrize("interp", [0, 1])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("shape,kind", [((9, 9), "smooth"), ((5, 6, 7), "noise"),
                                        ((33,), "smooth"), ((4, 8, 8), "ramp")])
def test_partial_planes_within_guaranteed_bound(oracle, interp, dtype, shape, kind):
    """Theorem 1: dropping planes keeps the L-inf error within
    eb + sum of the per-level costs (checked in FP64 for random selections)."""
    x = synth.random_field(shape, seed=11, dtype=dtype, kind=kind)
    for eb in (1e-2, 1e-5):
        f = oracle.compress(x, eb, oracle.REL, interp)
        K = f.info()["K"]
        rng = np.random.default_rng(K * 7 + interp)
        sels = [[0] * K, [32] * K] + [list(rng.integers(0, 33, size=K)) for _ in range(40)]
        sels += [list(rng.integers(0, 6, size=K)) for _ in range(40)]
        for b in sels:
            y = f.reconstruct(b)
            err = np.abs(y.astype(np.float64) - x.astype(np.float64)).max()
            G = consistent_bound(f, b, oracle)
            assert err <= G, (b, err, G)


def test_paper_mode_bound_is_smaller(oracle):
    x = synth.random_field((16, 16), seed=2, dtype=np.float64)
    fs = oracle.compress(x, 1e-4, oracle.REL, oracle.CUBIC, oracle.STRICT)
    fp = oracle.compress(x, 1e-4, oracle.REL, oracle.CUBIC, oracle.PAPER)
    cs, _ = fs.option_tables(1e-2)
    cp, _ = fp.option_tables(1e-2)
    assert (cp <= cs).all()


def brute_select(cost, byts, mandatory, kind, limit):
    K = cost.shape[0]
    best = None
    for b in itertools.product(range(33), repeat=K):
        c = sum(int(cost[l, b[l]]) for l in range(K))
        y = mandatory + sum(int(byts[l, b[l]]) for l in range(K))
        if kind == 0:
            if c > limit:
                continue
            key = (y, c, tuple(-v for v in b))
        else:
            if y > limit:
                continue
            key = (c, y, tuple(-v for v in b))
        if best is None or key < best[0]:
            best = (key, list(b))
    return None if best is None else best[1]


@pytest.mark.parametrize("shape,interp", [((8, 8), 1), ((3, 7), 0), ((5, 6, 7), 1), ((8,), 1)])
def test_selector_matches_brute_force(oracle, shape, interp):
    x = synth.random_field(shape, seed=21, dtype=np.float32)
    f = oracle.compress(x, 1e-4, oracle.REL, interp)
    info = f.info()
    assert info["K"] <= 3
    rng_ = info["xmax"] - info["xmin"]
    for E in (1e-4, 3e-4, 1e-3, 1e-2, 1e-1, 1.0):
        y, v = f.retrieve(oracle.EB, E)
        b, byts, bound = v.selection()
        Eabs = E * rng_
        cost, tab = f.option_tables(Eabs)
        B = math.floor(((Eabs - info["eb"]) / info["eb"]) * 65536.0)
        assert b == brute_select(cost, tab, info["mandatory"], 0, B)
        assert bound <= Eabs * (1 + 1e-12)
        assert np.abs(y.astype(np.float64) - x).max() <= bound
    for br in (0.5, 2.0, 4.0, 8.0, 16.0, 32.0):
        Sb = math.floor(br * info["n"] / 8.0)
        if Sb < info["mandatory"]:
            with pytest.raises(oracle.OracleError) as e:
                f.retrieve(oracle.BITRATE, br)
            assert e.value.rc == oracle.EBUDGET
            continue
        y, v = f.retrieve(oracle.BITRATE, br)
        b, byts, bound = v.selection()
        cost, tab = f.option_tables(-1.0)
        assert b == brute_select(cost, tab, info["mandatory"], 1, Sb)
        assert byts <= Sb


def test_bytes_monotone_in_fidelity(oracle):
    x = synth.gaussians3d((24, 24, 24), seed=5)
    f = oracle.compress(x, 1e-5, oracle.REL)
    prev = None
    for E in [max(float(e), 1e-5) for e in np.logspace(-1, -5, 17)]:
        _, v = f.retrieve(oracle.EB, E)
        _, byts, bound = v.selection()
        assert bound <= E * (f.info()["xmax"] - f.info()["xmin"]) * (1 + 1e-12)
        if prev is not None:
            assert byts >= prev
        prev = byts


def test_eb_below_compression_bound_rejected(oracle):
    x = synth.random_field((8, 8), seed=1)
    f = oracle.compress(x, 1e-3, oracle.REL)
    with pytest.raises(oracle.OracleError) as e:
        f.retrieve(oracle.EB, 5e-4)
    assert e.value.rc == oracle.EBOUND


def test_refine_chain_equals_fresh_reconstruction(oracle):
    x = synth.sinusoids3d((20, 18, 16), seed=1401)
    f = oracle.compress(x, 1e-8, oracle.REL)
    y, v = f.retrieve(oracle.EB, 1e-2)
    b_prev, by_prev, _ = v.selection()
    for E in (1e-4, 1e-6, 1e-8):
        y = v.refine(oracle.EB, E)
        b, byts, bound = v.selection()
        assert all(nb_ <= ob for nb_, ob in zip(b, b_prev))
        assert byts >= by_prev
        assert np.array_equal(y, f.reconstruct(b))
        assert np.abs(y - x).max() <= bound
        b_prev, by_prev = b, byts
    # at E = eb everything is loaded: equal to full retrieval
    assert b_prev == [0] * f.info()["K"]
    full, _ = f.retrieve(oracle.EB, 1e-8)
    assert np.array_equal(y, full)
    # a looser target leaves the view unchanged
    y2 = v.refine(oracle.EB, 1e-1)
    assert np.array_equal(y2, full) and v.selection()[0] == b_prev


@pytest.mark.parametrize("bad", [dict(eb=0.0), dict(eb=-1.0), dict(eb=float("nan")),
                                 dict(dims=(0, 4)), dict(dims=(2, 2, 2, 2))])
def test_invalid_arguments(oracle, bad):
    x = np.ones((4, 4), dtype=np.float32)
    assert oracle.compress_rc(x, bad.get("eb", 1e-3), dims=bad.get("dims")) == oracle.EINVAL
