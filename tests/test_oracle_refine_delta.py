"""Pins of the oracle's incremental refinement (Algorithm 2, Sec. 4.3).

* The window decode of the new planes, given only the two lowest loaded
  digits as prefix, returns the textbook negabinary digits (brute force).
* On fields whose arithmetic is exact (values on a dyadic grid, built
  backwards from chosen codes), x^old + Delta equals a fresh reconstruction of
  the new selection bit for bit: no rounding separates the two forms.
* On random fields it stays within the rounding tolerance of the canonical
  refinement and within its own reported bound (checked in FP64), and the
  selections and loaded bytes are the canonical ones.
"""
import numpy as np
import pytest

from paper_2502_04093_gb300 import synth
from test_oracle_cost_tables import CODES_2D, build_field, nb_digits
from fractions import Fraction as Fr
from helpers import eb_for_bin


def textbook_e(n):
    """Predictive XOR from the definition e_k = n_k ^ n_{k+1} ^ n_{k+2}."""
    e = 0
    for k in range(32):
        d = [(n >> j) & 1 if j < 32 else 0 for j in (k, k + 1, k + 2)]
        e |= (d[0] ^ d[1] ^ d[2]) << k
    return e


def test_decode_window_brute_force(oracle):
    rng = np.random.default_rng(7)
    qs = list(range(-300, 301)) + [int(v) for v in rng.integers(-2 ** 30, 2 ** 30, size=400)]
    for q in qs:
        n = nb_digits(q) & 0xFFFFFFFF
        e = textbook_e(n)
        for bo in (1, 2, 3, 5, 8, 17, 31, 32):
            for bn in sorted({0, max(0, bo - 1), max(0, bo - 2), bo // 2}):
                if bn > bo:
                    continue
                mask_hi = (0xFFFFFFFF << bo) & 0xFFFFFFFF if bo < 32 else 0
                mask_lo = (0xFFFFFFFF << bn) & 0xFFFFFFFF
                want = n & mask_lo & ~mask_hi & 0xFFFFFFFF
                # the encoded bits outside [bn, bo) must not matter
                e_win = e & mask_lo & ~mask_hi & 0xFFFFFFFF
                assert oracle.decode_window(e_win, n & mask_hi, bn, bo) == want


def exact_field(oracle, interp):
    g = 2.0 ** -7
    x, st = build_field((5, 5), CODES_2D, interp == 1, 0.75, Fr(g))
    eb = eb_for_bin(float(np.abs(x).max()), False, g / 2)
    return x, oracle.compress(x, eb, oracle.ABS, interp, oracle.STRICT)


@pytest.mark.parametrize("interp", [0, 1])
def test_exact_field_delta_equals_fresh(oracle, interp):
    x, f = exact_field(oracle, interp)
    info = f.info()
    n = info["n"]
    mand = info["mandatory"]
    seen = 0
    # budgets a few stream bytes above the mandatory part (header and tables)
    for k0 in (0, 12, 40):
        for k1 in (16, 48, 100, 400):
            br0, br1 = (mand + k0 + 0.5) * 8.0 / n, (mand + k1 + 0.5) * 8.0 / n
            y, v = f.retrieve(oracle.BITRATE, br0)
            b0 = v.selection()[0]
            _, inc = v.refine_delta(oracle.BITRATE, br1)
            b1 = v.selection()[0]
            if b1 == b0:
                continue
            assert inc
            seen += 1
            assert all(c <= p for c, p in zip(b1, b0))
            fresh = f.reconstruct(b1)
            assert np.array_equal(v.out.view(np.uint64), fresh.view(np.uint64)), (b0, b1)
    assert seen >= 3


def canonical_tolerance(f, E_abs):
    """C14's tolerance between the two forms: 2 kappa u A sum_t a_t."""
    info = f.info()
    S = info["S"]
    u = 2.0 ** -24 if f.dtype == np.float32 else 2.0 ** -53
    A = info["xmaxabs"] + E_abs
    return 2 * 24 * u * A * sum(1.25 ** k for k in range(S))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("shape,kind", [((33, 20, 17), "smooth"), ((40, 37), "noise"),
                                        ((200,), "spiky")])
def test_chain_close_to_canonical_and_within_bound(oracle, dtype, shape, kind):
    x = synth.random_field(shape, seed=31, dtype=dtype, kind=kind)
    if kind == "spiky":
        x[5] = np.nan
        x[17] = np.inf  # non-finite values are outliers, stored exactly
    eb = 1e-6 if dtype == np.float32 else 1e-9
    f = oracle.compress(x, eb, oracle.REL)
    rng = f.info()["xmax"] - f.info()["xmin"]
    ok = np.isfinite(x)
    yd, vd = f.retrieve(oracle.EB, 1e-1)
    yd = yd.copy()
    vd.out = yd
    yc, vc = f.retrieve(oracle.EB, 1e-1)
    ran_incremental = 0
    for E in (3e-2, 1e-2, 1e-3, 1e-4, 1e-5):
        if E * rng < f.info()["eb"]:
            break
        _, inc = vd.refine_delta(oracle.EB, E)
        vc.refine(oracle.EB, E)
        bd, byd, Gd = vd.selection()
        bc, byc, Gc = vc.selection()
        assert bd == bc and byd == byc
        assert Gd >= Gc and Gd <= E * rng * (1 + 1e-12)
        xd = x.astype(np.float64)
        err = np.abs(yd.astype(np.float64)[ok] - xd[ok]).max()
        assert err <= Gd, (E, err, Gd)
        diff = np.abs(yd.astype(np.float64)[ok] - yc.astype(np.float64)[ok]).max()
        assert diff <= canonical_tolerance(f, E * rng), (E, diff)
        # outliers (here the non-finite values) are untouched
        assert np.array_equal(np.isnan(yd), np.isnan(x))
        assert np.array_equal(np.isinf(yd), np.isinf(x))
        ran_incremental += inc
        if not inc:
            assert np.array_equal(yd, yc, equal_nan=True)
    assert ran_incremental >= 1


def test_falls_back_when_the_increment_bound_misses(oracle):
    # f32 with a coarse-level change: the increment's rounding margin does not
    # fit under the target, so the refinement reconstructs from scratch and
    # equals the canonical result bit for bit.
    x = synth.grf_k53((24, 24, 24), seed=3, dtype=np.float32).numpy()
    f = oracle.compress(x, 1e-7, oracle.ABS)
    yd, vd = f.retrieve(oracle.EB, 1e-1)
    yd = yd.copy()
    vd.out = yd
    yc, vc = f.retrieve(oracle.EB, 1e-1)
    fell_back = 0
    for E in (1e-3, 1e-5, 1e-7):
        _, inc = vd.refine_delta(oracle.EB, E)
        vc.refine(oracle.EB, E)
        assert vd.selection()[0] == vc.selection()[0]
        if not inc:
            fell_back += 1
            assert np.array_equal(yd, yc)
            assert vd.selection()[2] == vc.selection()[2]
    assert fell_back >= 1


def test_outlier_at_a_coarse_point_has_no_increment(oracle):
    # a finite outlier (far beyond the quantizer's range) on a coarse point:
    # its increment is zero, so its neighbours' increments are interpolated
    # from 0 there, not from its value
    x = synth.random_field((256,), seed=5, dtype=np.float32, kind="smooth")
    x[64] = 1e6
    f = oracle.compress(x, 1e-6, oracle.ABS)
    assert sum(f.stage(t)["noutliers"] for t in range(f.info()["S"])) >= 1
    mand, n = f.info()["mandatory"], f.info()["n"]
    yd, vd = f.retrieve(oracle.BITRATE, (mand + 8.5) * 8 / n)
    yd = yd.copy()
    vd.out = yd
    steps = 0
    for k in (40, 120, 400, 2000):
        b0 = vd.selection()[0]
        _, inc = vd.refine_delta(oracle.BITRATE, (mand + k + 0.5) * 8 / n)
        steps += vd.selection()[0] != b0
        assert inc or vd.selection()[0] == b0
        assert yd[64] == x[64]
        y = f.reconstruct(vd.selection()[0])
        assert np.abs(yd.astype(np.float64) - y).max() <= 1e-4
    assert steps >= 2


def test_increment_bound_values(oracle):
    """The incremental bound written out for a hand-built f32 field (H and Q
    known; all arithmetic exact in f32):
    G = eb + (truncation of the new selection + rounding part of the old +
    ceil(12 u D/eb 2^16 sum_{t at levels <= l_c} a_t) + ceil(u (max|x| + 2D)/eb 2^16))
    * eb 2^-16, D = G_old + G_new."""
    import math
    from test_oracle_cost_tables import expected_costs, stage_stats, exact_f32, P
    U24 = Fr(1, 2 ** 24)
    g = 2.0 ** -12
    x, st = build_field((5, 5), CODES_2D, True, 0.75, Fr(g), exact_f32)
    x = x.astype(np.float32)
    xmaxabs = float(np.abs(x).max())
    eb = eb_for_bin(xmaxabs, True, g / 2)
    f = oracle.compress(x, eb, oracle.ABS, oracle.CUBIC, oracle.STRICT)
    for t, qs in enumerate(CODES_2D):
        assert list(f.codes(t)) == qs
    HQ = [stage_stats(qs) for qs in CODES_2D]
    K, S = 3, len(st)

    def tables(E):
        A_over_eb = (Fr(xmaxabs) + Fr(E)) / Fr(eb)
        cost = expected_costs(st, HQ, K, True, True, Fr(g) / Fr(eb), A_over_eb, U24)
        rho = [math.ceil(24 * U24 * A_over_eb * 65536 *
                         sum(P ** (S - 1 - t) for t in range(S) if st[t][0] <= l))
               for l in range(1, K + 1)]
        return cost, rho

    checked = 0
    for E0 in (0.2, 0.08, 0.03):
        for E1 in (0.02, 0.005, 0.001):
            y, v = f.retrieve(oracle.EB, E0)
            b0, _, G0 = v.selection()
            c0, r0 = tables(E0)
            racc0 = sum(r0[l] for l in range(K) if b0[l] > 0)
            _, inc = v.refine_delta(oracle.EB, E1)
            b1, _, G1 = v.selection()
            if b1 == b0:
                continue
            c1, r1 = tables(E1)
            total1 = sum(int(c1[l, b1[l]]) for l in range(K))
            trunc1 = total1 - sum(r1[l] for l in range(K) if b1[l] > 0)
            Gnew = eb + total1 * eb / 65536.0
            lc = max(l + 1 for l in range(K) if b1[l] < b0[l])
            D = Fr(G0) + Fr(Gnew)
            asum = sum(P ** (S - 1 - t) for t in range(S) if st[t][0] <= lc)
            e1 = 12 * U24 * D / Fr(eb) * 65536 * asum
            assert e1 > 20  # large enough that kappa, l_c and D show
            eps = math.ceil(e1) + math.ceil(U24 * (Fr(xmaxabs) + 2 * D) / Fr(eb) * 65536)
            Gd = eb + (trunc1 + racc0 + eps) * eb / 65536.0
            if inc:
                assert G1 == Gd, (b0, b1, G1, Gd)
                checked += 1
            else:
                assert Gd > E1 and G1 == Gnew
    assert checked >= 2
