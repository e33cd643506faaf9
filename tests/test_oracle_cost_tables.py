"""Value pins of the oracle's error-cost tables (Theorem 1, Sec. 5.1-5.2).

The fields here are built backwards from chosen quantization codes: every
prediction is evaluated in exact rational arithmetic (Eq. 1 / Eq. 2 and the
copy rule at the right edge), the value is set to prediction + q * bin, and the
construction checks that every intermediate of the element-type arithmetic is
exactly representable, so the compressor reproduces the chosen codes without
any rounding. The per-stage digit statistics H (highest nonzero negabinary
digit) and Q (max |q|) are then known by hand, and the expected cost of every
option b is written down from the definitions:

* uncertainty of b dropped digits, U(b) = (2/3)2^b - 1/3 (b odd) or
  (2/3)2^b - 2/3 (b even) (Sec. 4.4.2); the per-stage bound
  M(b) = 0 (b = 0), U(b) (b <= H), Q (b > H);
* paper mode (Theorem 1 as printed, err(l, b) = p^(l-1) * delta_l, Sec. 5.2):
  cost = ceil(p^(l-1) * max_t M_t(b) * bin/eb * 2^16);
* strict mode: each stage is amplified by p once per later sweep,
  a_t = p^(S-1-t), cost = sum_t ceil(a_t * M_t(b) * bin/eb * 2^16) + rho_l for
  b > 0, with the rounding margin rho_l = ceil(kappa * u * A/eb * 2^16 *
  sum_{t at levels <= l} a_t), kappa = 24 (cubic) / 12 (linear).

Costs are integers in units of eb * 2^-16. A mistake in the exponent of p,
in the stage order, in kappa, in the margin's stage set or in the bin width
changes at least one of the numbers checked here.
"""
from fractions import Fraction as Fr
import math

import numpy as np
import pytest

from helpers import eb_for_bin

P = Fr(5, 4)          # infinity norm of the cubic stencil (Sec. 5.1)
U53 = Fr(1, 2 ** 53)  # unit roundoff of f64


def uncert(b):
    if b <= 0:
        return 0
    return (2 ** (b + 1) - 1) // 3 if b % 2 == 1 else (2 ** (b + 1) - 2) // 3


def stage_list(shape):
    """Stages (level, dim, [targets in row-major lattice order]) of a padded
    3-D grid, coarse to fine, dims 0..2 inside a level (Sec. 4.1)."""
    N = (1,) * (3 - len(shape)) + tuple(shape)
    K = 0
    while (1 << K) < max(N):
        K += 1
    out = []
    for l in range(K, 0, -1):
        s = 1 << (l - 1)
        for d in range(3):
            axes = []
            for e in range(3):
                if e == d:
                    axes.append(range(s, N[e], 2 * s))
                elif e < d:
                    axes.append(range(0, N[e], s))
                else:
                    axes.append(range(0, N[e], 2 * s))
            pts = [(a, b, c) for a in axes[0] for b in axes[1] for c in axes[2]]
            if pts:
                out.append((l, d, pts))
    return N, K, out


def exact_f64(v: Fr) -> float:
    f = float(v)
    assert Fr(f) == v, "not exactly representable: %s" % v
    return f


def exact_f32(v: Fr) -> float:
    f = float(np.float32(float(v)))
    assert Fr(f) == v, "not exactly representable in f32: %s" % v
    return f


def build_field(shape, codes, cubic, anchor, g, exact_f64=exact_f64):
    """Values whose codes are exactly `codes` (one list per stage) for bin g.
    Checks that every intermediate of the predictor is exact (in f64, or in
    the type whose check is passed as exact_f64)."""
    N, K, st = stage_list(shape)
    assert len(st) == len(codes)
    xh = {(0, 0, 0): Fr(anchor)}
    for (l, d, pts), qs in zip(st, codes):
        s = 1 << (l - 1)
        assert len(pts) == len(qs)
        for p, q in zip(pts, qs):
            i = p[d]

            def at(off):
                c = list(p)
                c[d] = i + off
                return xh[tuple(c)]
            b = at(-s)
            if i + s > N[d] - 1:
                pred = b
            elif cubic and i - 3 * s >= 0 and i + 3 * s <= N[d] - 1:
                a, c_, dd = at(-3 * s), at(s), at(3 * s)
                u = b + c_
                v = a + dd
                w = 9 * u
                z = w - v
                for t in (u, v, w, z):
                    exact_f64(t)
                pred = z / 16
            else:
                u = b + at(s)
                exact_f64(u)
                pred = u / 2
            exact_f64(pred)
            xh[p] = pred + q * g
            exact_f64(xh[p])
    x = np.zeros(N, dtype=np.float64)
    for p, v in xh.items():
        x[p] = exact_f64(v)
    return x.reshape(shape), st


def nb_digits(q):
    """Negabinary digits of q by repeated division by -2 (textbook)."""
    out, k, v = 0, 0, q
    while v != 0:
        r = v % 2
        out |= r << k
        v = (v - r) // -2
        k += 1
    return out


def stage_stats(qs):
    orr = 0
    for q in qs:
        orr |= nb_digits(q)
    H = orr.bit_length() - 1
    return H, max(abs(q) for q in qs)


def M_of(H, Q, b):
    if b == 0:
        return 0
    return uncert(b) if b <= H else Q


def expected_costs(st, HQ, K, cubic, strict, bin_rel, A_over_eb, u=U53):
    """The cost table of the module docstring, in exact rationals (u: the
    element type's unit roundoff)."""
    S = len(st)
    p = P if cubic else Fr(1)
    kappa = 24 if cubic else 12
    cost = np.zeros((K, 33), dtype=np.int64)
    for l in range(1, K + 1):
        ts = [t for t in range(S) if st[t][0] == l]
        asum = sum((p ** (S - 1 - t) if strict else 1) for t in range(S) if st[t][0] <= l)
        rho_exact = kappa * u * A_over_eb * 65536 * asum
        if strict:
            # the oracle evaluates the margin in f64: keep it off an integer
            assert abs(rho_exact - round(rho_exact)) > Fr(1, 10 ** 9)
        rho = math.ceil(rho_exact)
        for b in range(33):
            if strict:
                c = sum(math.ceil(p ** (S - 1 - t) * M_of(*HQ[t], b) * bin_rel * 65536)
                        for t in ts)
                if b > 0:
                    c += rho
            else:
                m = max(M_of(*HQ[t], b) for t in ts)
                c = math.ceil(p ** (l - 1) * m * bin_rel * 65536)
            cost[l - 1, b] = c
    return cost


# 1-D, N = 9: K = 4, one stage per level (levels 4, 3, 2, 1).
CODES_1D = [[32], [-16], [48, 0], [5, -3, 7, -1]]
# 2-D, 5 x 5: K = 3, two stages per level, S = 6.
CODES_2D = [[12], [-7, 20], [3, -40], [9, 0, -2],
            [1, -1, 6, 0, 2, -5], [0, 1, -3, 4, 0, 0, 2, -1, 5, 0]]


def hand_field(oracle, shape, codes, interp, bound, g=2.0 ** -7):
    """g is the exact bin of the quantizer. A small bin against max|x| = 0.75
    makes the f64 rounding margin rho_l a few hundred units."""
    x, st = build_field(shape, codes, interp == 1, 0.75, Fr(g))
    A = float(np.abs(x).max())
    eb = eb_for_bin(A, False, g / 2)
    f = oracle.compress(x, eb, oracle.ABS, interp, bound)
    info = f.info()
    assert info["S"] == len(codes) and info["eb"] == eb
    for t, qs in enumerate(codes):
        assert list(f.codes(t)) == qs
        assert f.stage(t)["noutliers"] == 0
    return x, st, f, eb, g


@pytest.mark.parametrize("bound", ["strict", "paper"])
def test_1d_cost_values(oracle, bound):
    strict = bound == "strict"
    x, st, f, eb, g = hand_field(oracle, (9,), CODES_1D, oracle.CUBIC,
                                 oracle.STRICT if strict else oracle.PAPER)
    HQ = [stage_stats(qs) for qs in CODES_1D]
    # by hand: 32 = 64 - 32 -> digits 6,5; -16 = -32 + 16; 48 = 64 - 32 + 16;
    # 5 = 101, -3 = 1101, 7 = 11011, -1 = 11 (base -2)
    assert HQ == [(6, 32), (5, 16), (6, 48), (4, 7)]
    for t, (H, Q) in enumerate(HQ):
        s = f.stage(t)
        assert (s["H"], s["Q"]) == (H, Q)
    E = 0.5
    cost, _ = f.option_tables(E)
    A_over_eb = (Fr(float(np.abs(x).max())) + Fr(E)) / Fr(eb)
    want = expected_costs(st, HQ, 4, True, strict, Fr(g) / Fr(eb), A_over_eb)
    assert np.array_equal(cost, want)
    # spot values written out: level 4 (p^3 = 1.953125) at b = 1 drops U(1) = 1,
    # level 1 (p^0) at b = 3 drops U(3) = 5; bin/eb is 2 less a few ulps.
    if not strict:
        assert cost[3, 1] == math.ceil(Fr(125, 64) * 1 * Fr(g) / Fr(eb) * 65536)
        assert cost[3, 1] == 256000
        assert cost[0, 3] == 655360
        assert cost[1, 32] == math.ceil(Fr(5, 4) * 48 * Fr(g) / Fr(eb) * 65536)


def test_2d_strict_stage_exponents(oracle):
    x, st, f, eb, g = hand_field(oracle, (5, 5), CODES_2D, oracle.CUBIC, oracle.STRICT)
    HQ = [stage_stats(qs) for qs in CODES_2D]
    for t, (H, Q) in enumerate(HQ):
        s = f.stage(t)
        assert (s["H"], s["Q"]) == (H, Q)
    for E in (0.25, 3.0):
        cost, _ = f.option_tables(E)
        A_over_eb = (Fr(float(np.abs(x).max())) + Fr(E)) / Fr(eb)
        want = expected_costs(st, HQ, 3, True, True, Fr(g) / Fr(eb), A_over_eb)
        assert np.array_equal(cost, want)
    # the margin differs between b = 0 and b = 1 exactly by rho_l plus the
    # stages' U(1) terms: level 3 holds stages 0 and 1 (a = p^5, p^4)
    cost, _ = f.option_tables(0.25)
    A_over_eb = (Fr(float(np.abs(x).max())) + Fr(0.25)) / Fr(eb)
    asum3 = sum(P ** k for k in range(6))
    rho3 = math.ceil(24 * U53 * A_over_eb * 65536 * asum3)
    u1 = sum(math.ceil(P ** k * 1 * Fr(g) / Fr(eb) * 65536) for k in (5, 4))
    assert cost[2, 1] - cost[2, 0] == rho3 + u1


def test_2d_paper_mode_values(oracle):
    x, st, f, eb, g = hand_field(oracle, (5, 5), CODES_2D, oracle.CUBIC, oracle.PAPER)
    HQ = [stage_stats(qs) for qs in CODES_2D]
    cost, _ = f.option_tables(1.0)
    want = expected_costs(st, HQ, 3, True, False, Fr(g) / Fr(eb), Fr(1))
    assert np.array_equal(cost, want)
    # level 2 holds the codes 3, -40 and 9, 0, -2: Q = 40 once every digit is
    # dropped, times p^(2-1)
    assert cost[1, 32] == math.ceil(Fr(5, 4) * 40 * Fr(g) / Fr(eb) * 65536)


def test_linear_kappa_and_unit_amplification(oracle):
    codes = [[32], [-16], [48, 0], [5, -3, 7, -1]]
    x, st, f, eb, g = hand_field(oracle, (9,), codes, oracle.LINEAR, oracle.STRICT)
    HQ = [stage_stats(qs) for qs in codes]
    cost, _ = f.option_tables(0.5)
    A_over_eb = (Fr(float(np.abs(x).max())) + Fr(0.5)) / Fr(eb)
    want = expected_costs(st, HQ, 4, False, True, Fr(g) / Fr(eb), A_over_eb)
    assert np.array_equal(cost, want)
    # linear: every stage has amplification 1, the margin of level l counts
    # the l stages at levels <= l with kappa = 12
    for l in range(1, 5):
        rho = math.ceil(12 * U53 * A_over_eb * 65536 * l)
        H, Q = HQ[4 - l]
        assert cost[l - 1, 1] == math.ceil(1 * Fr(g) / Fr(eb) * 65536) + rho


def test_bytes_table_is_suffix_sum_of_stream_sizes(oracle):
    x, st, f, eb, g = hand_field(oracle, (5, 5), CODES_2D, oracle.CUBIC, oracle.STRICT)
    _, byts = f.option_tables(1.0)
    for l in range(1, 4):
        ts = [t for t in range(len(st)) if st[t][0] == l]
        for b in range(33):
            want = sum(f.stream_size(t, k) for t in ts for k in range(b, 32))
            assert byts[l - 1, b] == want
        assert byts[l - 1, 32] == 0


@pytest.mark.parametrize("interp", ["linear", "cubic"])
def test_margin_kappa_with_small_bin(oracle, interp):
    """With a bin of 2^-40 against max|x| = 0.75 the f64 rounding margin is a
    few hundred units per level, so kappa (24 cubic, 12 linear) and the set
    of stages it sums over show in every b > 0 entry."""
    cubic = interp == "cubic"
    g = 2.0 ** -40
    for shape, codes in (((9,), CODES_1D), ((5, 5), CODES_2D)):
        x, st, f, eb, _ = hand_field(oracle, shape, codes,
                                     oracle.CUBIC if cubic else oracle.LINEAR,
                                     oracle.STRICT, g)
        K = f.info()["K"]
        HQ = [stage_stats(qs) for qs in codes]
        for E in (1e-9, 2.0 ** -20 * 3):
            cost, _ = f.option_tables(E)
            A_over_eb = (Fr(float(np.abs(x).max())) + Fr(E)) / Fr(eb)
            want = expected_costs(st, HQ, K, cubic, True, Fr(g) / Fr(eb), A_over_eb)
            assert np.array_equal(cost, want)
            # the finest level's margin alone: kappa * u * A/eb * 2^16 * sum of
            # the finest stages' amplifications (1 and, in 2-D, p)
            fine = [t for t in range(len(st)) if st[t][0] == 1]
            a = [(P if cubic else 1) ** (len(st) - 1 - t) for t in fine]
            rho1 = math.ceil((24 if cubic else 12) * U53 * A_over_eb * 65536 * sum(a))
            assert rho1 > 100
            terms = sum(math.ceil(at * 1 * Fr(g) / Fr(eb) * 65536) for at in a)
            assert cost[0, 1] == terms + rho1
