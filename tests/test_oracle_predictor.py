"""Pins of the oracle's level schedule (Sec. 4.1, Fig. 3) and interpolation
predictor (Eq. 1, Eq. 2): coverage by an independent formula, the printed
coefficients via impulse responses, and polynomial exactness."""
import itertools
import json
import os

import numpy as np
import pytest

import pyref
from helpers import exact_eb
from paper_2502_04093_gb300 import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))

SHAPES = ([(n,) for n in range(1, 40)] +
          [(a, b) for a in range(1, 10) for b in range(1, 10)] +
          [(a, b, c) for a in (1, 2, 3, 5) for b in (1, 4, 7) for c in (1, 2, 6, 9)] +
          [(9, 9, 9), (3, 5, 7), (33, 1, 17), (2, 2, 2), (1, 1, 1), (16, 8, 4)])


@pytest.mark.parametrize("shape", SHAPES)
def test_every_point_produced_once(oracle, shape):
    sp = oracle.point_stage(shape).reshape(-1)
    assert sp[0] == -1
    assert (sp[1:] >= 0).all(), "a point was missed (-2) or produced twice (-3)"
    st, K = pyref.stages(shape)
    assert (1 << K) >= max(shape) and (K == 0 or (1 << (K - 1)) < max(shape))
    # stage t of the oracle is the t-th non-empty (level desc, dim asc) class
    cls, _ = pyref.point_class(shape)
    for t, (l, d, pts) in enumerate(st):
        assert set(np.nonzero(sp == t)[0].tolist()) == set(pts)
    assert sp.max() == len(st) - 1 if len(st) else True


def _impulse_code(oracle, p, interp):
    eb = 2.0 ** -6  # 2eb = 1/32; impulse height 16 bins keeps every step exact
    h = 2 * eb * 16
    x = np.zeros(9, dtype=np.float32)
    x[p] = h
    f = oracle.compress(x, eb, oracle.ABS, interp)
    # 1-D, N = 9: level 1 targets are 1, 3, 5, 7; target 3 is code 1.
    t = f.info()["S"] - 1
    assert f.stage(t)["level"] == 1
    return f.codes(t)[1]


def test_cubic_coefficients_eq2(oracle):
    g = GOLD["cubic_coefficients"]
    for off, c in zip(g["offsets"], g["coefficients"]):
        q = _impulse_code(oracle, 3 + off, oracle.CUBIC)
        # q = rint((0 - c*h) / 2eb) = -16 c exactly
        assert q == -round(16 * c) and -q / 16.0 == c


def test_linear_coefficients_eq1(oracle):
    g = GOLD["linear_coefficients"]
    for off, c in zip(g["offsets"], g["coefficients"]):
        q = _impulse_code(oracle, 3 + off, oracle.LINEAR)
        assert -q / 16.0 == c
    # outside the linear stencil the impulse does not reach target 3
    assert _impulse_code(oracle, 0, oracle.LINEAR) == 0


def test_inf_norms_from_impulse_responses(oracle):
    g = GOLD["interp_inf_norm"]
    cub = sum(abs(_impulse_code(oracle, 3 + o, oracle.CUBIC)) / 16.0 for o in (-3, -1, 1, 3))
    lin = sum(abs(_impulse_code(oracle, 3 + o, oracle.LINEAR)) / 16.0 for o in (-1, 1))
    assert cub == g["cubic"] and lin == g["linear"]


def _positions_1d(N, l, ncodes):
    s = 1 << (l - 1)
    return [s + 2 * s * c for c in range(ncodes)]


@pytest.mark.parametrize("N", [9, 17, 33, 65, 100])
def test_cubic_exact_on_cubic_polynomials(oracle, N):
    i = np.arange(N, dtype=np.float64)
    x = (i ** 3 - 7 * i ** 2 + 3 * i - 11).astype(np.float32)
    f = oracle.compress(x, exact_eb(x), oracle.ABS, oracle.CUBIC)
    checked = 0
    for t in range(f.info()["S"]):
        st = f.stage(t)
        q = f.codes(t)
        s = 1 << (st["level"] - 1)
        for c, pos in enumerate(_positions_1d(N, st["level"], st["ncodes"])):
            if pos - 3 * s >= 0 and pos + 3 * s <= N - 1:
                assert q[c] == 0, (pos, s)
                checked += 1
        assert st["noutliers"] == 0
    assert checked > 0


@pytest.mark.parametrize("N", [9, 20, 64])
def test_linear_exact_on_linear_functions(oracle, N):
    i = np.arange(N, dtype=np.float64)
    x = (3 * i - 5).astype(np.float32)
    f = oracle.compress(x, exact_eb(x), oracle.ABS, oracle.LINEAR)
    for t in range(f.info()["S"]):
        st = f.stage(t)
        q = f.codes(t)
        s = 1 << (st["level"] - 1)
        for c, pos in enumerate(_positions_1d(N, st["level"], st["ncodes"])):
            if pos + s <= N - 1:
                assert q[c] == 0


def test_separable_cubic_3d(oracle):
    # f = p(i0) + p(i1) + p(i2): along every sweep line it is a cubic, so each
    # target whose cubic stencil fits gets q = 0.
    N = (17, 13, 19)
    g = np.indices(N).astype(np.float64)
    p = lambda v: v ** 3 - 4 * v ** 2 + v
    x = (p(g[0]) + p(g[1]) + p(g[2])).astype(np.float32)
    f = oracle.compress(x, exact_eb(x), oracle.ABS, oracle.CUBIC)
    st_list, _ = pyref.stages(N)
    zeros = 0
    for t, (l, d, pts) in enumerate(st_list):
        q = f.codes(t)
        s = 1 << (l - 1)
        for c, pidx in enumerate(pts):
            idx = np.unravel_index(pidx, N)
            if idx[d] - 3 * s >= 0 and idx[d] + 3 * s <= N[d] - 1:
                assert q[c] == 0
                zeros += 1
    assert zeros > 100


@pytest.mark.parametrize("N", [9, 17, 33, 65, 100])
def test_quadratic_boundaries_exact_on_quadratics(oracle, N):
    """Mode 2: a quadratic sequence is predicted exactly wherever a target has
    both near neighbours and at least one of the far ones: by Eq. 2 inside,
    by the three-point quadratic where one far neighbour is missing. Plain
    cubic mode falls back to Eq. 1 there, which misses the curvature."""
    i = np.arange(N, dtype=np.float64)
    x = (2 * i ** 2 - 9 * i + 4).astype(np.float32)
    eb = exact_eb(x)
    fq = oracle.compress(x, eb, oracle.ABS, oracle.CUBIC_QUAD)
    fc = oracle.compress(x, eb, oracle.ABS, oracle.CUBIC)
    boundary = 0
    for t in range(fq.info()["S"]):
        st = fq.stage(t)
        q, qc = fq.codes(t), fc.codes(t)
        s = 1 << (st["level"] - 1)
        for c, pos in enumerate(_positions_1d(N, st["level"], st["ncodes"])):
            if pos + s > N - 1:
                continue  # copy rule
            left, right = pos - 3 * s >= 0, pos + 3 * s <= N - 1
            if left or right:
                assert q[c] == 0, (pos, s)
            if left != right:
                boundary += 1
                assert qc[c] != 0  # Eq. 1 is not exact on a quadratic
        assert st["noutliers"] == 0
    assert boundary > 0


def test_quadratic_weights_and_norm():
    """The three-point weights are the Lagrange weights at 0 of the nodes
    -1, 1, 3 (left end) and -3, -1, 1 (right end), in units of s; their
    absolute sum is 1.25, the cubic stencil's infinity norm (Sec. 5.1)."""
    from fractions import Fraction as Fr

    def lagrange_at0(nodes):
        out = []
        for j, xj in enumerate(nodes):
            w = Fr(1)
            for m, xm in enumerate(nodes):
                if m != j:
                    w *= Fr(0 - xm, xj - xm)
            out.append(w)
        return out
    assert lagrange_at0([-1, 1, 3]) == [Fr(3, 8), Fr(6, 8), Fr(-1, 8)]
    assert lagrange_at0([-3, -1, 1]) == [Fr(-1, 8), Fr(6, 8), Fr(3, 8)]
    assert sum(abs(w) for w in lagrange_at0([-1, 1, 3])) == Fr(5, 4)


def test_quadratic_mode_errors_and_costs(oracle):
    """Mode 2 keeps the error guarantee (Theorem 1 with the cubic mode's
    p = 1.25), at the full precision and at every selection; an unknown
    interpolation mode is refused."""
    x = synth.random_field((33, 20, 17), seed=4, dtype=np.float32, kind="smooth")
    f = oracle.compress(x, 1e-5, oracle.REL, oracle.CUBIC_QUAD)
    y, v = f.retrieve(oracle.EB, 1e-5)
    assert np.abs(y.astype(np.float64) - x).max() <= f.info()["eb"]
    for E in (1e-2, 1e-3):
        y, v = f.retrieve(oracle.EB, E)
        assert np.abs(y.astype(np.float64) - x).max() <= v.selection()[2]
    assert oracle.compress_rc(x, 1e-3, interp=4) == oracle.EINVAL  # 3 is the per-field choice
