"""Pins of the oracle's coding primitives (Sec. 4.4) against the paper's
printed values, textbook base -2 arithmetic and brute force."""
import json
import os

import numpy as np
import pytest

import pyref

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def base_minus2(q: int) -> int:
    """Textbook conversion to base -2 by repeated division."""
    out, k = 0, 0
    while q != 0:
        r = q % 2
        out |= r << k
        q = (q - r) // -2
        k += 1
    return out


def test_paper_example_encodings(oracle):
    # Sec. 4.4.2: 1 -> 00000001 and -1 -> 00000011 in 8-bit negabinary.
    g = GOLD["negabinary_8bit"]["negabinary"]
    for v, s in g.items():
        assert format(oracle.negabinary(int(v)) & 0xFF, "08b") == s
        assert oracle.negabinary(int(v)) >> 8 == 0
    # and the contrast the paper draws with the other two encodings
    assert format(-1 & 0xFF, "08b") == GOLD["negabinary_8bit"]["twos_complement"]["-1"]
    assert format(0x80 | 1, "08b") == GOLD["negabinary_8bit"]["sign_magnitude"]["-1"]


def test_negabinary_matches_repeated_division(oracle):
    for q in range(-(1 << 16), (1 << 16) + 1):
        if q % 97 and abs(q) > 300:
            continue
        assert oracle.negabinary(q) == base_minus2(q), q
    rng = np.random.default_rng(5)
    for q in rng.integers(-(1 << 30), (1 << 30), size=3000):
        assert oracle.negabinary(int(q)) == base_minus2(int(q))


def test_negabinary_inverse_range(oracle):
    rng = np.random.default_rng(6)
    for n in list(rng.integers(0, 1 << 32, size=3000)) + [0, 0xFFFFFFFF, 0xAAAAAAAA, 0x55555555]:
        n = int(n)
        v = oracle.negabinary_inv(n)
        assert v == sum(((n >> k) & 1) * (-2) ** k for k in range(32))
    assert oracle.negabinary_inv(0xAAAAAAAA) == -2863311530
    assert oracle.negabinary_inv(0x55555555) == 1431655765


def paper_uncertainty(d: int) -> float:
    a, b = GOLD["uncertainty"]["negabinary_odd" if d % 2 else "negabinary_even"]
    return a * 2 ** d + b


def test_uncertainty_formula_is_max_of_d_digits():
    # Sec. 4.4.2: brute force over every d-digit negabinary number.
    for d in range(1, 21):
        vals = np.zeros(1, dtype=np.int64)
        for k in range(d):
            vals = np.concatenate([vals, vals + (-2) ** k])
        assert int(np.abs(vals).max()) == round(paper_uncertainty(d))
        # sign-magnitude comparison of the same passage: 2^d - 1
        assert (1 << d) - 1 >= round(paper_uncertainty(d))


def test_truncation_bounded_by_uncertainty(oracle):
    rng = np.random.default_rng(7)
    for q in rng.integers(-(1 << 21), 1 << 21, size=2000):
        n = oracle.negabinary(int(q))
        for b in range(0, 33):
            mask = 0 if b >= 32 else (0xFFFFFFFF >> b) << b
            qp = oracle.negabinary_inv(n & mask)
            assert abs(int(q) - qp) <= round(paper_uncertainty(b)) if b else qp == q
            assert qp % (1 << b) == 0 if b < 32 else qp == 0


def test_xor_prefix_definition(oracle):
    # Sec. 4.4.1: encoded bit = prefix_1 xor prefix_2 xor b, the prefix bits
    # being the two more significant bits of the same integer.
    rng = np.random.default_rng(8)
    assert GOLD["prefix_bits"]["value"] == 2
    for n in rng.integers(0, 1 << 32, size=2000):
        n = int(n)
        e = oracle.xor_encode(n)
        bits = [(n >> k) & 1 for k in range(32)] + [0, 0]
        for k in range(32):
            assert (e >> k) & 1 == bits[k] ^ bits[k + 1] ^ bits[k + 2]
        assert oracle.xor_decode(e) == n


def test_xor_progressive_sweep(oracle):
    # Every 4093rd word of the 32-bit range (a full-range stride), plus the
    # low 2^18 words: decode inverts encode, and planes >= b decode to the
    # digits >= b without the dropped planes.
    assert oracle.xor_check(0, 1 << 18, 1) == 0
    assert oracle.xor_check(12345, (1 << 32) // 4093, 4093) == 0


def test_pyref_coding_agrees(oracle):
    rng = np.random.default_rng(9)
    for q in rng.integers(-(1 << 21), 1 << 21, size=500):
        q = int(q)
        assert pyref.nb(q) == oracle.negabinary(q)
        assert pyref.nb_value(pyref.nb(q)) == q
        assert pyref.xor_dec(pyref.xor_enc(pyref.nb(q))) == pyref.nb(q)
