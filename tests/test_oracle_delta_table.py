"""The data maximum of |q - q'_b| (Sec. 5.1: the error of dropping b planes
of a stage "can be pre-computed during compression"), as the oracle computes
it from a stage's codes, against brute force from the definition: truncate
each code's negabinary digits, invert, subtract. The selection under this
tighter table keeps the guarantee (Theorem 1 needs only a true bound on
|q - q'|) and never loads more bytes than under the closed form."""
import numpy as np
import pytest

from paper_2502_04093_gb300 import synth

MASK = 0xAAAAAAAA


def nb(q):
    return ((q.astype(np.int64) + MASK) ^ MASK) & 0xFFFFFFFF


def nb_inv(n):
    return (n.astype(np.int64) ^ MASK) - MASK


def brute(q):
    """max |q - negabinary^-1(N & ~(2^b - 1))| for b = 0..32."""
    n = nb(q)
    out = np.zeros(33, dtype=np.uint64)
    for b in range(1, 33):
        keep = n & ~((1 << b) - 1) & 0xFFFFFFFF
        d = np.abs(q.astype(np.int64) - nb_inv(keep))
        out[b] = d.max() if d.size else 0
    return out


def uncert(b):
    return 0 if b <= 0 else ((2 << b) - 1) // 3 if b & 1 else ((2 << b) - 2) // 3


@pytest.mark.parametrize("shape,kind,eb", [((33, 20, 17), "smooth", 1e-5), ((40, 50), "noise", 1e-3),
                                           ((300,), "spiky", 1e-4), ((9, 9, 9), "smooth", 1e-7)])
def test_table_equals_brute_force(oracle, shape, kind, eb):
    x = synth.random_field(shape, seed=sum(shape), dtype=np.float32, kind=kind)
    f = oracle.compress(x, eb, oracle.REL)
    for t in range(f.info()["S"]):
        q = f.codes(t)
        m = f.delta_table(t)
        assert np.array_equal(m, brute(q)), t
        st = f.stage(t)
        H, Q = st["H"], st["Q"]
        # the closed form bounds it, and is reached once every digit is dropped
        for b in range(33):
            assert m[b] <= (0 if b == 0 else uncert(b) if b <= H else Q)
        for b in range(max(H, 0) + 1, 33):
            assert m[b] == Q


def test_hand_codes(oracle):
    """The last stage of a hand-built 9-point field has the codes 5, -3, 7, -1
    (base -2: 101, 1101, 11011, 11). Dropping b low digits changes them by
    b = 1: 1, 1, 1, 1; b = 2: 1, 1, 1, 1 (11011 -> 11000 = 8); b = 3: 5 (101
    -> 0), 5 (1101 -> 1000 = -8), 1, 1; b = 4: 5, 3, 9 (-> 10000 = 16), 1;
    b >= 5: the codes themselves, max 7. The closed form gives U(2) = 2 and
    U(4) = 10 where the data reach 1 and 9."""
    from test_oracle_cost_tables import CODES_1D, hand_field
    _, _, f, _, _ = hand_field(oracle, (9,), CODES_1D, oracle.CUBIC, oracle.STRICT)
    t = len(CODES_1D) - 1
    assert list(f.codes(t)) == [5, -3, 7, -1]
    assert list(f.delta_table(t)) == [0, 1, 1, 5, 9] + [7] * 28
    assert [uncert(b) for b in range(5)] == [0, 1, 2, 5, 10]


def test_data_model_keeps_bound_and_saves_bytes(oracle):
    x = synth.grf_k53((40, 48, 56), seed=21).numpy()
    f = oracle.compress(x, 1e-6, oracle.ABS)
    closed = []
    for E in (1e-1, 1e-2, 1e-3, 1e-4, 1e-5):
        _, v = f.retrieve(oracle.EB, E)
        closed.append(v.selection())
    f.set_delta_model(1)
    for E, (bc, yc, gc) in zip((1e-1, 1e-2, 1e-3, 1e-4, 1e-5), closed):
        y, v = f.retrieve(oracle.EB, E)
        b, by, g = v.selection()
        assert by <= yc and g <= E
        assert np.abs(y.astype(np.float64) - x).max() <= g
    f.set_delta_model(0)
    _, v = f.retrieve(oracle.EB, 1e-3)
    assert v.selection() == closed[2]
