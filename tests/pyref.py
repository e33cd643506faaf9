"""Independent pure-Python restatement of IPComp for tiny grids (N-version pin).

Written from the paper's definitions without looking at the C++ oracle's
structure: a point's level and sweep come from the 2-adic valuation of its
coordinates instead of an enumerated stage list, and a stage's code order is
simply increasing linear index. Used only by the CPU tests to pin the oracle
byte-for-byte on grids of a few hundred points.

* level of a point i != 0: l = 1 + min_d v2(i_d) (v2(0) = inf); its sweep is
  the largest dimension e with v2(i_e) = l - 1 (Sec. 4.1, Fig. 3).
* prediction along that dimension with stride s = 2^(l-1): Eq. 2 (cubic) when
  i-3s and i+3s are inside, Eq. 1 when i+s is inside, else copy of i-s.
* quantization with bin 2(eb - 4u(max|x| + eb)), outliers stored exactly
  (Sec. 4.2.2).
* negabinary + 2-prefix XOR (Sec. 4.4), 32 planes per stage (Sec. 4.3).
"""
from __future__ import annotations

import math
import struct

import numpy as np


def v2(x: int) -> int:
    if x == 0:
        return 10 ** 9
    c = 0
    while x % 2 == 0:
        x //= 2
        c += 1
    return c


def padded(shape):
    shape = tuple(int(s) for s in shape)
    return (1,) * (3 - len(shape)) + shape


def point_class(shape):
    """Return dict point-linear-index -> (level, dim3) (anchor excluded) and K."""
    N = padded(shape)
    K = 0
    while (1 << K) < max(N):
        K += 1
    cls = {}
    for i0 in range(N[0]):
        for i1 in range(N[1]):
            for i2 in range(N[2]):
                i = (i0, i1, i2)
                if i == (0, 0, 0):
                    continue
                vals = [v2(c) for c in i]
                lm1 = min(vals)
                d = max(e for e in range(3) if vals[e] == lm1)
                cls[(i0 * N[1] + i1) * N[2] + i2] = (lm1 + 1, d)
    return cls, K


def stages(shape):
    """Ordered list of (level, dim3, [linear indices in increasing order])."""
    cls, K = point_class(shape)
    out = []
    for l in range(K, 0, -1):
        for d in range(3):
            pts = sorted(p for p, c in cls.items() if c == (l, d))
            if pts:
                out.append((l, d, pts))
    return out, K


def nb(q: int) -> int:
    """Negabinary digits of q as a 32-bit word (repeated division by -2)."""
    digits = 0
    k = 0
    v = q
    while v != 0:
        r = v % 2  # 0 or 1 (Python's % is non-negative)
        digits |= r << k
        v = (v - r) // -2
        k += 1
    assert k <= 32
    return digits


def nb_value(n: int) -> int:
    return sum(((n >> k) & 1) * (-2) ** k for k in range(32))


def xor_enc(n: int) -> int:
    e = 0
    for k in range(32):
        b = (n >> k) & 1
        p1 = (n >> (k + 1)) & 1 if k + 1 < 32 else 0
        p2 = (n >> (k + 2)) & 1 if k + 2 < 32 else 0
        e |= (b ^ p1 ^ p2) << k
    return e


def xor_dec(e: int) -> int:
    n = 0
    for k in range(31, -1, -1):
        p1 = (n >> (k + 1)) & 1 if k + 1 < 32 else 0
        p2 = (n >> (k + 2)) & 1 if k + 2 < 32 else 0
        n |= (((e >> k) & 1) ^ p1 ^ p2) << k
    return n


class _T:
    """Arithmetic in the element type: numpy scalars round every op."""

    def __init__(self, dtype):
        self.t = np.dtype(dtype).type
        self.is32 = np.dtype(dtype) == np.float32


def _pred(T, xh, N, idx3, d, s, cubic):
    i = idx3[d]

    def at(pos):
        j = list(idx3)
        j[d] = pos
        return xh[(j[0] * N[1] + j[1]) * N[2] + j[2]]

    b = at(i - s)
    if i + s > N[d] - 1:
        return b
    c = at(i + s)
    left, right = i - 3 * s >= 0, i + 3 * s <= N[d] - 1
    if cubic and left and right:
        a = at(i - 3 * s)
        dd = at(i + 3 * s)
        return (T.t(9) * (b + c) - (a + dd)) * T.t(0.0625)
    # mode 2: the quadratic through the three neighbours that exist
    # (Lagrange weights 3/8, 6/8, -1/8 at distances s, s, 3s)
    if cubic == 2 and right:
        return (T.t(3) * b + T.t(6) * c - at(i + 3 * s)) * T.t(0.125)
    if cubic == 2 and left:
        return (T.t(6) * b + T.t(3) * c - at(i - 3 * s)) * T.t(0.125)
    return (b + c) * T.t(0.5)


def _unlin(p, N):
    return (p // (N[1] * N[2]), (p // N[2]) % N[1], p % N[2])


def half_bin(eb, xmaxabs, is32):
    """Quantizer half bin: eb less 4u(max|x| + eb), at least eb/2, so that
    the value rebuilt in the element type stays within eb."""
    u = 2.0 ** -24 if is32 else 2.0 ** -53
    eq = eb - 4.0 * u * (xmaxabs + eb)
    return eq if eq >= 0.5 * eb else 0.5 * eb


def compress(x: np.ndarray, eb_user: float, eb_mode=0, cubic=True, bound=0):
    """Returns (container bytes, per-stage codes)."""
    T = _T(x.dtype)
    N = padded(x.shape)
    flat = [T.t(v) for v in x.reshape(-1)]
    fin = [float(v) for v in flat if math.isfinite(float(v))]
    xmin = min(fin) if fin else 0.0
    xmax = max(fin) if fin else 0.0
    xmaxabs = max(abs(v) for v in fin) if fin else 0.0
    eb = eb_user
    if eb_mode == 1:
        r = xmax - xmin
        eb = eb_user * r if r > 0 else eb_user
    eq = half_bin(eb, xmaxabs, T.is32)
    inv2eb = T.t(1.0 / (2.0 * eq))
    twoeb = T.t(2.0 * eq)
    ebchk = T.t(eb * ((1 - 2.0 ** -20) if T.is32 else (1 - 2.0 ** -50)))
    R = T.t(2.0 ** 21 if T.is32 else 2.0 ** 30)
    xh = list(flat)  # targets are overwritten in stage order
    st, K = stages(x.shape)
    codes, outl = [], []
    with np.errstate(all="ignore"):
        for (l, d, pts) in st:
            s = 1 << (l - 1)
            q = []
            ol = []
            for ci, p in enumerate(pts):
                idx3 = _unlin(p, N)
                pred = _pred(T, xh, N, idx3, d, s, cubic)
                xv = flat[p]
                t = (xv - pred) * inv2eb
                code = 0
                rec = xv
                bad = not (abs(t) <= R)
                if not bad:
                    qf = T.t(np.rint(t))
                    rec = pred + qf * twoeb
                    if not (abs(xv - rec) <= ebchk):
                        bad = True
                    else:
                        code = int(qf)
                if bad:
                    code = 0
                    rec = xv
                    ol.append((ci, float(xv)))
                xh[p] = rec
                q.append(code)
            codes.append(q)
            outl.append(ol)
    # container
    hdr = struct.pack("<6I", 0x31435049, 1, 0 if T.is32 else 1, int(cubic), bound,
                      x.ndim)
    dims = list(x.shape) + [0] * (3 - x.ndim)
    hdr += struct.pack("<3Q", *dims)
    hdr += struct.pack("<2I", eb_mode, K)
    hdr += struct.pack("<6d", eb_user, eb, xmin, xmax, xmaxabs, float(flat[0]))
    hdr += struct.pack("<2I", len(st), 0)
    streams = []
    table = b""
    for si, (l, d, pts) in enumerate(st):
        q = codes[si]
        orv = 0
        for v in q:
            orv |= nb(v)
        H = orv.bit_length() - 1
        Q = max(abs(v) for v in q)
        ndim_off = 3 - x.ndim
        table += struct.pack("<IIQiIQ", l, d - ndim_off, len(q), H, Q, len(outl[si]))
        # rows of the lattice = runs of equal (i0, i1)
        rows = {}
        for ci, p in enumerate(pts):
            i0, i1, _ = _unlin(p, N)
            rows.setdefault((i0, i1), []).append(ci)
        row_list = [rows[k] for k in sorted(rows)]
        E = [xor_enc(nb(v)) for v in q]
        for k in range(31, -1, -1):
            words = []
            for r in row_list:
                for j in range(0, len(r), 32):
                    w = 0
                    for i, ci in enumerate(r[j:j + 32]):
                        w |= ((E[ci] >> k) & 1) << i
                    words.append(w)
            streams.append(_stream(words))
    sizes = b"".join(struct.pack("<Q", len(s)) for s in streams)
    outs = b"".join(struct.pack("<Qd", ci, v) for ol in outl for (ci, v) in ol)
    return hdr + table + sizes + outs + b"".join(streams), codes


def _stream(words):
    W = len(words)
    nz = [w for w in words if w]
    out = struct.pack("<I", len(nz))
    if not nz:
        return out
    nbm = (W + 31) // 32
    if nbm + len(nz) < W:
        for j in range(nbm):
            bits = 0
            for i in range(32):
                if 32 * j + i < W and words[32 * j + i]:
                    bits |= 1 << i
            out += struct.pack("<I", bits)
        out += b"".join(struct.pack("<I", w) for w in nz)
    else:
        out += b"".join(struct.pack("<I", w) for w in words)
    return out


def reconstruct(x_shape, dtype, codes, outliers, anchor, eb, b_per_level, cubic=True,
                xmaxabs=0.0):
    """Algorithm 1 from per-stage codes: drop b_l low planes at level l."""
    T = _T(dtype)
    N = padded(x_shape)
    n = N[0] * N[1] * N[2]
    out = [T.t(0)] * n
    out[0] = T.t(anchor)
    twoeb = T.t(2.0 * half_bin(eb, xmaxabs, T.is32))
    st, K = stages(x_shape)
    with np.errstate(all="ignore"):
        for si, (l, d, pts) in enumerate(st):
            s = 1 << (l - 1)
            b = b_per_level[l - 1]
            mask = 0 if b >= 32 else (0xFFFFFFFF >> b) << b
            ol = dict(outliers[si])
            for ci, p in enumerate(pts):
                if ci in ol:
                    out[p] = T.t(ol[ci])
                    continue
                idx3 = _unlin(p, N)
                pred = _pred(T, out, N, idx3, d, s, cubic)
                nprime = xor_dec(xor_enc(nb(codes[si][ci])) & mask) & mask
                qv = nb_value(nprime)
                out[p] = pred + T.t(qv) * twoeb
    return np.array(out, dtype=dtype).reshape(x_shape)
