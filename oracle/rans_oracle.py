"""Plain-Python restatement of the library's lossless stage (test
infrastructure, like the rest of oracle/): the coded container format and
its order-0 rANS, written from the definitions, one symbol at a time.

The lossless stage stands where the paper runs zstd after predictive coding
(Sec. 6.2.1). Its definition is the identity decode(encode(x)) == x; the
format (block table, frequency normalisation, state interval) is this
build's own and is fixed here independently of the C++ implementation so
that the two can be checked against each other byte for byte.

Range asymmetric numeral systems (Duda, 2013): a state x in [L, 256 L)
with L = 2^23 codes a symbol s of frequency f_s (of M = 4096) starting at
cumulative c_s as x' = floor(x / f_s) * M + (x mod f_s) + c_s, after
shifting out low bytes of x while x >= 2^15 f_s (so that x' < 2^31); the
decoder inverts it: s is the symbol whose range holds x mod M, x =
f_s * floor(x / M) + (x mod M) - c_s, then bytes are shifted in while
x < L. Symbols are coded last to first, so they decode first to last.

Version 2 records (mode 2) run two such states that take the symbols in
turn, symbol i with state i mod 2, over one shared byte stream
(interleaved rANS, Giesen 2014): the encoder walks the symbols backwards,
each step shifting bytes out of its own state; the stream starts with the
final states 0 and 1, and the decoder, walking forwards, reads each
symbol's bytes into the state that decoded it. Version 1 records (mode 1)
have one state; both versions are read.
"""
MAGIC = 0x5A435049  # "IPCZ"
VERSION = 2
SCALE = 12
M = 1 << SCALE
L = 1 << 23


class CodecError(ValueError):
    pass


def frequencies(block: bytes):
    """Counts scaled to M: absent bytes 0, present ones max(1, floor(c M / n));
    then one unit at a time to (or from) the largest frequency, the lowest
    byte value first on ties, never below 1."""
    n = len(block)
    c = [0] * 256
    for v in block:
        c[v] += 1
    f = [0 if c[s] == 0 else max(1, c[s] * M // n) for s in range(256)]
    total = sum(f)
    while total < M:
        s = max(range(256), key=lambda k: (f[k], -k))
        f[s] += 1
        total += 1
    while total > M:
        s = max((k for k in range(256) if f[k] > 1), key=lambda k: (f[k], -k))
        f[s] -= 1
        total -= 1
    return f


def encode_block(block: bytes, nstates: int = 2) -> bytes:
    f = frequencies(block)
    cum = [0] * 256
    for s in range(1, 256):
        cum[s] = cum[s - 1] + f[s - 1]
    out = bytearray()  # emitted bytes, in emission order (reversed below)
    x = [L] * nstates
    for i in range(len(block) - 1, -1, -1):
        v = block[i]
        j = i % nstates
        while x[j] >= ((L >> SCALE) << 8) * f[v]:
            out.append(x[j] & 0xFF)
            x[j] >>= 8
        x[j] = (x[j] // f[v]) * M + (x[j] % f[v]) + cum[v]
    stream = b"".join(xj.to_bytes(4, "little") for xj in x) + bytes(reversed(out))
    if 1 + 512 + len(stream) >= 1 + len(block):
        return b"\x00" + bytes(block)
    table = b"".join(fs.to_bytes(2, "little") for fs in f)
    return bytes([nstates]) + table + stream


def decode_block(rec: bytes, n: int) -> bytes:
    if not rec:
        raise CodecError("empty record")
    if rec[0] == 0:
        if len(rec) != 1 + n:
            raise CodecError("stored record size")
        return bytes(rec[1:])
    nstates = rec[0]
    if nstates not in (1, 2) or len(rec) < 1 + 512 + 4 * nstates:
        raise CodecError("record mode")
    f = [int.from_bytes(rec[1 + 2 * s:3 + 2 * s], "little") for s in range(256)]
    if sum(f) != M:
        raise CodecError("frequency sum")
    cum = [0] * 256
    for s in range(1, 256):
        cum[s] = cum[s - 1] + f[s - 1]
    sym = []
    for s in range(256):
        sym += [s] * f[s]
    p = 1 + 512
    x = [int.from_bytes(rec[p + 4 * j:p + 4 * j + 4], "little") for j in range(nstates)]
    p += 4 * nstates
    out = bytearray()
    for i in range(n):
        j = i % nstates
        slot = x[j] % M
        s = sym[slot]
        out.append(s)
        x[j] = f[s] * (x[j] // M) + slot - cum[s]
        while x[j] < L:
            if p >= len(rec):
                raise CodecError("stream overrun")
            x[j] = (x[j] << 8) | rec[p]
            p += 1
    if p != len(rec) or any(xj != L for xj in x):
        raise CodecError("stream does not end in the initial states")
    return bytes(out)


def encode(raw: bytes, block_log2: int = 20, version: int = VERSION) -> bytes:
    """Version 2 (two states per record), or version 1 (one state) as
    earlier containers hold."""
    bs = 1 << block_log2
    blocks = [raw[i:i + bs] for i in range(0, len(raw), bs)]
    recs = [encode_block(b, nstates=2 if version == 2 else 1) for b in blocks]
    head = (MAGIC.to_bytes(4, "little") + version.to_bytes(4, "little") +
            len(raw).to_bytes(8, "little") + block_log2.to_bytes(4, "little") +
            len(blocks).to_bytes(4, "little"))
    return head + b"".join(len(r).to_bytes(4, "little") for r in recs) + b"".join(recs)


def decode(coded: bytes) -> bytes:
    if len(coded) < 24 or int.from_bytes(coded[0:4], "little") != MAGIC or \
            int.from_bytes(coded[4:8], "little") not in (1, 2):
        raise CodecError("header")
    n = int.from_bytes(coded[8:16], "little")
    lg = int.from_bytes(coded[16:20], "little")
    nb = int.from_bytes(coded[20:24], "little")
    if not 12 <= lg <= 26:
        raise CodecError("block size")
    bs = 1 << lg
    if nb != (n + bs - 1) // bs or 24 + 4 * nb > len(coded):
        raise CodecError("block count")
    sizes = [int.from_bytes(coded[24 + 4 * i:28 + 4 * i], "little") for i in range(nb)]
    pos = 24 + 4 * nb
    if pos + sum(sizes) != len(coded):
        raise CodecError("block sizes")
    out = bytearray()
    for i, sz in enumerate(sizes):
        out += decode_block(coded[pos:pos + sz], min(bs, n - i * bs))
        pos += sz
    return bytes(out)
