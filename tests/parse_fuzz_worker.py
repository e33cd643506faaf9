"""Child process of test_parse_fuzz.py: seeded mutations of oracle
containers and coded containers fed to the host-side parsers. Prints the
count of accepted and refused inputs; a crash ends the process."""
import os
import random
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import oracle  # noqa: E402
from paper_2502_04093_gb300 import ipc, synth  # noqa: E402


def mutate(rng, b):
    b = bytearray(b)
    k = rng.randrange(6)
    if k == 0 and b:  # a few random bytes
        for _ in range(rng.randint(1, 8)):
            b[rng.randrange(len(b))] = rng.randrange(256)
    elif k == 1 and b:  # one bit
        b[rng.randrange(len(b))] ^= 1 << rng.randrange(8)
    elif k == 2:  # truncation
        b = b[:rng.randrange(len(b) + 1)]
    elif k == 3:  # insertion
        i = rng.randrange(len(b) + 1)
        b[i:i] = bytes(rng.randrange(256) for _ in range(rng.randint(1, 16)))
    elif k == 4 and len(b) >= 8:  # an extreme 32-bit field in the tables
        i = rng.randrange(0, min(len(b) - 4, 400))
        b[i:i + 4] = rng.choice([b"\xff\xff\xff\xff", b"\x00\x00\x00\x80", b"\x00\x00\x00\x00",
                                 b"\xff\xff\xff\x7f"])
    elif len(b) >= 8:  # a random 64-bit field in the header
        i = rng.randrange(0, min(len(b) - 7, 200))
        b[i:i + 8] = rng.randrange(1 << 64).to_bytes(8, "little")
    return bytes(b)


def main(seed, iters):
    oracle.build()
    rng = random.Random(seed)
    bases = []
    for shape, kind, interp in (((20, 17, 9), "smooth", 1), ((33, 40), "spiky", 0),
                                ((100,), "noise", 2), ((5, 6, 7), "smooth", 2)):
        x = synth.random_field(shape, seed=len(shape) + seed, kind=kind)
        bases.append(oracle.compress(x, 1e-4, oracle.REL, interp=interp).export())
    coded = [ipc.ipc_encode_container(b, block_log2=12) for b in bases]
    ok = err = 0
    for _ in range(iters):
        j = rng.randrange(len(bases))
        m = mutate(rng, bases[j])
        calls = [
            lambda: ipc.ipc_select_container(m, rng.choice([0, 1]),
                                             rng.choice([1e-3, 1e-1, 4.0, 1e-9, 0.0, -1.0,
                                                         float("nan")])),
            lambda: ipc.ipc_container_ranges(
                m, [rng.randrange(-2, 35) for _ in range(rng.randint(0, 12))]),
            lambda: ipc.ipc_decode_container(mutate(rng, coded[j]), nthreads=1),
        ]
        for call in calls:
            try:
                call()
                ok += 1
            except ipc.IpcError:
                err += 1
    print(ok, err)


if __name__ == "__main__":
    main(int(sys.argv[1]), int(sys.argv[2]))
