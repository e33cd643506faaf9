"""Oracle work run in spawned worker processes by the full-size GPU tests
(no torch here, so a worker starts quickly). Each job returns digests of
the oracle's container and reconstructions, and its selections."""
import hashlib

import numpy as np

from oracle import oracle


def _digest(a) -> str:
    return hashlib.sha256(a.tobytes() if isinstance(a, np.ndarray) else a).hexdigest()


def compress_retrieve(job):
    """(x, eb, eb_mode, [(kind, value)]) -> (container digest, [(selection,
    output digest)]), kind 0 = eb, 1 = bitrate."""
    x, eb, mode, targets = job
    f = oracle.compress(x, eb, mode)
    out = []
    for kind, v in targets:
        y, view = f.retrieve(kind, v)
        out.append((view.selection()[0], _digest(y)))
    return _digest(f.export()), out


def compress_refine_chain(job):
    """(x, eb, eb_mode, [E0, E1, ...]) -> (container digest, [selection after
    each step], digest of the final reconstruction): retrieve at E0, then
    refine to E1, E2, ..."""
    x, eb, mode, chain = job
    f = oracle.compress(x, eb, mode)
    y, view = f.retrieve(oracle.EB, chain[0])
    sels = [view.selection()[0]]
    for E in chain[1:]:
        y = view.refine(oracle.EB, E)
        sels.append(view.selection()[0])
    return _digest(f.export()), sels, _digest(y)


def compress_delta_chain(job):
    """(x, eb, eb_mode, [(kind, value), ...]) -> (container digest, [(selection,
    incremental, bound, output digest) per step]): retrieve at the first
    target, then refine incrementally (Algorithm 2) to the others."""
    x, eb, mode, chain = job
    f = oracle.compress(x, eb, mode)
    y, view = f.retrieve(*chain[0])
    sel, _, bound = view.selection()
    steps = [(sel, False, bound, _digest(y))]
    for kind, v in chain[1:]:
        y, inc = view.refine_delta(kind, v)
        sel, _, bound = view.selection()
        steps.append((sel, inc, bound, _digest(y)))
    return _digest(f.export()), steps
