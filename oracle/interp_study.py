"""Study: how much a choice of interpolation per field, or per level, would
save over a fixed mode (the per-level and dimension-order tuning of the
QoZ line of interpolation compressors; the paper fixes cubic, Sec. 4.1).
For each workload the oracle compresses with each mode (linear, cubic,
cubic with quadratic boundaries) and prints the container bytes, the bytes
a retrieval at a looser target loads, and an estimate of what a per-level
choice could reach: the sum over levels of the smallest of the three
modes' stream bytes for that level (plus the smallest mandatory part). The
estimate treats levels as independent, which they nearly are: a level's
codes depend on the coarser levels only through reconstructions that
differ by at most the error bound. The second table compares the per-field choice (interp 3: the mode with
the smallest container on a sample) with the fixed cubic mode. The third
covers the order in which a level sweeps its
dimensions: compressing a transposed copy of a field sweeps its axes in the
permuted order, so each permutation (with each mode) is compressed and the
best is compared with the natural order's best. Oracle only (test
infrastructure):

    python -m oracle.interp_study
"""
import itertools
import time

import numpy as np

from oracle import oracle
from paper_2502_04093_gb300 import synth

MODES = (oracle.LINEAR, oracle.CUBIC, oracle.CUBIC_QUAD)


def workloads():
    grf = synth.grf_k53((128,) * 3, seed=1002).numpy()
    yield "k^-5/3 GRF 128^3 f32, eb 1e-6 abs", grf, 1e-6, oracle.ABS, 1e-3
    yield "k^-5/3 GRF 128^3 f32, eb 1e-3 abs", grf, 1e-3, oracle.ABS, 1e-1
    yield ("8 Gaussians + noise 64^3 f32, eb 1e-3 rel", synth.gaussians3d((64,) * 3, seed=1001),
           1e-3, oracle.REL, 1e-2)
    yield ("zonal 2-D 900x1800 f32, eb 1e-4 rel", synth.zonal2d((900, 1800), seed=1301),
           1e-4, oracle.REL, 1e-2)
    yield ("sinusoids 96x96x64 f64, eb 1e-8 rel", synth.sinusoids3d((96, 96, 64), seed=1401),
           1e-8, oracle.REL, 1e-4)
    yield ("white noise 64^3 f32, eb 1e-3 rel", synth.random_field((64,) * 3, 3, kind="noise"),
           1e-3, oracle.REL, 1e-2)
    yield ("smooth + rare spikes 64^3 f32, eb 1e-4 rel",
           synth.random_field((64,) * 3, 3, kind="spiky"), 1e-4, oracle.REL, 1e-2)


def level_bytes(f):
    """Stream bytes per level (index l, 1..K) and the mandatory bytes."""
    inf = f.info()
    by = np.zeros(inf["K"] + 1, dtype=np.int64)
    for t in range(inf["S"]):
        by[f.stage(t)["level"]] += sum(f.stream_size(t, k) for k in range(32))
    return by, inf["mandatory"]


def main():
    oracle.build()
    print("| workload | container bytes linear / cubic / quad | per-level estimate (vs best mode) "
          "| per-level best | retrieval at E: bytes linear / cubic / quad |")
    print("|---|---|---|---|---|")
    for name, x, eb, mode, E in workloads():
        t0 = time.perf_counter()
        tot, lev, mand, ret = [], [], [], []
        for m in MODES:
            f = oracle.compress(x, eb, mode, interp=m)
            tot.append(len(f.export()))
            lb, md = level_bytes(f)
            lev.append(lb)
            mand.append(md)
            ret.append(f.retrieve(oracle.EB, E)[1].selection()[1])
        est = int(np.minimum.reduce(lev).sum()) + min(mand)
        best = min(tot)
        pick = "".join("LCQ"[int(np.argmin([lb[l] for lb in lev]))] for l in range(len(lev[0]) - 1, 0, -1))
        print("| %s | %d / %d / %d | %d (%.2f %%) | %s | %g: %d / %d / %d |"
              % (name, tot[0], tot[1], tot[2], est, 100.0 * (best - est) / best, pick, E,
                 ret[0], ret[1], ret[2]))
        print("<!-- %s: %.1f s -->" % (name, time.perf_counter() - t0))
    print()
    print("| workload | mode chosen on the sample | container vs cubic | retrieval at E vs cubic |")
    print("|---|---|---|---|")
    for name, x, eb, mode, E in workloads():
        m = oracle.auto_interp(x, eb, mode)
        fa = oracle.compress(x, eb, mode, interp=oracle.AUTO)
        fc = oracle.compress(x, eb, mode, interp=oracle.CUBIC)
        ca, cc = len(fa.export()), len(fc.export())
        ra = fa.retrieve(oracle.EB, E)[1].selection()[1]
        rc = fc.retrieve(oracle.EB, E)[1].selection()[1]
        print("| %s | %s | %+.2f %% | %g: %+.2f %% |" % (name, "LCQ"[m], 100.0 * (ca - cc) / cc, E,
                                                        100.0 * (ra - rc) / rc))
    print()
    print("| workload | best (order, mode) by container | container below the natural order's best "
          "| retrieval at E below the natural order's best |")
    print("|---|---|---|---|")
    for name, x, eb, mode, E in workloads():
        rows = []
        for perm in itertools.permutations(range(x.ndim)):
            xp = np.ascontiguousarray(x.transpose(perm))
            for m in MODES:
                f = oracle.compress(xp, eb, mode, interp=m)
                rows.append((perm, m, len(f.export()), f.retrieve(oracle.EB, E)[1].selection()[1]))
        nat = [r for r in rows if r[0] == tuple(range(x.ndim))]
        c0, c1 = min(r[2] for r in nat), min(r[2] for r in rows)
        r0, r1 = min(r[3] for r in nat), min(r[3] for r in rows)
        best = min(rows, key=lambda r: r[2])
        print("| %s | %s, %s | %.2f %% | %g: %.2f %% |" % (name, best[0], "LCQ"[best[1]],
                                                          100.0 * (c0 - c1) / c0, E,
                                                          100.0 * (r0 - r1) / r0))


if __name__ == "__main__":
    main()
