"""Study: the closed-form bound on |q - q'_b| (U(b) up to a stage's top
digit H, then max|q|) against the data maximum over the stage's codes
(Sec. 5.1: precomputable during compression). For each workload and target
it prints the bytes the selection loads, its guaranteed bound and the
measured max error under both tables. Oracle only (test infrastructure):

    python -m oracle.delta_study
"""
import time

import numpy as np

from oracle import oracle
from paper_2502_04093_gb300 import synth


def workloads():
    yield ("k^-5/3 GRF 256^3 f32, eb 1e-6 abs", synth.grf_k53((256,) * 3, seed=1002).numpy(),
           1e-6, oracle.ABS, [1e-1, 1e-2, 1e-3, 1e-4, 1e-5])
    yield ("8 Gaussians + noise 64^3 f32, eb 1e-3 rel", synth.gaussians3d((64,) * 3, seed=1001),
           1e-3, oracle.REL, [1e-1, 1e-2])
    yield ("zonal 2-D 900x1800 f32, eb 1e-4 rel", synth.zonal2d((900, 1800), seed=1301),
           1e-4, oracle.REL, [1e-1, 1e-2, 1e-3])
    yield ("sinusoids 96x96x64 f64, eb 1e-8 rel", synth.sinusoids3d((96, 96, 64), seed=1401),
           1e-8, oracle.REL, [1e-2, 1e-4, 1e-6])


def main():
    oracle.build()
    print("| workload | E | bytes closed / data (saved) | bound closed / data | max err closed / data |")
    print("|---|---|---|---|---|")
    for name, x, eb, mode, targets in workloads():
        t0 = time.perf_counter()
        f = oracle.compress(x, eb, mode)
        xr = x.astype(np.float64)
        for E in targets:
            res = []
            for model in (0, 1):
                f.set_delta_model(model)
                y, v = f.retrieve(oracle.EB, E)
                _, by, g = v.selection()
                res.append((by, g, float(np.abs(y.astype(np.float64) - xr).max())))
            (b0, g0, e0), (b1, g1, e1) = res
            print("| %s | %g | %d / %d (%.1f %%) | %.3g / %.3g | %.3g / %.3g |"
                  % (name, E, b0, b1, 100.0 * (b0 - b1) / b0, g0, g1, e0, e1))
        f.set_delta_model(0)
        print("<!-- %s: %.1f s -->" % (name, time.perf_counter() - t0))


if __name__ == "__main__":
    main()
