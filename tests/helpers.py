"""Shared helpers of the CPU tests."""
import numpy as np

import pyref


def eb_for_bin(A: float, is32: bool, half: float = 0.25) -> float:
    """An error bound whose quantizer half bin (eb less the element-type
    rounding allowance 4u(A + eb)) is exactly `half` in the element type,
    found by stepping through neighbouring doubles."""
    u = 2.0 ** -24 if is32 else 2.0 ** -53
    eb = (half + 4 * u * A) / (1 - 4 * u)
    T = np.float32 if is32 else np.float64
    for _ in range(400):
        eq = pyref.half_bin(eb, A, is32)
        if T(2.0 * eq) == 2 * half and T(1.0 / (2.0 * eq)) == 1 / (2 * half):
            return eb
        eb = np.nextafter(eb, 1e300) if 2.0 * eq < 2 * half else np.nextafter(eb, 0.0)
    raise AssertionError("no eb with an exact bin")


def exact_eb(x: np.ndarray, half: float = 0.25) -> float:
    return eb_for_bin(float(np.abs(x[np.isfinite(x)]).max()), x.dtype == np.float32, half)
