"""Helpers shared by the GPU parity tests."""
import math

import numpy as np

# Float SUM/AVG pass bar: |got - ref| <= 1e-6 * max(|ref|, 2^-24 * sum|x|).
# The second term only matters for groups whose sum cancels to far below the
# magnitude of their items, where a relative bar on |ref| is meaningless.
FP_REL = 1e-6


def fp_close(got: float, ref: float, abs_sum: float) -> bool:
    if math.isnan(ref):
        return math.isnan(got)
    return abs(got - ref) <= FP_REL * max(abs(ref), 2.0 ** -24 * abs_sum)


def rel_err(got: float, ref: float) -> float:
    if ref == 0:
        return abs(got)
    return abs(got - ref) / abs(ref)


def same_float(a: float, b: float) -> bool:
    """Bit-identical floats (so -0.0 != +0.0)."""
    return np.float64(a).tobytes() == np.float64(b).tobytes()
