"""Exact rational helpers for pinning floating-point steps."""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def frac(x) -> Fraction:
    return Fraction(float(x))


def rn(value: Fraction, dtype) -> float:
    """Round a rational to the nearest value of ``dtype`` (ties to even),
    decided exactly by comparing rational distances to the two neighbours."""
    dt = np.dtype(dtype).type
    c = dt(float(value))  # within one ulp of the answer
    cands = {c, np.nextafter(c, dt(np.inf)), np.nextafter(c, dt(-np.inf))}
    best = None
    for q in cands:
        if not np.isfinite(q):
            continue
        d = abs(Fraction(float(q)) - value)
        if best is None or d < best[0]:
            best = (d, q)
        elif d == best[0]:
            # tie: choose the even significand
            bits_new = np.array([q], dtype=dt).view(np.uint32 if dt == np.float32 else np.uint64)[0]
            if int(bits_new) % 2 == 0:
                best = (d, q)
    return best[1]
