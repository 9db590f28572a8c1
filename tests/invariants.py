"""Properties every correct MSz result has, whatever edits produced it
(Sec. 3 problem statement): the bound |f - g| <= xi, identical extremum
sets and identical max/min labels, and an edit list that is exactly the set
of changed vertices."""
from __future__ import annotations

from fractions import Fraction

import numpy as np

import oracle


def within_bound(f: np.ndarray, g: np.ndarray, xi: float) -> bool:
    dt = f.dtype.type
    X = float(dt(xi))
    if f.dtype == np.float32:
        d = np.abs(g.astype(np.float64) - f.astype(np.float64))  # exact for float32
        return bool((d <= X).all())
    d = np.abs(g.astype(np.longdouble) - f.astype(np.longdouble))
    near = np.flatnonzero(np.abs(d - np.longdouble(X)) <= np.longdouble(X) * 1e-9)
    ok = d <= np.longdouble(X)
    for i in near:
        ok.flat[i] = abs(Fraction(float(g.flat[i])) - Fraction(float(f.flat[i]))) <= Fraction(X)
    return bool(ok.all())


def bits_of(a: np.ndarray) -> np.ndarray:
    return a.reshape(-1).view(np.uint32 if a.dtype == np.float32 else np.uint64)


def check_result(f, fhat, xi, g, edit_idx, edit_val, label_max=None, label_min=None):
    """Assert the invariants; returns the oracle-computed labels of f."""
    assert within_bound(f, g, xi), "edited value outside the error bound"
    uf, df = oracle.directions(f)
    ug, dg = oracle.directions(g)
    n = f.size
    ar = np.arange(n)
    assert np.array_equal(uf == ar, ug == ar), "maximum sets differ"
    assert np.array_equal(df == ar, dg == ar), "minimum sets differ"
    M = oracle.labels(f.shape, uf)
    m = oracle.labels(f.shape, df)
    assert np.array_equal(oracle.labels(f.shape, ug), M), "maximum labels differ"
    assert np.array_equal(oracle.labels(f.shape, dg), m), "minimum labels differ"
    if label_max is not None:
        assert np.array_equal(np.asarray(label_max).reshape(-1), M)
    if label_min is not None:
        assert np.array_equal(np.asarray(label_min).reshape(-1), m)
    changed = np.flatnonzero(bits_of(g) != bits_of(fhat))
    assert np.array_equal(np.asarray(edit_idx, dtype=np.int64), changed), "edit list != changed set"
    assert np.array_equal(bits_of(np.asarray(edit_val, dtype=f.dtype)), bits_of(g)[changed])
    # every vertex either only decreased (Eq. 1) or was reset to f (freeze guard)
    gf, ff, hf = g.reshape(-1), f.reshape(-1), fhat.reshape(-1)
    assert ((gf <= hf) | (bits_of(g) == bits_of(f))).all()
    return M, m
