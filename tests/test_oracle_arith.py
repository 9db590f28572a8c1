"""Pins for the oracle's error-bound arithmetic (Sec. 3 constraint
|f - g| <= xi; Eq. (1) lower bound f - xi; Eqs. (2)-(6) halving step),
checked with exact rational arithmetic."""
import numpy as np
import pytest

import oracle
from tests.exact import frac, rn

DTYPES = [np.float32, np.float64]


def _samples(dtype, rng, n=400):
    fi = np.finfo(dtype)
    vals = list(rng.standard_normal(n // 2) * 10.0) + list(rng.uniform(-1e-3, 1e-3, n // 4))
    vals += [0.0, -0.0, 1.0, -1.0, fi.tiny, -fi.tiny, fi.tiny * 0.5, fi.eps, 1e30, -1e30,
             float(fi.smallest_subnormal), 3 * float(fi.smallest_subnormal)]
    return np.array(vals, dtype=dtype)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("xi", [0.0, 1e-7, 0.1, 0.3, 1.0, 1e-40, 12345.678])
def test_bounds_are_tightest_representable(dtype, xi):
    rng = np.random.default_rng(3)
    f = _samples(dtype, rng)
    xi_eff = dtype(xi)
    lb, ub = oracle.bounds(f, xi)
    X = frac(xi_eff)
    for fv, l, u in zip(f, lb, ub):
        lo = frac(fv) - X
        hi = frac(fv) + X
        assert frac(l) >= lo
        assert frac(np.nextafter(l, dtype(-np.inf))) < lo
        assert frac(u) <= hi
        assert frac(np.nextafter(u, dtype(np.inf))) > hi


@pytest.mark.parametrize("dtype", DTYPES)
def test_decrease_is_rounded_midpoint_or_snaps(dtype):
    rng = np.random.default_rng(5)
    lb = (rng.standard_normal(3000) * 4).astype(dtype)
    gap = np.abs(rng.standard_normal(3000)).astype(dtype) * dtype(10.0) ** rng.integers(-8, 3, 3000).astype(dtype)
    g = (lb + gap).astype(dtype)
    # include adjacent floats (no representable midpoint -> snap to lb)
    lb2 = (rng.standard_normal(200) * 4).astype(dtype)
    g2 = np.nextafter(lb2, dtype(np.inf))
    g = np.concatenate([g, g2]).astype(dtype)
    lb = np.concatenate([lb, lb2]).astype(dtype)
    keep = g > lb
    g, lb = g[keep], lb[keep]
    out = oracle.decrease(g, lb)
    for gv, lv, mv in zip(g, lb, out):
        assert frac(lv) <= frac(mv) < frac(gv)
        mid = rn((frac(gv) + frac(lv)) / 2, dtype)
        expect = mid if frac(mid) < frac(gv) else lv
        assert frac(mv) == frac(expect)


@pytest.mark.parametrize("dtype", DTYPES)
def test_decrease_subnormal_range_stays_in_interval(dtype):
    s = float(np.finfo(dtype).smallest_subnormal)
    lb = np.array([k * s for k in (1, 3, 5, -1, -3, 0)], dtype=dtype)
    g = np.array([k * s for k in (2, 4, 6, 0, 1, 1)], dtype=dtype)
    out = oracle.decrease(g, lb)
    assert (out >= lb).all() and (out < g).all()


@pytest.mark.parametrize("dtype", DTYPES)
def test_repeated_decrease_reaches_lb_in_finite_steps(dtype):
    # Eq. (1): values decrease monotonically towards the lower bound; in
    # floating point the sequence reaches lb after finitely many halvings.
    g = np.array([1.0, 1e6, -3.0, 0.5], dtype=dtype)
    lb = np.array([-1.0, 0.0, -3.5, 0.25], dtype=dtype)
    for _ in range(2000):
        nxt = oracle.decrease(g, lb)
        nxt = np.where(g > lb, nxt, g)
        assert (nxt <= g).all()
        g = nxt
        if (g == lb).all():
            break
    assert (g == lb).all()
