"""Pins of the oracle's evaluation metrics (Appendix B: PSNR and the right
labelled ratio) against closed forms and brute-force label walks."""
import itertools
import math

import numpy as np
import pytest

import oracle


def _ring(shape, v):
    """Closed 1-ring of v in the Freudenthal mesh: v and v +- e for every
    nonzero e in {0,1}^d that stays in the grid (numpy shape, x fastest)."""
    dims = list(shape)[::-1]  # (nx, ny[, nz])
    d = len(dims)
    c = []
    t = v
    for n in dims:
        c.append(t % n)
        t //= n
    out = [v]
    for e in itertools.product((0, 1), repeat=d):
        if not any(e):
            continue
        for s in (1, -1):
            q = [c[k] + s * e[k] for k in range(d)]
            if all(0 <= q[k] < dims[k] for k in range(d)):
                idx, mul = 0, 1
                for k in range(d):
                    idx += q[k] * mul
                    mul *= dims[k]
                out.append(idx)
    return out


def _labels_brute(a):
    """Maximum / minimum label of every vertex by walking to the (value,
    index)-greatest / -least vertex of the closed ring until it is the vertex
    itself."""
    flat = a.ravel()
    key = lambda u: (float(flat[u]), u)
    up, dn = [], []
    for v in range(flat.size):
        u = v
        while True:
            w = max(_ring(a.shape, u), key=key)
            if w == u:
                break
            u = w
        up.append(u)
        u = v
        while True:
            w = min(_ring(a.shape, u), key=key)
            if w == u:
                break
            u = w
        dn.append(u)
    return np.array(up), np.array(dn)


def test_identical_fields():
    rng = np.random.default_rng(0)
    f = rng.standard_normal((9, 11)).astype(np.float32)
    m = oracle.metrics(f, f)
    assert m["mse"] == 0.0 and m["psnr"] == math.inf
    assert m["wrong"] == 0 and m["right_labelled"] == 1.0
    assert m["value_range"] == float(f.max()) - float(f.min())


def test_exact_shift_closed_form():
    # integer values + 0.5 are exact in float32 and keep the order, so the
    # labels agree, mse = 0.25 and psnr = 20 log10(range / 0.5)
    rng = np.random.default_rng(1)
    f = rng.integers(-1000, 1000, size=(5, 6, 7)).astype(np.float32)
    g = f + np.float32(0.5)
    m = oracle.metrics(f, g)
    assert m["mse"] == 0.25
    r = float(f.max()) - float(f.min())
    assert m["value_range"] == r
    assert m["psnr"] == pytest.approx(20.0 * math.log10(r / 0.5), rel=1e-15)
    assert m["wrong"] == 0


def test_single_vertex_change_closed_form():
    f = np.linspace(0.0, 1.0, 64, dtype=np.float64).reshape(8, 8)
    g = f.copy()
    g[3, 4] += 0.25
    m = oracle.metrics(f, g)
    assert m["mse"] == pytest.approx(0.0625 / 64, rel=1e-15)
    assert m["psnr"] == pytest.approx(20.0 * math.log10(1.0 / math.sqrt(0.0625 / 64)), rel=1e-14)


@pytest.mark.parametrize("shape,seed", [((4, 5), 2), ((6, 3), 3), ((3, 3, 3), 4), ((2, 4, 3), 5)])
def test_wrong_labels_match_brute_force(shape, seed):
    rng = np.random.default_rng(seed)
    f = rng.integers(0, 6, size=shape).astype(np.float32)  # ties, resolved by index
    g = f + rng.integers(-2, 3, size=shape).astype(np.float32)
    uf, df = _labels_brute(f)
    ug, dg = _labels_brute(g)
    wrong = int(np.count_nonzero((uf != ug) | (df != dg)))
    m = oracle.metrics(f, g)
    assert m["wrong"] == wrong
    assert m["right_labelled"] == 1.0 - wrong / f.size
