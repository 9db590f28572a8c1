"""Pure-Python brute-force restatements used to pin the oracle on tiny grids.

They are written from the definitions independently of the oracle's C++:
adjacency is decided pairwise from the difference vector, the order is
Python tuple comparison of (value, index), labels are plain walks.
"""
from __future__ import annotations

import numpy as np


def coords(shape):
    """All vertex coordinates (x, y[, z]) in linear-index order (x fastest);
    ``shape`` is the numpy shape (ny, nx) or (nz, ny, nx)."""
    return _coords(tuple(shape)[::-1])


def _coords(rev):
    # rev = (nx, ny[, nz]); linear index = x + nx*(y + ny*z)
    if len(rev) == 2:
        nx, ny = rev
        return [(x, y) for y in range(ny) for x in range(nx)]
    nx, ny, nz = rev
    return [(x, y, z) for z in range(nz) for y in range(ny) for x in range(nx)]


def adjacent(a, b):
    """Freudenthal edge test: b - a is a nonzero vector of {0,1}^d or its negation."""
    d = tuple(bi - ai for ai, bi in zip(a, b))
    if all(c == 0 for c in d):
        return False
    return all(c in (0, 1) for c in d) or all(c in (0, -1) for c in d)


def adjacency(shape):
    cs = coords(shape)
    n = len(cs)
    return [[u for u in range(n) if adjacent(cs[v], cs[u])] for v in range(n)]


def directions(g: np.ndarray, adj=None):
    flat = [float(x) for x in np.asarray(g).reshape(-1)]
    adj = adj if adj is not None else adjacency(np.asarray(g).shape)
    up, dn = [], []
    for v, nb in enumerate(adj):
        ring = [v] + nb
        up.append(max(ring, key=lambda u: (flat[u], u)))
        dn.append(min(ring, key=lambda u: (flat[u], u)))
    return up, dn


def walk_labels(direction):
    out = []
    for v in range(len(direction)):
        w = v
        while direction[w] != w:
            w = direction[w]
        out.append(w)
    return out


def extrema(up, dn):
    maxs = {v for v, u in enumerate(up) if u == v}
    mins = {v for v, d in enumerate(dn) if d == v}
    return maxs, mins
