"""Pins for the oracle's mesh, order, directions and labels (Sec. 3).

Each check compares the oracle with a formulation written independently
from the definitions: pairwise edge tests, closed-form edge counts and the
Euler characteristic of the triangulated square, tuple-ordered brute force
and plain integral-line walks, and closed forms (ramps, single bumps).
"""
import numpy as np
import pytest

import oracle
from tests import bruteforce as bf

SHAPES_2D = [(1, 1), (1, 5), (4, 1), (2, 2), (3, 3), (4, 7), (6, 5)]
SHAPES_3D = [(1, 1, 1), (2, 2, 2), (3, 3, 3), (2, 3, 4), (4, 3, 2), (5, 1, 3)]


@pytest.mark.parametrize("shape", SHAPES_2D + SHAPES_3D)
def test_neighbours_match_pairwise_freudenthal(shape):
    adj = bf.adjacency(shape)
    for v in range(len(adj)):
        assert sorted(oracle.neighbours(shape, v)) == sorted(adj[v])


def _edges_closed_form(shape):
    if len(shape) == 2:
        ny, nx = shape
        return (nx - 1) * ny + nx * (ny - 1) + (nx - 1) * (ny - 1)
    nz, ny, nx = shape
    a, b, c = nx - 1, ny - 1, nz - 1
    return (a * ny * nz + nx * b * nz + nx * ny * c          # axis edges
            + a * b * nz + a * ny * c + nx * b * c           # face diagonals (+,+)
            + a * b * c)                                     # body diagonal


@pytest.mark.parametrize("shape", SHAPES_2D + SHAPES_3D + [(9, 11), (5, 6, 7)])
def test_edge_count_closed_form(shape):
    n = int(np.prod(shape))
    deg = sum(len(oracle.neighbours(shape, v)) for v in range(n))
    assert deg % 2 == 0
    assert deg // 2 == _edges_closed_form(shape)


@pytest.mark.parametrize("shape", [(2, 2), (3, 4), (7, 5), (10, 10)])
def test_2d_triangulation_euler_characteristic(shape):
    # A triangulated rectangle is a disk: V - E + F = 1, where the faces are
    # the triangles {v, v+e1, v+e1+e2} of every cell (two per cell).
    ny, nx = shape
    n = nx * ny
    adj = {v: set(oracle.neighbours(shape, v)) for v in range(n)}
    edges = sum(len(s) for s in adj.values()) // 2
    tri = 0
    for v in range(n):
        for u in adj[v]:
            for w in adj[u] & adj[v]:
                if v < u < w:
                    tri += 1
    assert tri == 2 * (nx - 1) * (ny - 1)
    assert n - edges + tri == 1


def _random_field(rng, shape, dtype, ties):
    if ties:
        return rng.integers(0, 4, shape).astype(dtype)  # heavy plateaus: SoS decides
    return rng.standard_normal(shape).astype(dtype)


@pytest.mark.parametrize("shape", SHAPES_2D + SHAPES_3D + [(8, 9), (4, 5, 6)])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("ties", [False, True])
def test_directions_match_bruteforce(shape, dtype, ties):
    rng = np.random.default_rng(hash((shape, ties)) & 0xFFFF)
    adj = bf.adjacency(shape)
    for _ in range(3):
        g = _random_field(rng, shape, dtype, ties)
        up, dn = oracle.directions(g)
        bup, bdn = bf.directions(g, adj)
        assert list(up) == bup
        assert list(dn) == bdn


def test_signed_zero_compares_equal():
    # -0 == +0 under IEEE comparison, so the index decides.
    g = np.array([[0.0, -0.0, 0.0]], dtype=np.float32)
    up, dn = oracle.directions(g)
    assert list(up) == [1, 2, 2]
    assert list(dn) == [0, 0, 1]


def test_hand_worked_3x3_plateau():
    # g (rows are y, x fastest):  1 1 0 / 1 2 1 / 0 1 1.  The centre is the
    # only maximum. Vertex 0 lies on a plateau of 1s with its neighbours 1
    # and 3; the index breaks the tie, so vertex 0 is a minimum, and vertex 8
    # descends to 5, the lowest-indexed of its equal neighbours 5 and 7.
    g = np.array([[1, 1, 0], [1, 2, 1], [0, 1, 1]], dtype=np.float32)
    up, dn = oracle.directions(g)
    assert list(up) == [4, 4, 5, 4, 4, 4, 7, 4, 4]
    assert list(dn) == [0, 2, 2, 6, 0, 2, 6, 6, 5]
    assert list(oracle.labels(g.shape, up)) == [4] * 9
    assert list(oracle.labels(g.shape, dn)) == [0, 2, 2, 6, 0, 2, 6, 6, 2]


def test_hand_worked_2x2x2_cube():
    # Freudenthal cube: 0 and 7 touch every vertex, the others four each.
    # Vertex 5 (value 6) is a maximum beside the global maximum 3 (value 7)
    # because 3 and 5 differ by (0, -1, 1) and share no edge.
    g = np.array([3, 5, 1, 7, 2, 6, 0, 4], dtype=np.float64).reshape(2, 2, 2)
    assert [sorted(oracle.neighbours(g.shape, v)) for v in range(8)] == [
        [1, 2, 3, 4, 5, 6, 7], [0, 3, 5, 7], [0, 3, 6, 7], [0, 1, 2, 7],
        [0, 5, 6, 7], [0, 1, 4, 7], [0, 2, 4, 7], [0, 1, 2, 3, 4, 5, 6]]
    up, dn = oracle.directions(g)
    assert list(up) == [3, 3, 3, 3, 5, 5, 7, 3]
    assert list(dn) == [6, 0, 6, 2, 6, 4, 6, 6]
    assert list(oracle.labels(g.shape, up)) == [3, 3, 3, 3, 5, 5, 3, 3]
    assert list(oracle.labels(g.shape, dn)) == [6] * 8


@pytest.mark.parametrize("shape", SHAPES_2D + SHAPES_3D + [(8, 9), (4, 5, 6)])
@pytest.mark.parametrize("ties", [False, True])
def test_labels_match_walks(shape, ties):
    rng = np.random.default_rng(7 + len(shape))
    adj = bf.adjacency(shape)
    for _ in range(3):
        g = _random_field(rng, shape, np.float64, ties)
        bup, bdn = bf.directions(g, adj)
        assert list(oracle.labels(shape, np.array(bup))) == bf.walk_labels(bup)
        assert list(oracle.labels(shape, np.array(bdn))) == bf.walk_labels(bdn)


@pytest.mark.parametrize("shape", [(5, 7), (3, 4, 5), (16, 16), (6, 6, 6)])
def test_ramp_has_one_max_and_one_min(shape):
    # f = linear index (and a constant field, where the index order decides)
    # is strictly increasing along +x, +y, +z: the only maximum is the last
    # vertex, the only minimum the first, and every label points there.
    n = int(np.prod(shape))
    for f in (np.arange(n, dtype=np.float64).reshape(shape), np.zeros(shape)):
        up, dn = oracle.directions(f)
        M = oracle.labels(shape, up)
        m = oracle.labels(shape, dn)
        assert set(np.flatnonzero(up == np.arange(n))) == {n - 1}
        assert set(np.flatnonzero(dn == np.arange(n))) == {0}
        assert (M == n - 1).all() and (m == 0).all()


def test_single_bump_has_one_maximum():
    y, x = np.mgrid[0:21, 0:25]
    f = np.exp(-((x - 11.3) ** 2 + (y - 9.6) ** 2) / 30.0)
    up, dn = oracle.directions(f)
    maxs = np.flatnonzero(up == np.arange(f.size))
    assert list(maxs) == [int(np.argmax(f))]
    assert (oracle.labels(f.shape, up) == maxs[0]).all()


@pytest.mark.parametrize("shape", [(3, 3), (4, 4), (2, 2, 3)])
def test_false_bits_are_set_differences(shape):
    rng = np.random.default_rng(11)
    adj = bf.adjacency(shape)
    for _ in range(20):
        f = rng.standard_normal(shape)
        g = f + rng.normal(0, 0.7, shape)
        fu, fd = bf.directions(f, adj)
        gu, gd = bf.directions(g, adj)
        fmax, fmin = bf.extrema(fu, fd)
        gmax, gmin = bf.extrema(gu, gd)
        bits = oracle.false_bits(f, g)
        assert set(np.flatnonzero(bits & 1)) == gmax - fmax
        assert set(np.flatnonzero(bits & 2)) == gmin - fmin
        assert set(np.flatnonzero(bits & 4)) == fmax - gmax
        assert set(np.flatnonzero(bits & 8)) == fmin - gmin
