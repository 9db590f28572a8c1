"""Full-size properties of the correction through msz_fix: the 512^3 float32
turbulence field the benchmark times (same generator, bounds and entry
point), the 3600 x 2400 ocean field and the 256^3 lognormal field. The
oracle would need many minutes per fix at these sizes, so the checks are the
properties every correct result has (Sec. 3 problem statement): the error
bound, an edit list equal to the set of changed vertices, identical
extremum sets of f and g (recomputed here with plain torch comparisons under
the (value, index) order), and, for sampled vertices, max/min labels that
agree with integral lines followed on the host in f and in g."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2406_09423_gb300 import synth

pytestmark = pytest.mark.gpu

POS3 = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)]  # (dx, dy, dz)
POS2 = [(1, 0, 0), (0, 1, 0), (1, 1, 0)]


def _msz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2406_09423_gb300 as msz

    return msz


def _vecs(nd):
    pos = POS3 if nd == 3 else POS2
    return pos + [(-a, -b, -c) for a, b, c in pos]


def _extrema(a):
    """Max / min flags of every vertex of a (torch, (nz, ny, nx) or (ny, nx))
    under u < v iff a_u < a_v or (a_u == a_v and index u < index v)."""
    a3 = a if a.dim() == 3 else a.unsqueeze(0)
    nz, ny, nx = a3.shape
    is_max = torch.ones_like(a3, dtype=torch.bool)
    is_min = torch.ones_like(a3, dtype=torch.bool)
    for dx, dy, dz in _vecs(a.dim()):
        def sl(d, n):  # (slice of v, slice of v + d) along one axis
            return (slice(0, n - 1), slice(1, n)) if d > 0 else ((slice(1, n), slice(0, n - 1)) if d < 0 else
                                                                  (slice(0, n), slice(0, n)))
        (vz, uz), (vy, uy), (vx, ux) = sl(dz, nz), sl(dy, ny), sl(dx, nx)
        av, au = a3[vz, vy, vx], a3[uz, uy, ux]
        later = dx + dy * nx + dz * nx * ny > 0  # the neighbour's index is the larger one
        above = (au > av) | ((au == av) & later)
        below = (au < av) | ((au == av) & (not later))
        is_max[vz, vy, vx] &= ~above
        is_min[vz, vy, vx] &= ~below
    return is_max.reshape(a.shape), is_min.reshape(a.shape)


def _walk(a, dims, starts, up):
    """Extremum reached from each start by steepest ascent (up) or descent in
    the flat host array a, one step per iteration for all starts at once."""
    nx, ny, nz, nd = dims
    cur = starts.astype(np.int64)
    vecs = _vecs(nd)
    while True:
        x, y, z = cur % nx, (cur // nx) % ny, cur // (nx * ny)
        best, bv = cur.copy(), a[cur]
        for dx, dy, dz in vecs:
            X, Y, Z = x + dx, y + dy, z + dz
            ok = (X >= 0) & (X < nx) & (Y >= 0) & (Y < ny) & (Z >= 0) & (Z < nz)
            u = np.where(ok, cur + dx + dy * nx + dz * nx * ny, cur)
            au = a[u]
            if up:
                better = ok & ((au > bv) | ((au == bv) & (u > best)))
            else:
                better = ok & ((au < bv) | ((au == bv) & (u < best)))
            best, bv = np.where(better, u, best), np.where(better, au, bv)
        if np.array_equal(best, cur):
            return cur
        cur = best


CASES = [
    ("turbulence512-1e-3", lambda: synth.turbulence3d(512, 3, device="cuda"), 1e-3),
    ("turbulence512-1e-5", lambda: synth.turbulence3d(512, 3, device="cuda"), 1e-5),
    ("ocean3600x2400-1e-3", lambda: synth.ocean2d(3600, 2400, 2, device="cuda"), 1e-3),
    ("lognormal256-1e-4", lambda: synth.lognormal3d(256, 1, device="cuda"), 1e-4),
]


@pytest.mark.parametrize("name,make,rel", CASES, ids=[c[0] for c in CASES])
def test_fullsize_properties(name, make, rel):
    msz = _msz()
    f = make().contiguous()
    xi = synth.xi_for(f, rel)
    fh = synth.quantise_torch(f, xi)
    plan = msz.Plan(tuple(f.shape), f.dtype)
    r = plan.fix(f, fh, xi)
    plan.close()
    assert r.status == 0
    # g = fhat with the edits applied (the decompression-side call)
    g = fh.clone()
    msz.apply(g, r.edit_idx, r.edit_val)
    # error bound, exactly (float32 differences are exact in float64)
    x32 = float(np.float32(xi))
    assert ((g.double() - f.double()).abs() <= x32).all()
    # the edit list is the set of changed vertices, ascending
    gi, hi, fi = g.view(torch.int32).reshape(-1), fh.view(torch.int32).reshape(-1), f.view(torch.int32).reshape(-1)
    changed = torch.nonzero(gi != hi).reshape(-1)
    assert torch.equal(r.edit_idx.reshape(-1).to(torch.int64), changed)
    # every edited vertex only decreased (Eq. 1) or was reset to f
    assert ((g.reshape(-1) <= fh.reshape(-1)) | (gi == fi)).all()
    # identical extremum sets
    fmax, fmin = _extrema(f)
    gmax, gmin = _extrema(g)
    assert torch.equal(fmax, gmax) and torch.equal(fmin, gmin)
    # labels of sampled vertices: the returned labels, and integral lines in f and g
    nd = f.dim()
    nz, ny, nx = (tuple(f.shape) if nd == 3 else (1,) + tuple(f.shape))
    dims = (nx, ny, nz, nd)
    rng = np.random.default_rng(11)
    starts = rng.integers(0, f.numel(), 2000)
    fh_, gh_ = f.reshape(-1).cpu().numpy(), g.reshape(-1).cpu().numpy()
    lmax = r.label_max.reshape(-1).cpu().numpy().astype(np.int64)
    lmin = r.label_min.reshape(-1).cpu().numpy().astype(np.int64)
    for up, lab in ((True, lmax), (False, lmin)):
        wf = _walk(fh_, dims, starts, up)
        wg = _walk(gh_, dims, starts, up)
        assert np.array_equal(wf, wg), "labels of g differ from those of f"
        assert np.array_equal(lab[starts], wg), "returned labels differ from the integral lines"
