"""Parity of the CUDA path (through the C ABI) with the CPU oracle: bit-exact
directions, edited values, edit lists, labels and counters (the method's
floating-point tolerance is 0 ulp), on seeded inputs with several tiles and
ragged tails, degenerate shapes and the error paths."""
import glob
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2406_09423_gb300 import synth
from tests.invariants import bits_of, check_result

pytestmark = pytest.mark.gpu

SLOTS3 = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)]
SLOTS2 = [(1, 0), (0, 1), (1, 1)]


def _msz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2406_09423_gb300 as msz

    return msz


def decode(dirs: np.ndarray, shape):
    """Slot bytes -> (up, dn) vertex indices (x fastest)."""
    nd = len(shape)
    dims = list(shape)[::-1]
    vecs = SLOTS3 if nd == 3 else SLOTS2
    strides = [1, dims[0], dims[0] * dims[1]][:nd]
    offs = [sum(c * s for c, s in zip(e, strides)) for e in vecs]
    table = np.zeros(16, dtype=np.int64)
    table[: len(offs)] = offs
    table[len(offs): 2 * len(offs)] = [-o for o in offs]
    d = dirs.reshape(-1).astype(np.int64)
    v = np.arange(d.size)
    return v + table[d & 15], v + table[d >> 4]


def _field(kind, shape, dtype, seed):
    rng = np.random.default_rng(seed)
    if kind == "noise":
        return rng.standard_normal(shape).astype(dtype)
    if kind == "ties":
        return rng.integers(0, 4, shape).astype(dtype)
    if kind == "smooth":
        a = rng.standard_normal(shape)
        for ax in range(len(shape)):
            a = np.cumsum(a, axis=ax)
        return a.astype(dtype)
    raise KeyError(kind)


DIR_SHAPES = [(1, 1), (1, 7), (9, 1), (2, 2), (37, 23), (130, 257), (1, 1, 1), (2, 2, 2), (5, 1, 3),
              (19, 17, 33), (40, 36, 65)]


@pytest.mark.parametrize("shape", DIR_SHAPES)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("kind", ["noise", "ties"])
def test_directions_match_oracle(shape, dtype, kind):
    msz = _msz()
    g = _field(kind, shape, dtype, 17)
    d = msz.directions(torch.from_numpy(g).cuda()).cpu().numpy()
    up, dn = decode(d, shape)
    oup, odn = oracle.directions(g)
    assert np.array_equal(up, oup)
    assert np.array_equal(dn, odn)


def _compare(msz, f, fhat, xi, use_tma=True):
    ref = oracle.fix(f, fhat, xi)
    plan = msz.Plan(f.shape, torch.float32 if f.dtype == np.float32 else torch.float64, use_tma=use_tma)
    res = plan.fix(torch.from_numpy(f).cuda(), torch.from_numpy(fhat).cuda(), xi)
    plan.close()
    assert res.status == ref.status == 0
    assert res.counts == ref.counts
    assert np.array_equal(res.edit_idx.cpu().numpy(), ref.edit_idx.astype(np.int64))
    assert np.array_equal(bits_of(res.edit_val.cpu().numpy()), bits_of(ref.edit_val))
    assert np.array_equal(res.label_max.cpu().numpy().reshape(-1), ref.label_max)
    assert np.array_equal(res.label_min.cpu().numpy().reshape(-1), ref.label_min)
    g = torch.from_numpy(fhat).cuda()
    msz.apply(g, res.edit_idx, res.edit_val)
    assert np.array_equal(bits_of(g.cpu().numpy()), bits_of(ref.g))
    return res, ref


CASES = [
    ("bumps128", lambda: synth.bumps2d(128, 128, 0), 1e-3),
    ("bumps128-1e-2", lambda: synth.bumps2d(128, 128, 0), 1e-2),
    ("bumps-ragged", lambda: synth.bumps2d(203, 77, 5), 3e-3),
    ("bumps-f64", lambda: synth.bumps2d(160, 90, 6, dtype=np.float64), 1e-3),
    ("bumps-f64-ragged", lambda: synth.bumps2d(150, 91, 6, dtype=np.float64), 1e-3),
    ("lognormal-40", lambda: synth.lognormal3d(seed=1, shape=(40, 36, 33)), 1e-3),
    ("lognormal-f64", lambda: synth.lognormal3d(seed=9, shape=(24, 31, 29), dtype=np.float64), 1e-4),
    ("turb-48", lambda: synth.turbulence3d(48, 3, kmax=6.0), 1e-3),
    ("turb-ragged", lambda: synth.turbulence3d(61, 4, kmax=8.0, shape=(27, 45, 61)), 1e-4),
    ("ocean-crop", lambda: synth.ocean2d(3600, 2400, 2, window=(0, 300, 0, 416)), 1e-3),
    ("ocean-crop-ragged", lambda: synth.ocean2d(3600, 2400, 2, window=(0, 301, 0, 420)), 1e-3),
    ("turb-f64", lambda: synth.turbulence3d(32, 8, kmax=4.0, dtype=np.float64, shape=(20, 24, 32)), 1e-3),
    ("strip-x", lambda: _field("smooth", (1, 300), np.float32, 3), 1e-2),
    ("strip-y", lambda: _field("smooth", (257, 1), np.float32, 4), 1e-2),
    ("column-z", lambda: _field("smooth", (70, 1, 1), np.float64, 5), 1e-2),
    ("tiny-2x2x2", lambda: _field("noise", (2, 2, 2), np.float32, 6), 3e-1),
    ("single-vertex", lambda: np.array([[1.5]], dtype=np.float32), 1e-1),
]


@pytest.mark.parametrize("name,make,rel", CASES, ids=[c[0] for c in CASES])
def test_fix_matches_oracle(name, make, rel):
    msz = _msz()
    f = make()
    xi = synth.xi_for(f, rel)
    fhat = synth.quantise(f, xi)
    res, ref = _compare(msz, f, fhat, xi)
    check_result(f, fhat, xi, ref.g, ref.edit_idx, ref.edit_val, ref.label_max, ref.label_min)


GOLDEN = sorted(p for p in glob.glob(os.path.join(os.path.dirname(__file__), "golden", "*.json"))
                if not os.path.basename(p).startswith("fullsize_"))  # hand-worked cases only


@pytest.mark.parametrize("path", GOLDEN, ids=[os.path.basename(p) for p in GOLDEN])
def test_golden_hand_worked(path):
    # the hand-worked cases of Sec. 4 (one per false type and per R-loop
    # direction): the same edits, values and counters on the device
    msz = _msz()
    case = json.load(open(path))
    dt = np.dtype(case["dtype"])
    shape = tuple(case["shape"])
    f = np.array(case["f"], dtype=dt).reshape(shape)
    fhat = np.array(case["fhat"], dtype=dt).reshape(shape)
    res, ref = _compare(msz, f, fhat, case["xi"])
    assert res.edit_idx.cpu().tolist() == case["edit_idx"]
    assert np.array_equal(bits_of(ref.g.reshape(-1)), bits_of(np.array(case["g"], dtype=dt)))
    for k, v in case["counts"].items():
        assert res.counts[k] == v, k


@pytest.mark.parametrize("name,make,rel", [c for c in CASES if c[0] in ("bumps128", "bumps-f64", "turb-48", "ocean-crop", "turb-f64")],
                         ids=lambda c: c if isinstance(c, str) else "")
def test_fix_matches_oracle_plain_loads(name, make, rel):
    # the same shapes without TMA staging (the path ragged rows always take)
    msz = _msz()
    f = make()
    xi = synth.xi_for(f, rel)
    _compare(msz, f, synth.quantise(f, xi), xi, use_tma=False)


def test_identity_input():
    msz = _msz()
    f = synth.bumps2d(64, 48, 1)
    res, _ = _compare(msz, f, f.copy(), 1e-3)
    assert res.n_edits == 0


def test_constant_decompression():
    msz = _msz()
    rng = np.random.default_rng(4)
    f = rng.uniform(0, 1, (9, 10, 11)).astype(np.float32)
    fhat = np.full(f.shape, 0.5, dtype=np.float32)
    res, ref = _compare(msz, f, fhat, 1.0)
    assert res.n_edits > 0


def test_lower_bound_collisions():
    msz = _msz()
    one = np.float32(1.0)
    vals = [one]
    for _ in range(63):
        vals.append(np.nextafter(vals[-1], np.float32(2)))
    f = np.array(vals[::-1], dtype=np.float32).reshape(8, 8)
    fhat = np.full((8, 8), 1.0, dtype=np.float32)
    res, _ = _compare(msz, f, fhat, float(np.float32(2.0 ** 20)))
    assert res.counts["freezes"] > 0


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_error_codes_match_oracle(dtype):
    msz = _msz()
    f = synth.bumps2d(32, 32, 2, dtype=dtype)
    xi = synth.xi_for(f, 1e-3)
    fhat = synth.quantise(f, xi)
    plan = msz.Plan(f.shape, torch.float32 if dtype == np.float32 else torch.float64)
    cases = []
    bad = fhat.copy(); bad[3, 4] = np.nan; cases.append((f, bad, xi))
    bad = f.copy(); bad[0, 0] = np.inf; cases.append((bad, fhat, xi))
    bad = fhat.copy(); bad[5, 5] = f[5, 5] + dtype(4 * xi); cases.append((f, bad, xi))
    cases.append((f, fhat, -1.0))
    for a, b, x in cases:
        want = oracle.fix(a, b, x).status
        got = plan.fix(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), x, check=False).status
        assert got == want != 0
    # the plan stays usable after errors
    res = plan.fix(torch.from_numpy(f).cuda(), torch.from_numpy(fhat).cuda(), xi)
    ref = oracle.fix(f, fhat, xi)
    assert res.counts == ref.counts
    plan.close()


def test_apply_rejects_out_of_range_and_accepts_empty():
    msz = _msz()
    from paper_2406_09423_gb300 import native

    g = torch.zeros(10, 10, device="cuda")
    idx = torch.tensor([3, 100], dtype=torch.int32, device="cuda")
    val = torch.tensor([1.0, 2.0], device="cuda")
    st = native.msz_apply(g.data_ptr(), (10, 10), torch.float32, idx.data_ptr(), val.data_ptr(), 2,
                          torch.cuda.current_stream().cuda_stream)
    assert st == -1
    assert float(g.view(-1)[3]) == 1.0
    assert native.msz_apply(g.data_ptr(), (10, 10), torch.float32, 0, 0, 0, 0) == 0


def test_fix_host_equals_fix():
    msz = _msz()
    from paper_2406_09423_gb300 import native

    f = synth.lognormal3d(seed=2, shape=(20, 30, 40))
    xi = synth.xi_for(f, 1e-3)
    fhat = synth.quantise(f, xi)
    plan = msz.Plan(f.shape, torch.float32)
    dres = plan.fix(torch.from_numpy(f).cuda(), torch.from_numpy(fhat).cuda(), xi)
    n = f.size
    idx = np.zeros(n, dtype=np.uint32)
    val = np.zeros(n, dtype=np.float32)
    lmax = np.zeros(n, dtype=np.int32)
    lmin = np.zeros(n, dtype=np.int32)
    r = native.msz_fix_host(plan._p, f.ctypes.data, fhat.ctypes.data, xi, idx.ctypes.data, val.ctypes.data,
                            lmax.ctypes.data, lmin.ctypes.data, 0)
    assert r.status == 0
    ne = int(r.n_edits)
    assert np.array_equal(idx[:ne].astype(np.int64), dres.edit_idx.cpu().numpy())
    assert np.array_equal(val[:ne], dres.edit_val.cpu().numpy())
    assert np.array_equal(lmax, dres.label_max.cpu().numpy().reshape(-1))
    assert np.array_equal(lmin, dres.label_min.cpu().numpy().reshape(-1))
    assert r.counts.as_dict() == dres.counts
    plan.close()


def test_repeated_fix_on_one_plan_is_deterministic():
    msz = _msz()
    f = synth.turbulence3d(40, 7, kmax=5.0)
    xi = synth.xi_for(f, 1e-3)
    fhat = synth.quantise(f, xi)
    plan = msz.Plan(f.shape, torch.float32)
    a = plan.fix(torch.from_numpy(f).cuda(), torch.from_numpy(fhat).cuda(), xi)
    b = plan.fix(torch.from_numpy(f).cuda(), torch.from_numpy(fhat).cuda(), xi)
    assert a.counts == b.counts
    assert torch.equal(a.edit_idx, b.edit_idx) and torch.equal(a.edit_val, b.edit_val)
    plan.close()
