"""msz_fix_noalloc: the correction loop for callers that cannot allocate device
memory (their allocator is owned by a framework or pool that must not grow,
or they run where an allocation may block or fail). It keeps its scratch in a
static device array inside the library; these tests check, through the C ABI,
that its results equal msz_fix's (bit for bit: the method's tolerance is
0 ulp) on two calls in a row, and that a field too large for that array is
rejected. It also runs two fields of the same vertex count but transposed
shapes back to back: the array is laid out identically for both, so the
second call rewrites the sweep's tensor maps at the addresses the first
used. This file is collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2406_09423_gb300 import synth

pytestmark = pytest.mark.gpu


def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2406_09423_gb300 as msz
    from paper_2406_09423_gb300 import native

    return msz, native


CASES = [
    ("bumps128-f32", lambda: synth.bumps2d(128, 128, 0), 1e-3),
    ("turb-f64-3d", lambda: synth.turbulence3d(32, 8, kmax=4.0, dtype=np.float64, shape=(20, 24, 32)), 1e-3),
    ("lognormal-ragged-f32", lambda: synth.lognormal3d(seed=1, shape=(21, 30, 37)), 1e-3),
]


@pytest.mark.parametrize("name,make,rel", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_fix_twice(name, make, rel):
    msz, native = _setup()
    f = make()
    xi = synth.xi_for(f, rel)
    fhat = synth.quantise(f, xi)
    tdt = torch.float32 if f.dtype == np.float32 else torch.float64
    fd, hd = torch.from_numpy(f).cuda(), torch.from_numpy(fhat).cuda()
    plan = msz.Plan(f.shape, tdt)
    ref = plan.fix(fd, hd, xi)
    plan.close()
    n = f.size
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        idx = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        val = torch.zeros(n, dtype=tdt, device="cuda")
        lmax = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        lmin = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        r = native.msz_fix_noalloc(f.shape, tdt, fd.data_ptr(), hd.data_ptr(), xi, idx.data_ptr(), val.data_ptr(),
                                   lmax.data_ptr(), lmin.data_ptr(), stream)
        assert r.status == 0, native.STATUS.get(r.status)
        ne = int(r.n_edits)
        assert ne == ref.n_edits
        assert torch.equal(idx[:ne].long(), ref.edit_idx)
        assert torch.equal(val[:ne].view(torch.int32 if tdt == torch.float32 else torch.int64),
                           ref.edit_val.view(torch.int32 if tdt == torch.float32 else torch.int64))
        assert torch.equal(lmax.view(f.shape), ref.label_max)
        assert torch.equal(lmin.view(f.shape), ref.label_min)
        assert r.counts.as_dict() == ref.counts


def _noalloc(native, f, fh, xi, tdt):
    n = f.numel()
    idx = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    val = torch.zeros(n, dtype=tdt, device="cuda")
    lmax = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    lmin = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    r = native.msz_fix_noalloc(tuple(f.shape), tdt, f.data_ptr(), fh.data_ptr(), xi, idx.data_ptr(),
                               val.data_ptr(), lmax.data_ptr(), lmin.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    return r, idx, val, lmax, lmin


def test_noalloc_transposed_shapes_back_to_back():
    msz, native = _setup()
    fields = []
    for shape, seed in (((64, 128), 3), ((128, 64), 4), ((64, 128), 5)):
        f = synth.bumps2d(shape[1], shape[0], seed)
        xi = synth.xi_for(f, 1e-3)
        fields.append((torch.from_numpy(f).cuda(), torch.from_numpy(synth.quantise(f, xi)).cuda(), xi))
    refs = [msz.fix(f, h, x) for f, h, x in fields]
    for (f, h, x), ref in zip(fields, refs):
        r, idx, val, lmax, lmin = _noalloc(native, f, h, x, torch.float32)
        assert r.status == 0
        ne = int(r.n_edits)
        assert ne == ref.n_edits and r.counts.as_dict() == ref.counts
        assert torch.equal(idx[:ne].long(), ref.edit_idx)
        assert torch.equal(val[:ne].view(torch.int32), ref.edit_val.view(torch.int32))
        assert torch.equal(lmax.view(f.shape), ref.label_max) and torch.equal(lmin.view(f.shape), ref.label_min)


def test_noalloc_rejects_fields_beyond_its_scratch():
    msz, native = _setup()
    shape = (1024, 4096)  # 4.2 M float32 vertices: more than the static scratch holds
    n = shape[0] * shape[1]
    # full-size buffers, so nothing could be read out of bounds even if the check failed
    f = torch.zeros(n, device="cuda")
    idx = torch.zeros(n, dtype=torch.int32, device="cuda")
    val = torch.zeros(n, device="cuda")
    lab = torch.zeros(2, n, dtype=torch.int32, device="cuda")
    r = native.msz_fix_noalloc(shape, torch.float32, f.data_ptr(), f.data_ptr(), 0.1, idx.data_ptr(),
                               val.data_ptr(), lab[0].data_ptr(), lab[1].data_ptr(), 0)
    assert r.status == -10
    assert "too large" in native.msz_strerror(-10)
