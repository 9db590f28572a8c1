"""Parity run of the bounds-checked library build (libmsz_checked.so).

Run as a separate process with MSZ_LIBRARY=checked (tests/test_gpu_checked.py
does): small and ragged fields, f32 and f64, 2D and 3D, the hand-worked
golden cases, a batch, the allocation-free entry point, a capped run and
the 3600 x 2400 ocean record at 1e-3 x range, each compared with the oracle
bit for bit. Any bounds check that fires ends
a fix with MSZ_ERR_CHECK, so a clean run also shows that no index read from
device data left its range. Prints "checked parity ok <cases>" and exits 0.
"""
import glob
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch  # noqa: E402

import oracle  # noqa: E402
import paper_2406_09423_gb300 as msz  # noqa: E402
from paper_2406_09423_gb300 import native, synth  # noqa: E402


def bits(a):
    a = np.ascontiguousarray(a)
    return a.view(np.uint32 if a.dtype == np.float32 else np.uint64)


def same(res, ref):
    assert res.status == ref.status, (res.status, ref.status)
    assert res.counts == ref.counts, (res.counts, ref.counts)
    assert np.array_equal(res.edit_idx.cpu().numpy(), ref.edit_idx.astype(np.int64))
    assert np.array_equal(bits(res.edit_val.cpu().numpy()), bits(ref.edit_val))
    if res.status == 0:
        assert np.array_equal(res.label_max.cpu().numpy().reshape(-1), ref.label_max)
        assert np.array_equal(res.label_min.cpu().numpy().reshape(-1), ref.label_min)


def main():
    assert native.LIB_PATH.endswith("libmsz_checked.so"), native.LIB_PATH
    n = 0
    cases = [
        (synth.bumps2d(128, 128, 0), 1e-3), (synth.bumps2d(203, 77, 5), 3e-3),
        (synth.bumps2d(150, 91, 6, dtype=np.float64), 1e-3),
        (synth.lognormal3d(seed=1, shape=(40, 36, 33)), 1e-3),
        (synth.turbulence3d(61, 4, kmax=8.0, shape=(27, 45, 61)), 1e-4),
        (synth.turbulence3d(48, 3, kmax=6.0), 1e-3),
        (synth.ocean2d(3600, 2400, 2, window=(0, 301, 0, 420)), 1e-3),
        (synth.turbulence3d(32, 8, kmax=4.0, dtype=np.float64, shape=(20, 24, 32)), 1e-3),
    ]
    fields = []
    for f, rel in cases:
        xi = synth.xi_for(f, rel)
        fh = synth.quantise(f, xi)
        fields.append((f, fh, xi))
        ref = oracle.fix(f, fh, xi)
        for tma in (True, False):
            same(msz.fix(torch.from_numpy(f).cuda(), torch.from_numpy(fh).cuda(), xi) if tma else
                 msz.Plan(f.shape, torch.from_numpy(f).dtype, use_tma=False).fix(
                     torch.from_numpy(f).cuda(), torch.from_numpy(fh).cuda(), xi), ref)
            n += 1
    for path in sorted(glob.glob(os.path.join(ROOT, "tests", "golden", "*.json"))):
        if os.path.basename(path).startswith("fullsize_"):
            continue
        c = json.load(open(path))
        dt = np.dtype(c["dtype"])
        f = np.array(c["f"], dtype=dt).reshape(tuple(c["shape"]))
        fh = np.array(c["fhat"], dtype=dt).reshape(tuple(c["shape"]))
        same(msz.fix(torch.from_numpy(f).cuda(), torch.from_numpy(fh).cuda(), c["xi"]), oracle.fix(f, fh, c["xi"]))
        n += 1
    # a batch of all of them
    td = [torch.from_numpy(f).cuda() for f, _, _ in fields]
    th = [torch.from_numpy(h).cuda() for _, h, _ in fields]
    b = msz.Batch([f.shape for f, _, _ in fields], [t.dtype for t in td])
    st, res = b.fix(td, th, [x for _, _, x in fields])
    b.close()
    assert st == 0
    for r, (f, fh, xi) in zip(res, fields):
        same(r, oracle.fix(f, fh, xi))
        n += 1
    # a capped run
    f, fh, xi = fields[0]
    p = msz.Plan(f.shape, torch.float32, max_rounds=5)
    r = p.fix(torch.from_numpy(f).cuda(), torch.from_numpy(fh).cuda(), xi, check=False)
    p.close()
    same(r, oracle.fix(f, fh, xi, max_rounds=5))
    n += 1
    # the allocation-free entry point
    f, fh, xi = fields[3]
    N = f.size
    idx = torch.zeros(N, dtype=torch.int32, device="cuda")
    val = torch.zeros(N, dtype=torch.float32, device="cuda")
    lab = torch.zeros(2, N, dtype=torch.int32, device="cuda")
    fd, hd = torch.from_numpy(f).cuda(), torch.from_numpy(fh).cuda()
    r = native.msz_fix_noalloc(f.shape, torch.float32, fd.data_ptr(), hd.data_ptr(), xi, idx.data_ptr(),
                               val.data_ptr(), lab[0].data_ptr(), lab[1].data_ptr(), 0)
    ref = oracle.fix(f, fh, xi)
    assert r.status == 0 and r.counts.as_dict() == ref.counts
    ne = int(r.n_edits)
    assert np.array_equal(idx[:ne].cpu().numpy(), ref.edit_idx.astype(np.int32))
    n += 1
    # a full-size record (rounds of more than 64K cases, the cluster kernel
    # handing the field back to the grid kernels, long label walks): every
    # digest and counter of the oracle's record
    import hashlib

    rec = json.load(open(os.path.join(ROOT, "tests", "golden", "fullsize_ocean_1e-3.json")))

    class OnDevice:
        def __getattr__(self, name):
            fn = getattr(synth, name)
            return lambda *a, **k: fn(*a, device="cuda", **k)

    def digest(a):
        if hasattr(a, "detach"):
            a = a.detach().cpu().numpy()
        return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()

    f = eval(rec["generator"], {"__builtins__": {}}, {"synth": OnDevice()}).contiguous()
    xi = synth.xi_for(f, rec["rel"])
    fh = synth.quantise_torch(f, xi)
    assert digest(f) == rec["sha256"]["f"] and digest(fh) == rec["sha256"]["fhat"]
    p = msz.Plan(tuple(f.shape), f.dtype)
    r = p.fix(f, fh, xi, check=False)
    p.close()
    assert r.status == rec["status"] and r.counts == rec["counts"], (r.status, r.counts)
    assert digest(r.edit_idx.to(torch.int32).cpu().numpy().astype("<u4")) == rec["sha256"]["edit_idx"]
    assert digest(r.edit_val) == rec["sha256"]["edit_val"]
    assert digest(r.label_max.reshape(-1).cpu().numpy().astype("<i4")) == rec["sha256"]["label_max"]
    assert digest(r.label_min.reshape(-1).cpu().numpy().astype("<i4")) == rec["sha256"]["label_min"]
    n += 1
    print(f"checked parity ok {n}", flush=True)


if __name__ == "__main__":
    main()
