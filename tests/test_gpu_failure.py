"""Failure paths of the correction loop on the GPU, none of which faults,
traps or spins a device:

* the round cap: a fix allowed k rounds stops after round k + 1 with
  MSZ_ERR_NOCONVERGE and returns the edits made so far; for every k, the
  field it leaves and its counters equal the oracle's capped run bit for
  bit (a round-by-round check of the loop of Sec. 4.1-4.3);
* the host's stall detection: with MSZ_OPT_TEST_STALL the fields start in a
  stage that no kernel serves, so no state machine moves and the plan, the
  batch and the server report MSZ_ERR_TIMEOUT;
* cancelling a served request (queued or running): it finishes with
  MSZ_ERR_CANCELLED while the other requests' results stay those of msz_fix.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2406_09423_gb300 import synth

pytestmark = pytest.mark.gpu

NOCONVERGE, TIMEOUT, CANCELLED = -6, -7, -11


def _msz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2406_09423_gb300 as msz

    return msz


def _bits(a):
    a = np.ascontiguousarray(a)
    return a.view(np.uint32 if a.dtype == np.float32 else np.uint64)


CAPPED = [
    ("bumps-64x48-f32", lambda: synth.bumps2d(64, 48, 1), 1e-3),
    ("turb-20x24x32-f64", lambda: synth.turbulence3d(32, 8, kmax=4.0, dtype=np.float64, shape=(20, 24, 32)), 1e-3),
    ("lognormal-16x20x24-f32", lambda: synth.lognormal3d(seed=4, shape=(16, 20, 24)), 3e-3),
]


@pytest.mark.parametrize("name,make,rel", CAPPED, ids=[c[0] for c in CAPPED])
def test_round_capped_fix_matches_oracle_round_by_round(name, make, rel):
    msz = _msz()
    f = make()
    xi = synth.xi_for(f, rel)
    fh = synth.quantise(f, xi)
    full = oracle.fix(f, fh, xi)
    assert full.status == 0
    c = full.counts
    rounds = sum(c[k] for k in ("c_rounds_fpmax", "c_rounds_fpmin", "c_rounds_fnmax", "c_rounds_fnmin",
                                "r_rounds"))
    assert rounds >= 3
    fd, hd = torch.from_numpy(f).cuda(), torch.from_numpy(fh).cuda()
    ks = list(range(1, rounds))
    if len(ks) > 40:  # every round early on, then an even sample
        ks = ks[:20] + ks[20::max(1, (len(ks) - 20) // 20)]
    for k in ks:
        ref = oracle.fix(f, fh, xi, max_rounds=k)
        assert ref.status == NOCONVERGE, k
        plan = msz.Plan(f.shape, fd.dtype, max_rounds=k)
        r = plan.fix(fd, hd, xi, check=False)
        plan.close()
        assert r.status == NOCONVERGE, (k, r.status)
        assert np.array_equal(r.edit_idx.cpu().numpy(), ref.edit_idx.astype(np.int64)), k
        g = hd.clone()
        msz.apply(g, r.edit_idx, r.edit_val)
        assert np.array_equal(_bits(g.cpu().numpy()), _bits(ref.g)), k
        assert r.counts == ref.counts, (k, r.counts, ref.counts)
    # past the last round the cap does not bind
    plan = msz.Plan(f.shape, fd.dtype, max_rounds=rounds)
    r = plan.fix(fd, hd, xi)
    plan.close()
    assert r.status == 0 and r.counts == full.counts


def test_stall_is_reported_as_timeout():
    msz = _msz()
    f = torch.from_numpy(synth.bumps2d(48, 40, 2)).cuda()
    xi = synth.xi_for(f, 1e-3)
    fh = torch.from_numpy(synth.quantise(f.cpu().numpy(), xi)).cuda()
    plan = msz.Plan(tuple(f.shape), f.dtype, flags=msz.native.MSZ_OPT_TEST_STALL)
    t0 = time.time()
    r = plan.fix(f, fh, xi, check=False)
    plan.close()
    assert r.status == TIMEOUT and r.n_edits == 0
    assert time.time() - t0 < 30
    # the context is still usable: a normal fix right after
    r = msz.fix(f, fh, xi)
    assert r.status == 0
    # batch: every field times out
    b = msz.Batch([tuple(f.shape)] * 2, [f.dtype] * 2, flags=msz.native.MSZ_OPT_TEST_STALL)
    st, rs = b.fix([f, f], [fh, fh], [xi, xi])
    b.close()
    assert st == TIMEOUT and all(x.status == TIMEOUT for x in rs)
    # server
    srv = msz.Server(1 << 30, max_slots=4, flags=msz.native.MSZ_OPT_TEST_STALL)
    rid = srv.submit(f, fh, xi)
    st, out = msz.native.msz_server_poll(srv._s, rid, 20000)
    srv.close()
    assert st == 0 and out.status == TIMEOUT


def _drain(msz, srv, ids, cases, plain, timeout=120):
    """Polls every request until finished; checks finished ones against the
    plain results; returns {id: status}."""
    got = {}
    t0 = time.time()
    while len(got) < len(ids) and time.time() - t0 < timeout:
        for rid in ids:
            if rid in got:
                continue
            st, r = msz.native.msz_server_poll(srv._s, rid, 5)
            if st != 0:
                continue
            got[rid] = r.status
            if r.status == 0:
                k = ids.index(rid)
                res = msz._result(torch, r, tuple(cases[k][0].shape), cases[k][0].dtype, True)
                torch.cuda.synchronize()
                assert res.counts == plain[k].counts
                assert torch.equal(res.edit_idx, plain[k].edit_idx)
                assert torch.equal(res.edit_val, plain[k].edit_val)
                assert torch.equal(res.label_max, plain[k].label_max)
                assert torch.equal(res.label_min, plain[k].label_min)
            srv.release(rid)
    return got


def test_cancelled_request_leaves_the_others_exact():
    msz = _msz()
    cases = []
    for make, rel in [(lambda: synth.ocean2d(3600, 2400, 2, device="cuda"), 1e-3),
                      (lambda: synth.turbulence3d(64, 3, kmax=8.0, device="cuda"), 1e-3),
                      (lambda: synth.lognormal3d(256, 1, device="cuda"), 1e-3),
                      (lambda: synth.turbulence3d(64, 5, kmax=8.0, device="cuda"), 1e-4)]:
        f = make()
        xi = synth.xi_for(f, rel)
        cases.append((f, synth.quantise_torch(f, xi), xi))
    plain = [msz.fix(f, h, x) for f, h, x in cases]
    # queued: one slot, the ocean field takes it, the 64^3 field waits
    srv = msz.Server(16 << 30, max_slots=1)
    ids = [srv.submit(*cases[0]), srv.submit(*cases[1])]
    assert srv.cancel(ids[1]) == 0
    got = _drain(msz, srv, ids, cases[:2], plain[:2])
    assert got == {ids[0]: 0, ids[1]: CANCELLED}
    assert srv.cancel(ids[0]) in (-1, -9)  # finished: unknown or not cancellable
    srv.close()
    # running: the 256^3 field is admitted at once (free slots) and cancelled
    # while it runs beside the other two
    srv = msz.Server(16 << 30, max_slots=4)
    ids = [srv.submit(*cases[2]), srv.submit(*cases[1]), srv.submit(*cases[3])]
    time.sleep(0.005)
    assert srv.cancel(ids[0]) == 0
    got = _drain(msz, srv, ids, [cases[2], cases[1], cases[3]], [plain[2], plain[1], plain[3]])
    srv.close()
    assert got[ids[0]] == CANCELLED
    assert got[ids[1]] == 0 and got[ids[2]] == 0
