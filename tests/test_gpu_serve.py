"""Served form (continuous batching): fields submitted while others are being
corrected are admitted as slots and memory free up; every result equals the
plain single-field result (and the oracle's on small fields), alone and in
the mix; a field larger than the budget is rejected."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2406_09423_gb300 import synth

pytestmark = pytest.mark.gpu


def _msz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2406_09423_gb300 as msz

    return msz


def _cases():
    out = []
    for k, (make, rel) in enumerate([
        (lambda: synth.bumps2d(128, 128, 0), 1e-3),
        (lambda: synth.lognormal3d(seed=1, shape=(24, 32, 40)), 1e-3),
        (lambda: synth.bumps2d(96, 70, 7, dtype=np.float64), 1e-3),
        (lambda: synth.turbulence3d(64, 3, kmax=8.0), 1e-3),
        (lambda: synth.ocean2d(3600, 2400, 2, window=(0, 200, 0, 320)), 1e-4),
        (lambda: synth.turbulence3d(40, 5, kmax=5.0, dtype=np.float64), 1e-3),
    ]):
        f = make()
        xi = synth.xi_for(f, rel)
        out.append((f, synth.quantise(f, xi), xi))
    return out


def _same(a, b):
    assert a.status == b.status == 0
    assert a.counts == b.counts
    assert torch.equal(a.edit_idx, b.edit_idx)
    assert torch.equal(a.edit_val, b.edit_val)
    assert torch.equal(a.label_max, b.label_max)
    assert torch.equal(a.label_min, b.label_min)


@pytest.mark.parametrize("budget_gb,slots", [(8, 16), (0.02, 2)])
def test_served_results_equal_plain(budget_gb, slots):
    msz = _msz()
    cases = _cases()
    dev = [(torch.from_numpy(f).cuda(), torch.from_numpy(h).cuda(), x) for f, h, x in cases]
    plain = []
    for f, h, x in dev:
        p = msz.Plan(tuple(f.shape), f.dtype)
        plain.append(p.fix(f, h, x))
        p.close()
    srv = msz.Server(int(budget_gb * (1 << 30)), max_slots=slots)
    ids = []
    for k, (f, h, x) in enumerate(dev):  # staggered arrivals: later fields join running ones
        ids.append(srv.submit(f, h, x))
        time.sleep(0.002 * (k % 3))
    got = {}
    t0 = time.time()
    while len(got) < len(ids) and time.time() - t0 < 120:
        for rid in ids:
            if rid not in got:
                r = srv.poll(rid, wait_ms=5)
                if r is not None:
                    got[rid] = r
    srv.close()
    assert len(got) == len(ids)
    for rid, ref, (f, h, x) in zip(ids, plain, cases):
        _same(got[rid], ref)
        assert got[rid].device_ms > 0
        if f.size <= 70000:
            o = oracle.fix(f, h, x)
            assert got[rid].counts == o.counts


def test_field_larger_than_budget_is_rejected():
    msz = _msz()
    f = torch.zeros(64, 64, 64, device="cuda")
    srv = msz.Server(1 << 20, max_slots=4)  # 1 MiB: too small for a 64^3 field
    rid = srv.submit(f, f, 0.1)
    st, r = msz.native.msz_server_poll(srv._s, rid, 2000)
    assert st == 0 and r.status == -5
    srv.close()
