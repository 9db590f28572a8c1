"""Batched form: fields of uneven shapes and mixed float32 / float64 in one
batch give, field by field, exactly the plain single-field results (and the
oracle's on the small ones); a failing field does not disturb the others."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2406_09423_gb300 import synth
from tests.invariants import bits_of

pytestmark = pytest.mark.gpu


def _msz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2406_09423_gb300 as msz

    return msz


def _tdt(a):
    return torch.float32 if a.dtype == np.float32 else torch.float64


def _fields():
    out = []
    out.append(synth.bumps2d(128, 128, 0))
    out.append(synth.bumps2d(77, 203, 5, dtype=np.float64))
    out.append(synth.lognormal3d(seed=1, shape=(20, 24, 33)))
    out.append(synth.turbulence3d(32, 8, kmax=4.0, dtype=np.float64, shape=(16, 32, 32)))
    out.append(synth.ocean2d(3600, 2400, 2, window=(0, 160, 0, 256)))
    out.append(np.array([[1.5]], dtype=np.float32))
    out.append(synth.turbulence3d(48, 3, kmax=6.0))
    return out


def _same(a, b):
    assert a.status == b.status
    assert a.counts == b.counts
    assert torch.equal(a.edit_idx, b.edit_idx)
    assert torch.equal(a.edit_val, b.edit_val) or bits_of(a.edit_val.cpu().numpy()).tolist() == \
        bits_of(b.edit_val.cpu().numpy()).tolist()
    assert torch.equal(a.label_max, b.label_max)
    assert torch.equal(a.label_min, b.label_min)


@pytest.mark.parametrize("use_tma", [True, False])
def test_batch_equals_plain_and_oracle(use_tma):
    msz = _msz()
    fs = _fields()
    rels = [1e-3, 3e-3, 1e-3, 1e-4, 1e-3, 1e-1, 1e-3]
    xis = [synth.xi_for(f, r) for f, r in zip(fs, rels)]
    hs = [synth.quantise(f, x) for f, x in zip(fs, xis)]
    td = [torch.from_numpy(f).cuda() for f in fs]
    th = [torch.from_numpy(h).cuda() for h in hs]
    b = msz.Batch([f.shape for f in fs], [_tdt(f) for f in fs], use_tma=use_tma)
    st, res = b.fix(td, th, xis)
    assert st == 0
    for f, h, x, t1, t2, r in zip(fs, hs, xis, td, th, res):
        plan = msz.Plan(f.shape, _tdt(f), use_tma=use_tma)
        _same(r, plan.fix(t1, t2, x))
        plan.close()
        if f.size <= 70000:
            ref = oracle.fix(f, h, x)
            assert r.counts == ref.counts
            assert np.array_equal(r.edit_idx.cpu().numpy(), ref.edit_idx.astype(np.int64))
    # a second run of the same batch object gives the same results
    st2, res2 = b.fix(td, th, xis)
    for r1, r2 in zip(res, res2):
        _same(r1, r2)
    b.close()


def test_failing_field_does_not_disturb_others():
    msz = _msz()
    fs = [synth.bumps2d(64, 64, 1), synth.bumps2d(64, 48, 2), synth.lognormal3d(seed=3, shape=(12, 16, 16))]
    xis = [synth.xi_for(f, 1e-3) for f in fs]
    hs = [synth.quantise(f, x) for f, x in zip(fs, xis)]
    bad = hs[1].copy()
    bad[3, 3] = fs[1][3, 3] + np.float32(5 * xis[1])
    b = msz.Batch([f.shape for f in fs], [torch.float32] * 3)
    st, res = b.fix([torch.from_numpy(f).cuda() for f in fs],
                    [torch.from_numpy(h).cuda() for h in (hs[0], bad, hs[2])], xis)
    assert st == -4
    assert res[1].status == -4
    for k in (0, 2):
        ref = oracle.fix(fs[k], hs[k], xis[k])
        assert res[k].status == 0 and res[k].counts == ref.counts
        assert np.array_equal(res[k].edit_idx.cpu().numpy(), ref.edit_idx.astype(np.int64))
    b.close()
