"""msz_field_metrics (Appendix B: PSNR and the right labelled ratio) against
the oracle's plain definitions, before and after a correction."""
import math

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


def _fields():
    return [
        ("bumps-2d-f32", synth.bumps2d(128, 96, 0), 1e-2),
        ("bumps-2d-f64", synth.bumps2d(70, 53, 1).astype(np.float64), 3e-2),
        ("turb-3d-f32-ragged", synth.turbulence3d(40, 7, kmax=6.0, shape=(27, 33, 40)), 1e-2),
        ("lognormal-3d-f32", synth.lognormal3d(seed=1, shape=(21, 30, 37)), 1e-2),
    ]


def _check(msz, f, g):
    ref = oracle.metrics(f, g)
    got = msz.field_metrics(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda())
    assert got["wrong"] == ref["wrong"]
    assert got["right_labelled"] == ref["right_labelled"]
    assert got["value_range"] == ref["value_range"]
    # the device sums the squares in another order than the correctly rounded
    # oracle sum: N rounded additions, relative error well below 1e-12 here
    assert got["mse"] == pytest.approx(ref["mse"], rel=1e-12, abs=0.0)
    if math.isinf(ref["psnr"]):
        assert math.isinf(got["psnr"])
    else:
        assert got["psnr"] == pytest.approx(ref["psnr"], abs=1e-9)
    return got


@pytest.mark.parametrize("name,f,rel", _fields(), ids=[c[0] for c in _fields()])
def test_metrics_before_and_after_the_fix(name, f, rel):
    msz = _msz()
    xi = synth.xi_for(f, rel)
    fhat = synth.quantise(f, xi)
    before = _check(msz, f, fhat)
    assert before["wrong"] > 0  # the quantiser breaks some labels at these bounds
    res = msz.fix(torch.from_numpy(f).cuda(), torch.from_numpy(fhat).cuda(), xi)
    g = torch.from_numpy(fhat).cuda()
    msz.apply(g, res.edit_idx, res.edit_val)
    after = _check(msz, f, g.cpu().numpy())
    assert after["wrong"] == 0 and after["right_labelled"] == 1.0
    assert after["mse"] <= xi * xi


def test_identical_fields_and_arguments():
    msz = _msz()
    f = torch.from_numpy(synth.bumps2d(33, 17, 2)).cuda()
    m = msz.field_metrics(f, f)
    assert m["wrong"] == 0 and m["mse"] == 0.0 and math.isinf(m["psnr"])
    with pytest.raises(ValueError):
        msz.field_metrics(f, f[:-1])
    from paper_2406_09423_gb300 import native

    st, _ = native.msz_field_metrics(0, f.data_ptr(), tuple(f.shape), f.dtype)
    assert st == -1  # MSZ_ERR_ARG: NULL field


def test_metrics_full_size_properties():
    """512^3 turbulence at 1e-4 x range: after the fix no label is wrong; the
    distortion matches a float64 evaluation of its definition."""
    msz = _msz()
    dev = torch.device("cuda", 0)
    f = synth.turbulence3d(512, 3, device=dev)
    xi = synth.xi_for(f, 1e-4)
    fhat = synth.quantise_torch(f, xi)
    before = msz.field_metrics(f, fhat)
    assert before["wrong"] > 0
    res = msz.Plan(tuple(f.shape), f.dtype).fix(f, fhat, xi)
    g = fhat.clone()
    msz.apply(g, res.edit_idx, res.edit_val)
    after = msz.field_metrics(f, g)
    assert after["wrong"] == 0
    d = (f.double() - g.double()).square().sum().item() / f.numel()
    assert after["mse"] == pytest.approx(d, rel=1e-9)
    assert after["value_range"] == (f.max().double() - f.min().double()).item()
