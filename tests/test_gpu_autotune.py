"""Launch parameters and the batch autotuner (msz_tuning, msz_batch_autotune):
they change how the correction loop is scheduled on the GPU, never its
results. Under every setting tried here - each parameter at the ends of its
range - a batch and a plan give, field by field, exactly the untuned plain
results (counters, edit lists, labels); the autotuner returns a valid
setting, keeps the results exact, and answers from its cache the second
time."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2406_09423_gb300 import synth
from tests.invariants import bits_of

pytestmark = pytest.mark.gpu


def _msz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2406_09423_gb300 as msz

    return msz


def _inputs():
    fs = [synth.bumps2d(128, 128, 0), synth.bumps2d(77, 203, 5, dtype=np.float64),
          synth.lognormal3d(seed=1, shape=(20, 24, 33)),
          synth.turbulence3d(32, 8, kmax=4.0, dtype=np.float64, shape=(16, 32, 32)),
          synth.turbulence3d(48, 3, kmax=6.0)]
    rels = [1e-3, 3e-3, 1e-3, 1e-4, 1e-3]
    xis = [synth.xi_for(f, r) for f, r in zip(fs, rels)]
    hs = [synth.quantise(f, x) for f, x in zip(fs, xis)]
    return ([torch.from_numpy(f).cuda() for f in fs], [torch.from_numpy(h).cuda() for h in hs], xis)


def _same(a, b):
    assert a.status == b.status == 0
    assert a.counts == b.counts
    assert torch.equal(a.edit_idx, b.edit_idx)
    assert bits_of(a.edit_val.cpu().numpy()).tolist() == bits_of(b.edit_val.cpu().numpy()).tolist()
    assert torch.equal(a.label_max, b.label_max) and torch.equal(a.label_min, b.label_min)


SETTINGS = [
    {"jumps_per_step": 1, "chase_steps": 4},
    {"jumps_per_step": 4, "chase_steps": 256, "graph_steps": 1},
    {"small_rounds": 0},
    {"small_rounds": 1, "small_cases": 1},
    {"small_rounds": 1024, "small_cases": 512, "graph_steps": 8},
    {"sweep_chunk": 4, "blocks_per_sm": 1},
    {"sweep_chunk": 17, "blocks_per_sm": 2, "jumps_per_step": 3, "chase_steps": 7},
]


def test_every_setting_gives_the_plain_results():
    msz = _msz()
    fs, hs, xis = _inputs()
    plain = [msz.fix(f, h, x) for f, h, x in zip(fs, hs, xis)]
    b = msz.Batch([f.shape for f in fs], [f.dtype for f in fs])
    default = b.tuning
    assert default == msz.native.msz_tuning_default()
    for setting in SETTINGS:
        b.tuning = dict(default, **setting)
        assert b.tuning == dict(default, **setting)
        st, res = b.fix(fs, hs, xis)
        assert st == 0, setting
        for r, p in zip(res, plain):
            _same(r, p)
    b.close()
    # a plan under a setting as well
    p = msz.Plan(tuple(fs[4].shape), fs[4].dtype)
    p.tuning = dict(default, **SETTINGS[6])
    _same(p.fix(fs[4], hs[4], xis[4]), plain[4])
    p.close()


def test_invalid_settings_are_rejected():
    msz = _msz()
    fs, _, _ = _inputs()
    b = msz.Batch([fs[0].shape], [fs[0].dtype])
    d = msz.native.msz_tuning_default()
    for bad in ({"jumps_per_step": 0}, {"chase_steps": 1000}, {"small_cases": 70000}, {"graph_steps": 9},
                {"sweep_chunk": 65}, {"blocks_per_sm": -1}):
        with pytest.raises(RuntimeError, match="MSZ_ERR_ARG"):
            b.tuning = dict(d, **bad)
    assert b.tuning == d
    b.close()


def test_autotuner_keeps_results_and_caches():
    msz = _msz()
    fs, hs, xis = _inputs()
    plain = [msz.fix(f, h, x) for f, h, x in zip(fs, hs, xis)]
    b = msz.Batch([f.shape for f in fs], [f.dtype for f in fs])
    tuned, tried = b.autotune(fs, hs, xis, force=True)
    assert tried > 10
    assert msz.native.msz_tuning_valid(tuned) == 0 and b.tuning == tuned
    st, res = b.fix(fs, hs, xis)
    assert st == 0
    for r, p in zip(res, plain):
        _same(r, p)
    b.close()
    # another batch with the same signature takes the cached setting
    b2 = msz.Batch([f.shape for f in fs], [f.dtype for f in fs], autotune=True)
    cached, tried2 = b2.autotune(fs, hs, xis)
    assert cached == tuned and tried2 == 0
    st, res = b2.fix(fs, hs, xis)
    assert st == 0 and b2.tuning == tuned
    for r, p in zip(res, plain):
        _same(r, p)
    b2.close()
