"""Kernel-timing instrumentation (msz_plan_kernel_stats): a plan with kernel
timing gives the same results as a plain one, and its per-kernel launch,
working-launch and work-unit counts agree with the fix's own counters."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2406_09423_gb300 import synth

pytestmark = pytest.mark.gpu


def _msz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2406_09423_gb300 as msz

    return msz


@pytest.mark.parametrize("shape", [(48, 40, 72), (300, 257)])
def test_kernel_stats_consistent(shape):
    msz = _msz()
    if len(shape) == 3:
        f = synth.turbulence3d(max(shape), 7, kmax=6.0, shape=shape)
    else:
        f = synth.bumps2d(shape[1], shape[0], 3)
    xi = synth.xi_for(f, 1e-3)
    fh = synth.quantise(f, xi)
    tf, th = torch.from_numpy(f).cuda(), torch.from_numpy(fh).cuda()
    plain = msz.Plan(f.shape, torch.float32)
    timed = msz.Plan(f.shape, torch.float32, time_kernels=True)
    a = plain.fix(tf, th, xi)
    b = timed.fix(tf, th, xi)
    assert a.counts == b.counts
    assert torch.equal(a.edit_idx, b.edit_idx)
    st = {s["name"]: s for s in timed.kernel_stats()}
    assert list(st) == ["k_csweep", "k_gather", "k_mark", "k_label_tile", "k_jump", "k_rcheck", "k_apply",
                        "k_reclass", "k_csmall"]
    steps = st["k_csweep"]["launches"]
    assert steps > 0
    per_step = {"k_jump": 2, "k_gather": 2, "k_mark": 2, "k_apply": 2, "k_reclass": 2, "k_label_tile": 2}
    for name, s in st.items():
        assert s["launches"] == per_step.get(name, 1) * steps
        assert 0 <= s["work_launches"] <= s["launches"]
        assert 0.0 <= s["work_ms"] <= s["ms"] + 1e-9
    c = b.counts
    n = f.size
    assert st["k_csweep"]["work_launches"] == 1 and st["k_csweep"]["units"] == n
    rounds = sum(c[k] for k in ("c_rounds_fpmax", "c_rounds_fpmin", "c_rounds_fnmax", "c_rounds_fnmin"))
    cases = sum(c[k] for k in ("c_cases_fpmax", "c_cases_fpmin", "c_cases_fnmax", "c_cases_fnmin"))
    # a C-loop round runs either through the grid kernels or whole in k_csmall
    small = st["k_csmall"]["units"]
    assert st["k_csmall"]["work_launches"] <= small
    assert st["k_mark"]["work_launches"] + small == rounds
    assert st["k_gather"]["work_launches"] <= rounds
    assert st["k_gather"]["units"] <= cases and st["k_mark"]["units"] <= cases
    assert st["k_apply"]["work_launches"] + small == rounds + c["r_rounds"]
    assert st["k_reclass"]["work_launches"] + small == rounds + c["r_rounds"]
    # f's labels once (k_rcheck resolves them in place), then g's at every evaluation
    evals = c["label_evals"] + 1
    for name in ("k_label_tile", "k_rcheck"):
        assert st[name]["work_launches"] == evals, name
    # the R-check counts algorithmic bytes: every vertex is examined by f's
    # resolution and by g's first evaluation (12 bytes each), exits cost 8
    assert 24 * n <= st["k_rcheck"]["units"] <= evals * (12 * n + 32 * n)
    # the label tiles count bytes: at most 14 per vertex and 16 per face cell
    # of every tile, per evaluation (and f's)
    if len(shape) == 3:
        tiles = -(-shape[0] // 16) * -(-shape[1] // 16) * -(-shape[2] // 16)
        faces = 1352
    else:
        tiles = -(-shape[0] // 32) * -(-shape[1] // 64)
        faces = 188
    assert 5 * n <= st["k_label_tile"]["units"] <= evals * (14 * n + 16 * faces * tiles)
    assert st["k_jump"]["work_launches"] >= evals
    # classification sweeps: one full, one incremental per apply
    assert c["sweeps"] == 1 + rounds + c["r_rounds"]
    plain.close()
    timed.close()


def test_kernel_stats_needs_timing_plan():
    msz = _msz()
    from paper_2406_09423_gb300 import native

    p = msz.Plan((16, 16), torch.float32)
    with pytest.raises(RuntimeError):
        native.msz_plan_kernel_stats(p._p)
    p.close()
