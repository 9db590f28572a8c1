"""The C-ABI library loads and exports every function include/msz.h declares
(no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(msz_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("msz_plan_create", "msz_plan_destroy", "msz_fix", "msz_apply", "msz_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2406_09423_gb300 import build

    lib_path = build.build()
    for path in (lib_path, build.LIB_CHECKED):  # the normal and the bounds-checked build
        lib = ctypes.CDLL(path)
        missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
        assert not missing, (path, missing)


def test_strerror_without_gpu():
    from paper_2406_09423_gb300 import native

    assert native.msz_strerror(-4) == "decompressed value outside the error bound"
    assert native.msz_strerror(-12) == "bounds check failed (checked build)"
    assert native.msz_version().startswith("msz-gb300")


def test_plan_bytes_and_argument_checks_without_gpu():
    from paper_2406_09423_gb300 import native

    assert native.msz_plan_bytes((512, 512, 512), "float32") > 512 ** 3 * 20
    L = native.lib()
    d = (ctypes.c_int64 * 3)(0, 4, 4)
    assert L.msz_plan_bytes(3, d, 0) == -1
    d = (ctypes.c_int64 * 3)(4, 4, 4)
    assert L.msz_plan_bytes(3, d, 7) == -2
    assert L.msz_plan_bytes(4, d, 0) == -1
    d = (ctypes.c_int64 * 3)(1 << 16, 1 << 16, 1)
    assert L.msz_plan_bytes(2, d, 0) == -1  # 2^32 vertices: too many


def test_no_device_is_an_error_not_a_fallback():
    # without a CUDA device every entry point fails loudly; plan creation
    # names the cause (a CUDA error, not a memory shortage)
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    import paper_2406_09423_gb300 as msz

    f = torch.zeros((8, 9))
    with pytest.raises(RuntimeError, match="MSZ_ERR_CUDA"):
        msz.Plan((8, 9), torch.float32)
    with pytest.raises(RuntimeError):
        msz.fix(f, f.clone(), 0.1)
    with pytest.raises(RuntimeError):
        msz.directions(f)


def test_tuning_defaults_and_validation_without_gpu():
    from paper_2406_09423_gb300 import native

    d = native.msz_tuning_default()
    assert d == {"jumps_per_step": 2, "chase_steps": 32, "small_rounds": 64, "small_cases": 65536,
                 "graph_steps": 4, "sweep_chunk": 64, "blocks_per_sm": 0}
    assert native.msz_tuning_valid(d) == 0
    for k, bad in (("jumps_per_step", 5), ("chase_steps", 3), ("small_rounds", -1), ("small_cases", 0),
                   ("graph_steps", 0), ("sweep_chunk", 3), ("blocks_per_sm", 65)):
        assert native.msz_tuning_valid(dict(d, **{k: bad})) == -1, k
    t = native.MszTuning.from_dict(d)
    t.reserved[2] = 1
    assert native.lib().msz_tuning_valid(ctypes.byref(t)) == -1
