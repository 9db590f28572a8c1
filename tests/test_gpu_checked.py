"""The bounds-checked build (libmsz_checked.so, compiled with MSZ_CHECKED):
every index the kernels read from device data - list entries and slots,
tile pointers, decoded terminals, exit-table ranks - is checked before use,
and an index out of range records an error (MSZ_ERR_CHECK) instead of an
access. The parity cases run through that build in a separate process
(tests/checked_parity.py) must give the oracle's results with no check
firing."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_parity():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_09423_gb300 import build

    build.build()
    assert os.path.exists(build.LIB_CHECKED)
    env = dict(os.environ, MSZ_LIBRARY="checked")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_parity.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked parity ok" in r.stdout
