"""CPU oracle for the MSz correction loop: test infrastructure only.

This package wraps ``msz_oracle.cpp``, a plain single-threaded C++
restatement of the MSz method (Li et al., Sec. 3-4: directions, labels,
false critical points of Definitions 1-3, the edits of Eqs. (2)-(6) and the
C/R-loop alternation). Only the tests, the smoke check and the CPU-baseline
leg of ``bench.py`` may import it. It shares no code with the CUDA library
and never imports it.

Parity status of each function (what pins it, see ``tests/test_oracle_*.py``):
  * directions / labels / false_bits: brute force on tiny grids, hand grids,
    closed forms (monotone ramps, single bumps).
  * bounds / decrease: exact rational arithmetic.
  * metrics: identical fields, exact shifts and single-vertex changes (closed
    forms), wrong-label counts against brute-force walks on tiny grids.
  * fix: invariants (bound, extremum sets, labels), special cases, six hand
    worked cases with their exact edits, counters and round trace (each of
    the targets of Eqs. (2)-(5) and both of Eq. (6), the paper's Fig. 5
    event chain), and the convergence argument of Sec. 4.3 checked round by
    round. Beyond those cases the particular edit values follow this
    restatement's readings and are otherwise "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msz_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libmsz_oracle.so")
_lock = threading.Lock()
_lib = None

COUNT_FIELDS = (
    "sweeps",
    "c_rounds_fpmax", "c_rounds_fpmin", "c_rounds_fnmax", "c_rounds_fnmin",
    "c_cases_fpmax", "c_cases_fpmin", "c_cases_fnmax", "c_cases_fnmin",
    "c_passes", "r_rounds", "r_cases_asc", "r_cases_desc", "label_evals",
    "mismatch_max", "mismatch_min", "dec_edits", "freezes", "edits",
    "freeze_req_fpmax", "freeze_req_fpmin", "freeze_req_fnmax", "freeze_req_fnmin",
    "freeze_req_rmax", "freeze_req_rmin",
    "freeze_req_frozen_fpmax", "freeze_req_frozen_fpmin", "freeze_req_frozen_fnmax",
    "freeze_req_frozen_fnmin", "freeze_req_frozen_rmax", "freeze_req_frozen_rmin",
)

STATUS = {0: "ok", -1: "arg", -2: "dtype", -3: "nonfinite", -4: "bound", -6: "noconverge"}


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++, no fast-math, no FMA contraction)."""
    with _lock:
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
            return _LIB_PATH
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        lib.oracle_counts_words.restype = ctypes.c_int
        lib.oracle_neighbours.argtypes = [ctypes.c_int, P, I64, P]
        lib.oracle_directions.argtypes = [ctypes.c_int, P, ctypes.c_int, P, P, P]
        lib.oracle_labels.argtypes = [ctypes.c_int, P, P, P]
        lib.oracle_false_bits.argtypes = [ctypes.c_int, P, ctypes.c_int, P, P, P]
        lib.oracle_troublemakers.argtypes = [ctypes.c_int, P, ctypes.c_int, P, P, P]
        lib.oracle_bounds.argtypes = [ctypes.c_int, I64, P, ctypes.c_double, P, P]
        lib.oracle_decrease.argtypes = [ctypes.c_int, I64, P, P, P]
        lib.oracle_fix.argtypes = [ctypes.c_int, P, ctypes.c_int, P, P, ctypes.c_double,
                                   ctypes.c_uint64, P, P, P, P, P, I64, P]
        assert lib.oracle_counts_words() == len(COUNT_FIELDS)
        _lib = lib
    return _lib


def _dims(shape):
    """numpy shape (ny, nx) or (nz, ny, nx) -> (ndim, int64[3] dims, x fastest)."""
    ndim = len(shape)
    if ndim not in (2, 3):
        raise ValueError("fields are 2D or 3D")
    d = np.ones(3, dtype=np.int64)
    d[:ndim] = shape[::-1]
    return ndim, d


def _dtype_code(a: np.ndarray) -> int:
    if a.dtype == np.float32:
        return 0
    if a.dtype == np.float64:
        return 1
    raise TypeError("float32 or float64 fields only")


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def neighbours(shape, v: int) -> list[int]:
    lib = _load()
    ndim, d = _dims(shape)
    out = np.zeros(14, dtype=np.int64)
    k = lib.oracle_neighbours(ndim, _ptr(d), int(v), _ptr(out))
    return [int(u) for u in out[:k]]


def directions(g: np.ndarray):
    """Steepest ascending / descending vertex (closed 1-ring) for every vertex."""
    lib = _load()
    g = np.ascontiguousarray(g)
    ndim, d = _dims(g.shape)
    up = np.empty(g.size, dtype=np.int64)
    dn = np.empty(g.size, dtype=np.int64)
    r = lib.oracle_directions(ndim, _ptr(d), _dtype_code(g), _ptr(g), _ptr(up), _ptr(dn))
    assert r == 0
    return up, dn


def labels(shape, direction: np.ndarray) -> np.ndarray:
    lib = _load()
    ndim, d = _dims(shape)
    direction = np.ascontiguousarray(direction, dtype=np.int64)
    lab = np.empty(direction.size, dtype=np.int32)
    assert lib.oracle_labels(ndim, _ptr(d), _ptr(direction), _ptr(lab)) == 0
    return lab


def metrics(f: np.ndarray, g: np.ndarray) -> dict:
    """Evaluation metrics of g against f (Appendix B), the plain definitions:
    mse = (1/N) sum (f_i - g_i)^2, the sum of the float64 squares rounded once
    (math.fsum); value_range = max f - min f; psnr = 20 log10(value_range /
    sqrt(mse)) (+inf for mse = 0); wrong = vertices whose maximum or minimum
    label (the fixed point of the steepest-neighbour walk, Sec. 3) differs
    between g and f; right_labelled = 1 - wrong / N."""
    import math

    f = np.ascontiguousarray(f)
    g = np.ascontiguousarray(g)
    assert f.shape == g.shape and f.dtype == g.dtype
    n = f.size
    f64 = f.astype(np.float64).ravel()
    d = f64 - g.astype(np.float64).ravel()
    mse = math.fsum((d * d).tolist()) / n
    rng = float(f64.max() - f64.min())
    psnr = math.inf if mse == 0.0 else 20.0 * math.log10(rng / math.sqrt(mse))
    uf, df = directions(f)
    ug, dg = directions(g)
    wrong = int(np.count_nonzero((labels(f.shape, uf) != labels(g.shape, ug)) |
                                 (labels(f.shape, df) != labels(g.shape, dg))))
    return {"mse": mse, "value_range": rng, "psnr": psnr, "wrong": wrong, "right_labelled": 1.0 - wrong / n}


def false_bits(f: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Per-vertex bit set: 1 FPmax, 2 FPmin, 4 FNmax, 8 FNmin."""
    lib = _load()
    f = np.ascontiguousarray(f)
    g = np.ascontiguousarray(g, dtype=f.dtype)
    ndim, d = _dims(f.shape)
    bits = np.empty(f.size, dtype=np.uint8)
    assert lib.oracle_false_bits(ndim, _ptr(d), _dtype_code(f), _ptr(f), _ptr(g), _ptr(bits)) == 0
    return bits


def troublemakers(f: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Per-vertex bits: 1 ascending troublemaker, 2 descending troublemaker."""
    lib = _load()
    f = np.ascontiguousarray(f)
    g = np.ascontiguousarray(g, dtype=f.dtype)
    ndim, d = _dims(f.shape)
    bits = np.empty(f.size, dtype=np.uint8)
    assert lib.oracle_troublemakers(ndim, _ptr(d), _dtype_code(f), _ptr(f), _ptr(g), _ptr(bits)) == 0
    return bits


def bounds(f: np.ndarray, xi: float):
    lib = _load()
    f = np.ascontiguousarray(f)
    lb = np.empty_like(f)
    ub = np.empty_like(f)
    assert lib.oracle_bounds(_dtype_code(f), f.size, _ptr(f), float(xi), _ptr(lb), _ptr(ub)) == 0
    return lb, ub


def decrease(g: np.ndarray, lb: np.ndarray) -> np.ndarray:
    lib = _load()
    g = np.ascontiguousarray(g)
    lb = np.ascontiguousarray(lb, dtype=g.dtype)
    out = np.empty_like(g)
    assert lib.oracle_decrease(_dtype_code(g), g.size, _ptr(g), _ptr(lb), _ptr(out)) == 0
    return out


class OracleResult:
    def __init__(self, status, g, label_max, label_min, counts, trace, edit_idx, edit_val):
        self.status = status
        self.g = g
        self.label_max = label_max
        self.label_min = label_min
        self.counts = counts
        self.trace = trace
        self.edit_idx = edit_idx
        self.edit_val = edit_val


def fix(f: np.ndarray, fhat: np.ndarray, xi: float, max_rounds: int = 10_000_000,
        trace_cap: int = 0) -> OracleResult:
    """Run the full correction loop. Returns g, labels, counts and the edit list."""
    lib = _load()
    f = np.ascontiguousarray(f)
    fhat = np.ascontiguousarray(fhat)
    if fhat.dtype != f.dtype or fhat.shape != f.shape:
        raise ValueError("f and fhat must share shape and dtype")
    ndim, d = _dims(f.shape)
    g = np.empty_like(f)
    M = np.empty(f.size, dtype=np.int32)
    m = np.empty(f.size, dtype=np.int32)
    counts = np.zeros(len(COUNT_FIELDS), dtype=np.uint64)
    tr = np.zeros((max(trace_cap, 1), 5), dtype=np.int64)
    tlen = np.zeros(1, dtype=np.int64)
    st = lib.oracle_fix(ndim, _ptr(d), _dtype_code(f), _ptr(f), _ptr(fhat), float(xi),
                        int(max_rounds), _ptr(g), _ptr(M), _ptr(m), _ptr(counts),
                        _ptr(tr), int(trace_cap), _ptr(tlen))
    cdict = {k: int(v) for k, v in zip(COUNT_FIELDS, counts)}
    gb = g.reshape(-1).view(np.uint32 if f.dtype == np.float32 else np.uint64)
    fb = fhat.reshape(-1).view(gb.dtype)
    idx = np.nonzero(gb != fb)[0].astype(np.uint32)
    vals = g.reshape(-1)[idx]
    trace = tr[: min(int(tlen[0]), trace_cap)] if trace_cap else None
    return OracleResult(st, g, M, m, cdict, trace, idx, vals)
