"""Thin ctypes binding of libmsz.so (include/msz.h). Argument marshalling only:
every step of the correction loop runs in the CUDA library.

The library is loaded from the package's ``_build`` directory; it must have
been built (``python -c "import __graft_entry__ as g; g.build()"``). There is
no CPU fallback: importing a function of this module on a machine without
the built library raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# MSZ_LIBRARY=checked selects the bounds-checked build (libmsz_checked.so)
LIB_PATH = os.path.join(HERE, "_build", "libmsz_checked.so" if os.environ.get("MSZ_LIBRARY") == "checked"
                        else "libmsz.so")

MSZ_F32, MSZ_F64 = 0, 1
MSZ_OPT_NO_TMA = 1
MSZ_OPT_TIME_KERNELS = 2
MSZ_OPT_TEST_STALL = 4
# msz_result.kernel_ms: classification (full sweep + incremental), labels
# (tile terminals + exit jumping), R-loop check, requests + apply
KERNEL_KINDS = ("classify", "labels", "rcheck", "mark_apply")
MSZ_NUM_KERNELS = 9
STATUS = {
    0: "MSZ_OK", -1: "MSZ_ERR_ARG", -2: "MSZ_ERR_DTYPE", -3: "MSZ_ERR_NONFINITE",
    -4: "MSZ_ERR_BOUND", -5: "MSZ_ERR_OOM", -6: "MSZ_ERR_NOCONVERGE", -7: "MSZ_ERR_TIMEOUT",
    -8: "MSZ_ERR_CUDA", -9: "MSZ_ERR_BUSY", -10: "MSZ_ERR_TOO_LARGE", -11: "MSZ_ERR_CANCELLED",
    -12: "MSZ_ERR_CHECK",
}

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


class MszCounts(ctypes.Structure):
    _fields_ = [
        ("sweeps", ctypes.c_uint64),
        ("c_rounds", ctypes.c_uint64 * 4),
        ("c_cases", ctypes.c_uint64 * 4),
        ("c_passes", ctypes.c_uint64),
        ("r_rounds", ctypes.c_uint64),
        ("r_cases", ctypes.c_uint64 * 2),
        ("label_evals", ctypes.c_uint64),
        ("mismatch", ctypes.c_uint64 * 2),
        ("dec_edits", ctypes.c_uint64),
        ("freezes", ctypes.c_uint64),
        ("edits", ctypes.c_uint64),
        ("freeze_req", ctypes.c_uint64 * 6),
        ("freeze_req_frozen", ctypes.c_uint64 * 6),
    ]

    def as_dict(self) -> dict:
        flat = [self.sweeps, *self.c_rounds, *self.c_cases, self.c_passes, self.r_rounds,
                *self.r_cases, self.label_evals, *self.mismatch, self.dec_edits, self.freezes,
                self.edits, *self.freeze_req, *self.freeze_req_frozen]
        return {k: int(v) for k, v in zip(COUNT_FIELDS, flat)}


class MszOptions(ctypes.Structure):
    _fields_ = [("max_rounds", ctypes.c_uint64), ("autotune", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_int32 * 6)]


TUNING_FIELDS = ("jumps_per_step", "chase_steps", "small_rounds", "small_cases", "graph_steps", "sweep_chunk",
                 "blocks_per_sm")


class MszTuning(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in TUNING_FIELDS] + [("reserved", ctypes.c_int32 * 5)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k in TUNING_FIELDS}

    @classmethod
    def from_dict(cls, d: dict) -> "MszTuning":
        t = cls()
        lib().msz_tuning_default(ctypes.byref(t))
        for k, v in d.items():
            setattr(t, k, int(v))
        return t


class MszResult(ctypes.Structure):
    _fields_ = [
        ("edit_idx", ctypes.c_void_p),
        ("edit_val", ctypes.c_void_p),
        ("n_edits", ctypes.c_uint64),
        ("label_max", ctypes.c_void_p),
        ("label_min", ctypes.c_void_p),
        ("counts", MszCounts),
        ("status", ctypes.c_int32),
        ("device_ms", ctypes.c_float),
        ("launches", ctypes.c_uint64),
        ("kernel_ms", ctypes.c_float * 4),
    ]


class MszKernelStat(ctypes.Structure):
    _fields_ = [
        ("name", ctypes.c_char_p),
        ("launches", ctypes.c_uint64),
        ("work_launches", ctypes.c_uint64),
        ("ms", ctypes.c_double),
        ("work_ms", ctypes.c_double),
        ("units", ctypes.c_uint64),
    ]


class MszMetricValues(ctypes.Structure):
    _fields_ = [
        ("mse", ctypes.c_double),
        ("value_range", ctypes.c_double),
        ("psnr", ctypes.c_double),
        ("right_labelled", ctypes.c_double),
        ("wrong", ctypes.c_uint64),
    ]


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libmsz.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, I, I64, U64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        L.msz_plan_create.argtypes = [ctypes.POINTER(P), I, P, I, P]
        L.msz_plan_create.restype = I
        L.msz_plan_bytes.argtypes = [I, P, I]
        L.msz_plan_bytes.restype = I64
        L.msz_plan_destroy.argtypes = [P]
        L.msz_plan_destroy.restype = I
        L.msz_plan_kernel_stats.argtypes = [P, ctypes.POINTER(MszKernelStat), I]
        L.msz_plan_kernel_stats.restype = I
        L.msz_fix.argtypes = [P, P, P, D, P, ctypes.POINTER(MszResult)]
        L.msz_fix.restype = I
        L.msz_fix_host.argtypes = [P, P, P, D, P, P, P, P, P, ctypes.POINTER(MszResult)]
        L.msz_fix_host.restype = I
        L.msz_apply.argtypes = [P, I, P, I, P, P, U64, P]
        L.msz_apply.restype = I
        L.msz_directions.argtypes = [P, I, P, I, P, P]
        L.msz_directions.restype = I
        L.msz_field_metrics.argtypes = [P, P, I, P, I, P, ctypes.POINTER(MszMetricValues)]
        L.msz_field_metrics.restype = I
        L.msz_edits_encoded_bound.argtypes = [U64, I]
        L.msz_edits_encoded_bound.restype = I64
        L.msz_encode_edits.argtypes = [P, P, U64, P, I, P, I, P, U64, ctypes.POINTER(U64), P]
        L.msz_encode_edits.restype = I
        L.msz_decode_edits.argtypes = [P, U64, P, I, P, I, P, P, U64, ctypes.POINTER(U64), P]
        L.msz_decode_edits.restype = I
        L.msz_batch_bytes.argtypes = [I, P, P, P]
        L.msz_batch_bytes.restype = I64
        L.msz_batch_create.argtypes = [ctypes.POINTER(P), I, P, P, P, P]
        L.msz_batch_create.restype = I
        L.msz_batch_fix.argtypes = [P, P, P, P, P, ctypes.POINTER(MszResult)]
        L.msz_batch_fix.restype = I
        L.msz_batch_destroy.argtypes = [P]
        L.msz_batch_destroy.restype = I
        L.msz_server_create.argtypes = [ctypes.POINTER(P), I64, I, P]
        L.msz_server_create.restype = I
        L.msz_server_submit.argtypes = [P, I, P, I, P, P, D, ctypes.POINTER(U64)]
        L.msz_server_submit.restype = I
        L.msz_server_poll.argtypes = [P, U64, I, ctypes.POINTER(MszResult)]
        L.msz_server_poll.restype = I
        L.msz_server_release.argtypes = [P, U64]
        L.msz_server_release.restype = I
        L.msz_server_cancel.argtypes = [P, U64]
        L.msz_server_cancel.restype = I
        L.msz_server_destroy.argtypes = [P]
        L.msz_server_destroy.restype = I
        L.msz_tuning_default.argtypes = [ctypes.POINTER(MszTuning)]
        L.msz_tuning_default.restype = None
        L.msz_tuning_valid.argtypes = [ctypes.POINTER(MszTuning)]
        L.msz_tuning_valid.restype = I
        for nm in ("msz_batch_set_tuning", "msz_batch_get_tuning", "msz_plan_set_tuning", "msz_plan_get_tuning"):
            getattr(L, nm).argtypes = [P, ctypes.POINTER(MszTuning)]
            getattr(L, nm).restype = I
        L.msz_batch_autotune.argtypes = [P, P, P, P, I, P, ctypes.POINTER(MszTuning), ctypes.POINTER(I)]
        L.msz_batch_autotune.restype = I
        L.msz_fix_noalloc.argtypes = [I, P, I, P, P, D, P, P, P, P, P, ctypes.POINTER(MszResult)]
        L.msz_fix_noalloc.restype = I
        L.msz_strerror.argtypes = [I]
        L.msz_strerror.restype = ctypes.c_char_p
        L.msz_version.restype = ctypes.c_char_p
        _lib = L
    return _lib


def dims_of(shape):
    """numpy/torch shape (ny, nx) or (nz, ny, nx) -> (ndim, int64[3] dims, x fastest)."""
    ndim = len(shape)
    if ndim not in (2, 3):
        raise ValueError("fields are 2D or 3D")
    d = [1, 1, 1]
    d[:ndim] = list(shape)[::-1]
    return ndim, (ctypes.c_int64 * 3)(*d)


def dtype_code(dtype) -> int:
    s = str(dtype)
    if s.endswith("float32"):
        return MSZ_F32
    if s.endswith("float64"):
        return MSZ_F64
    raise TypeError("float32 or float64 fields only")


def check(status: int, what: str = "msz"):
    if status != 0:
        raise RuntimeError(f"{what}: {STATUS.get(status, status)} ({lib().msz_strerror(status).decode()})")


# Same names as the C ABI ---------------------------------------------------

def msz_plan_create(shape, dtype, max_rounds: int = 0, flags: int = 0):
    ndim, d = dims_of(shape)
    opt = MszOptions()
    opt.max_rounds = max_rounds
    opt.flags = flags
    p = ctypes.c_void_p()
    st = lib().msz_plan_create(ctypes.byref(p), ndim, d, dtype_code(dtype), ctypes.byref(opt))
    check(st, "msz_plan_create")
    return p


def msz_plan_bytes(shape, dtype) -> int:
    ndim, d = dims_of(shape)
    return int(lib().msz_plan_bytes(ndim, d, dtype_code(dtype)))


def msz_plan_destroy(plan):
    check(lib().msz_plan_destroy(plan), "msz_plan_destroy")


def msz_plan_kernel_stats(plan) -> list[dict]:
    out = (MszKernelStat * MSZ_NUM_KERNELS)()
    m = lib().msz_plan_kernel_stats(plan, out, MSZ_NUM_KERNELS)
    check(m if m < 0 else 0, "msz_plan_kernel_stats")
    return [{"name": out[k].name.decode(), "launches": int(out[k].launches),
             "work_launches": int(out[k].work_launches), "ms": float(out[k].ms),
             "work_ms": float(out[k].work_ms), "units": int(out[k].units)} for k in range(m)]


def msz_fix(plan, orig_ptr: int, decomp_ptr: int, xi: float, stream: int = 0) -> MszResult:
    r = MszResult()
    lib().msz_fix(plan, ctypes.c_void_p(orig_ptr), ctypes.c_void_p(decomp_ptr), float(xi),
                  ctypes.c_void_p(stream), ctypes.byref(r))
    return r


def msz_fix_host(plan, orig_ptr: int, decomp_ptr: int, xi: float, edit_idx_ptr: int, edit_val_ptr: int,
                 label_max_ptr: int = 0, label_min_ptr: int = 0, stream: int = 0) -> MszResult:
    r = MszResult()
    lib().msz_fix_host(plan, ctypes.c_void_p(orig_ptr), ctypes.c_void_p(decomp_ptr), float(xi),
                       ctypes.c_void_p(edit_idx_ptr), ctypes.c_void_p(edit_val_ptr),
                       ctypes.c_void_p(label_max_ptr or None), ctypes.c_void_p(label_min_ptr or None),
                       ctypes.c_void_p(stream), ctypes.byref(r))
    return r


def _batch_arrays(shapes, dtypes):
    n = len(shapes)
    nd = (ctypes.c_int * n)()
    dims = (ctypes.c_int64 * (3 * n))()
    dts = (ctypes.c_int * n)()
    for i, (shp, dt) in enumerate(zip(shapes, dtypes)):
        k, d = dims_of(shp)
        nd[i] = k
        dims[3 * i:3 * i + 3] = list(d)
        dts[i] = dtype_code(dt)
    return n, nd, dims, dts


def msz_batch_bytes(shapes, dtypes) -> int:
    n, nd, dims, dts = _batch_arrays(shapes, dtypes)
    return int(lib().msz_batch_bytes(n, nd, dims, dts))


def msz_batch_create(shapes, dtypes, max_rounds: int = 0, flags: int = 0, autotune: bool = False):
    n, nd, dims, dts = _batch_arrays(shapes, dtypes)
    opt = MszOptions()
    opt.max_rounds = max_rounds
    opt.flags = flags
    opt.autotune = 1 if autotune else 0
    b = ctypes.c_void_p()
    check(lib().msz_batch_create(ctypes.byref(b), n, nd, dims, dts, ctypes.byref(opt)), "msz_batch_create")
    return b


def msz_batch_fix(batch, orig_ptrs, decomp_ptrs, xis, stream: int = 0):
    """Returns (status, [MszResult per field])."""
    n = len(orig_ptrs)
    fa = (ctypes.c_void_p * n)(*orig_ptrs)
    ha = (ctypes.c_void_p * n)(*decomp_ptrs)
    xa = (ctypes.c_double * n)(*[float(x) for x in xis])
    res = (MszResult * n)()
    st = lib().msz_batch_fix(batch, fa, ha, xa, ctypes.c_void_p(stream), res)
    return st, list(res)


def msz_tuning_default() -> dict:
    t = MszTuning()
    lib().msz_tuning_default(ctypes.byref(t))
    return t.as_dict()


def msz_tuning_valid(d: dict) -> int:
    return lib().msz_tuning_valid(ctypes.byref(MszTuning.from_dict(d)))


def msz_set_tuning(handle, d: dict, plan: bool = False):
    fn = lib().msz_plan_set_tuning if plan else lib().msz_batch_set_tuning
    check(fn(handle, ctypes.byref(MszTuning.from_dict(d))), "msz_set_tuning")


def msz_get_tuning(handle, plan: bool = False) -> dict:
    t = MszTuning()
    fn = lib().msz_plan_get_tuning if plan else lib().msz_batch_get_tuning
    check(fn(handle, ctypes.byref(t)), "msz_get_tuning")
    return t.as_dict()


def msz_batch_autotune(batch, orig_ptrs, decomp_ptrs, xis, force: bool = False, stream: int = 0):
    """(tuning dict, settings timed)."""
    n = len(orig_ptrs)
    fa = (ctypes.c_void_p * n)(*orig_ptrs)
    ha = (ctypes.c_void_p * n)(*decomp_ptrs)
    xa = (ctypes.c_double * n)(*[float(x) for x in xis])
    t = MszTuning()
    tried = ctypes.c_int(0)
    check(lib().msz_batch_autotune(batch, fa, ha, xa, 1 if force else 0, ctypes.c_void_p(stream), ctypes.byref(t),
                                   ctypes.byref(tried)), "msz_batch_autotune")
    return t.as_dict(), int(tried.value)


def msz_batch_destroy(batch):
    check(lib().msz_batch_destroy(batch), "msz_batch_destroy")


def msz_server_create(budget_bytes: int, max_slots: int = 64, max_rounds: int = 0, flags: int = 0):
    opt = MszOptions()
    opt.max_rounds = max_rounds
    opt.flags = flags
    srv = ctypes.c_void_p()
    check(lib().msz_server_create(ctypes.byref(srv), int(budget_bytes), int(max_slots), ctypes.byref(opt)),
          "msz_server_create")
    return srv


def msz_server_submit(srv, shape, dtype, orig_ptr: int, decomp_ptr: int, xi: float) -> int:
    ndim, d = dims_of(shape)
    rid = ctypes.c_uint64()
    check(lib().msz_server_submit(srv, ndim, d, dtype_code(dtype), ctypes.c_void_p(orig_ptr),
                                  ctypes.c_void_p(decomp_ptr), float(xi), ctypes.byref(rid)), "msz_server_submit")
    return int(rid.value)


def msz_server_poll(srv, request_id: int, wait_ms: int = 0):
    """(status, MszResult): status MSZ_OK when finished, MSZ_ERR_BUSY otherwise."""
    r = MszResult()
    st = lib().msz_server_poll(srv, int(request_id), int(wait_ms), ctypes.byref(r))
    return st, r


def msz_server_release(srv, request_id: int) -> int:
    return lib().msz_server_release(srv, int(request_id))


def msz_server_cancel(srv, request_id: int) -> int:
    return lib().msz_server_cancel(srv, int(request_id))


def msz_server_destroy(srv):
    check(lib().msz_server_destroy(srv), "msz_server_destroy")


def msz_fix_noalloc(shape, dtype, orig_ptr: int, decomp_ptr: int, xi: float, edit_idx_ptr: int,
                    edit_val_ptr: int, label_max_ptr: int, label_min_ptr: int, stream: int = 0) -> MszResult:
    """msz_fix with no device allocation (static scratch inside the library);
    all buffers are the caller's device memory."""
    ndim, d = dims_of(shape)
    r = MszResult()
    lib().msz_fix_noalloc(ndim, d, dtype_code(dtype), ctypes.c_void_p(orig_ptr), ctypes.c_void_p(decomp_ptr),
                          float(xi), ctypes.c_void_p(edit_idx_ptr), ctypes.c_void_p(edit_val_ptr),
                          ctypes.c_void_p(label_max_ptr), ctypes.c_void_p(label_min_ptr),
                          ctypes.c_void_p(stream), ctypes.byref(r))
    return r


def msz_apply(decomp_ptr: int, shape, dtype, edit_idx_ptr: int, edit_val_ptr: int, n_edits: int,
              stream: int = 0) -> int:
    ndim, d = dims_of(shape)
    return lib().msz_apply(ctypes.c_void_p(decomp_ptr), ndim, d, dtype_code(dtype),
                           ctypes.c_void_p(edit_idx_ptr), ctypes.c_void_p(edit_val_ptr),
                           int(n_edits), ctypes.c_void_p(stream))


def msz_directions(field_ptr: int, shape, dtype, dir_ptr: int, stream: int = 0) -> int:
    ndim, d = dims_of(shape)
    return lib().msz_directions(ctypes.c_void_p(field_ptr), ndim, d, dtype_code(dtype),
                                ctypes.c_void_p(dir_ptr), ctypes.c_void_p(stream))


def msz_field_metrics(f_ptr: int, g_ptr: int, shape, dtype, stream: int = 0):
    """(status, MszMetricValues) of g against f (device pointers)."""
    ndim, d = dims_of(shape)
    out = MszMetricValues()
    st = lib().msz_field_metrics(ctypes.c_void_p(f_ptr), ctypes.c_void_p(g_ptr), ndim, d, dtype_code(dtype),
                                 ctypes.c_void_p(stream), ctypes.byref(out))
    return st, out


def msz_edits_encoded_bound(n_edits: int, dtype) -> int:
    return lib().msz_edits_encoded_bound(int(n_edits), dtype_code(dtype))


def msz_encode_edits(idx_ptr: int, val_ptr: int, n_edits: int, fhat_ptr: int, shape, dtype, out_ptr: int,
                     out_cap: int, stream: int = 0):
    """(status, encoded bytes)."""
    ndim, d = dims_of(shape)
    nb = ctypes.c_uint64(0)
    st = lib().msz_encode_edits(ctypes.c_void_p(idx_ptr), ctypes.c_void_p(val_ptr), int(n_edits),
                                ctypes.c_void_p(fhat_ptr), ndim, d, dtype_code(dtype), ctypes.c_void_p(out_ptr),
                                int(out_cap), ctypes.byref(nb), ctypes.c_void_p(stream))
    return st, int(nb.value)


def msz_decode_edits(in_ptr: int, in_bytes: int, fhat_ptr: int, shape, dtype, idx_ptr: int, val_ptr: int,
                     cap_edits: int, stream: int = 0):
    """(status, number of edits)."""
    ndim, d = dims_of(shape)
    n = ctypes.c_uint64(0)
    st = lib().msz_decode_edits(ctypes.c_void_p(in_ptr), int(in_bytes), ctypes.c_void_p(fhat_ptr), ndim, d,
                                dtype_code(dtype), ctypes.c_void_p(idx_ptr), ctypes.c_void_p(val_ptr),
                                int(cap_edits), ctypes.byref(n), ctypes.c_void_p(stream))
    return st, int(n.value)


def msz_strerror(status: int) -> str:
    return lib().msz_strerror(status).decode()


def msz_version() -> str:
    return lib().msz_version().decode()
