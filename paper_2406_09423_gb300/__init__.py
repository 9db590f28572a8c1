"""GB300-native MSz: preserves the piecewise-linear Morse-Smale segmentation
of a scalar field through error-bounded lossy compression by editing the
decompressed field (Li et al., MSz, Sec. 4-5).

The correction loop runs entirely in libmsz.so (hand-written CUDA for
sm_103a, C ABI in include/msz.h). This package only moves torch tensors in
and out of that library:

    import torch, paper_2406_09423_gb300 as msz
    res = msz.fix(f, fhat, xi)           # f, fhat: CUDA tensors (ny, nx) or (nz, ny, nx)
    g = fhat.clone(); msz.apply(g, res.edit_idx, res.edit_val)
"""
from __future__ import annotations

from dataclasses import dataclass

from . import native

__all__ = ["Plan", "Batch", "Server", "FixResult", "fix", "apply", "directions", "field_metrics", "encode_edits", "decode_edits", "native"]


def _torch():
    import torch

    return torch


class _DeviceArray:
    """__cuda_array_interface__ view of plan-owned device memory."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {
            "shape": (n,), "typestr": typestr, "data": (int(ptr), False), "version": 3, "strides": None,
        }


def _view(torch, ptr, n, dtype):
    typestr = {torch.float32: "<f4", torch.float64: "<f8", torch.int32: "<i4", torch.uint32: "<u4"}[dtype]
    if n == 0 or not ptr:
        return torch.empty(0, dtype=dtype, device="cuda")
    return torch.as_tensor(_DeviceArray(ptr, n, typestr), device="cuda")


@dataclass
class FixResult:
    edit_idx: "object"     # int64 tensor (ascending vertex indices)
    edit_val: "object"     # new values, field dtype
    label_max: "object"    # int32 tensor, field shape
    label_min: "object"
    counts: dict
    status: int
    device_ms: float
    launches: int = 0
    kernel_ms: dict = None

    @property
    def n_edits(self) -> int:
        return int(self.edit_idx.numel())


def _result(torch, r, shape, dtype, copy):
    n = 1
    for s_ in shape:
        n *= int(s_)
    ok = r.status == 0
    # a fix stopped by the round cap still returns its edits so far
    ne = int(r.n_edits) if (ok or r.status == -6) and r.edit_idx else 0
    idx = _view(torch, r.edit_idx, ne, torch.int32)
    val = _view(torch, r.edit_val, ne, dtype)
    lmax = _view(torch, r.label_max, n if ok else 0, torch.int32)
    lmin = _view(torch, r.label_min, n if ok else 0, torch.int32)
    if copy:
        idx, val, lmax, lmin = idx.long(), val.clone(), lmax.clone(), lmin.clone()
    if ok:
        lmax = lmax.view(tuple(shape))
        lmin = lmin.view(tuple(shape))
    kms = {k: float(v) for k, v in zip(native.KERNEL_KINDS, r.kernel_ms)}
    return FixResult(idx, val, lmax, lmin, r.counts.as_dict(), int(r.status), float(r.device_ms),
                     int(r.launches), kms)


class Batch:
    """Many fields of uneven shapes and mixed float32 / float64, corrected
    together (msz_batch_create / msz_batch_fix); each result equals msz_fix
    on that field alone."""

    def __init__(self, shapes, dtypes, max_rounds: int = 0, use_tma: bool = True, flags: int = 0,
                 autotune: bool = False):
        self.shapes = [tuple(int(v) for v in s_) for s_ in shapes]
        self.dtypes = list(dtypes)
        flags |= 0 if use_tma else native.MSZ_OPT_NO_TMA
        self._b = native.msz_batch_create(self.shapes, self.dtypes, max_rounds, flags, autotune)

    def autotune(self, fs, fhats, xis, force: bool = False):
        """msz_batch_autotune on these inputs: (applied tuning, settings timed)."""
        torch = _torch()
        fs = [f.contiguous() for f in fs]
        fhats = [h.contiguous() for h in fhats]
        return native.msz_batch_autotune(self._b, [f.data_ptr() for f in fs], [h.data_ptr() for h in fhats], xis,
                                         force, torch.cuda.current_stream().cuda_stream)

    @property
    def tuning(self) -> dict:
        return native.msz_get_tuning(self._b)

    @tuning.setter
    def tuning(self, d: dict):
        native.msz_set_tuning(self._b, d)

    def fix(self, fs, fhats, xis, copy: bool = True):
        torch = _torch()
        if not (len(fs) == len(fhats) == len(xis) == len(self.shapes)):
            raise ValueError("one f, fhat and xi per field")
        fs = [f.contiguous() for f in fs]
        fhats = [h.contiguous() for h in fhats]
        for f, h, shp, dt in zip(fs, fhats, self.shapes, self.dtypes):
            if tuple(f.shape) != shp or tuple(h.shape) != shp or f.dtype != dt or h.dtype != dt or not f.is_cuda:
                raise ValueError("fields must match the batch's shapes and dtypes (CUDA tensors)")
        stream = torch.cuda.current_stream().cuda_stream
        st, res = native.msz_batch_fix(self._b, [f.data_ptr() for f in fs], [h.data_ptr() for h in fhats], xis,
                                       stream)
        return st, [_result(torch, r, shp, dt, copy) for r, shp, dt in zip(res, self.shapes, self.dtypes)]

    def close(self):
        if self._b:
            native.msz_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching correction service (msz_server_*): fields are
    admitted as slots and memory allow and corrected together with the
    fields already resident; each result equals msz_fix on that field."""

    def __init__(self, budget_bytes: int, max_slots: int = 64, max_rounds: int = 0, use_tma: bool = True,
                 flags: int = 0):
        flags |= 0 if use_tma else native.MSZ_OPT_NO_TMA
        self._s = native.msz_server_create(budget_bytes, max_slots, max_rounds, flags)
        self._inputs = {}

    def submit(self, f, fhat, xi: float) -> int:
        """Queues a correction; f and fhat (CUDA tensors) must stay alive and
        unchanged until the request finishes."""
        torch = _torch()
        f = f.contiguous()
        fhat = fhat.contiguous()
        torch.cuda.current_stream().synchronize()  # inputs ready before the worker reads them
        rid = native.msz_server_submit(self._s, tuple(f.shape), f.dtype, f.data_ptr(), fhat.data_ptr(), xi)
        self._inputs[rid] = (f, fhat)
        return rid

    def poll(self, rid: int, wait_ms: int = 0, copy: bool = True):
        """FixResult when finished (and released if copy), else None. The
        result's device_ms is the submit-to-result latency."""
        torch = _torch()
        st, r = native.msz_server_poll(self._s, rid, wait_ms)
        if st == -9:
            return None
        native.check(st, "msz_server_poll")
        f, _ = self._inputs[rid]
        res = _result(torch, r, tuple(f.shape), f.dtype, copy)
        if copy:
            torch.cuda.synchronize()
            native.msz_server_release(self._s, rid)
            del self._inputs[rid]
        return res

    def release(self, rid: int):
        native.msz_server_release(self._s, rid)
        self._inputs.pop(rid, None)

    def cancel(self, rid: int) -> int:
        """msz_server_cancel: the request finishes with MSZ_ERR_CANCELLED (its
        inputs stay referenced until it is polled or released)."""
        return native.msz_server_cancel(self._s, rid)

    def close(self):
        if self._s:
            native.msz_server_destroy(self._s)
            self._s = None
            self._inputs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """Device state for fields of one shape and dtype (msz_plan_create)."""

    def __init__(self, shape, dtype, max_rounds: int = 0, use_tma: bool = True, time_kernels: bool = False,
                 flags: int = 0):
        self.shape = tuple(int(s) for s in shape)
        self.dtype = dtype
        flags |= (0 if use_tma else native.MSZ_OPT_NO_TMA) | (native.MSZ_OPT_TIME_KERNELS if time_kernels else 0)
        self._p = native.msz_plan_create(self.shape, dtype, max_rounds, flags)

    def fix(self, f, fhat, xi: float, copy: bool = True, check: bool = True) -> FixResult:
        torch = _torch()
        if f.shape != fhat.shape or tuple(f.shape) != self.shape or f.dtype != fhat.dtype:
            raise ValueError("f and fhat must match the plan's shape and dtype")
        if not (f.is_cuda and fhat.is_cuda):
            raise ValueError("f and fhat must be CUDA tensors")
        f = f.contiguous()
        fhat = fhat.contiguous()
        stream = torch.cuda.current_stream().cuda_stream
        r = native.msz_fix(self._p, f.data_ptr(), fhat.data_ptr(), xi, stream)
        if check:
            native.check(r.status, "msz_fix")
        return _result(torch, r, self.shape, f.dtype, copy)

    @property
    def tuning(self) -> dict:
        return native.msz_get_tuning(self._p, plan=True)

    @tuning.setter
    def tuning(self, d: dict):
        native.msz_set_tuning(self._p, d, plan=True)

    def kernel_stats(self) -> list[dict]:
        """Per-kernel launches, device times and work units of the last fix
        (plans made with time_kernels=True; msz_plan_kernel_stats)."""
        return native.msz_plan_kernel_stats(self._p)

    def close(self):
        if self._p:
            native.msz_plan_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fix(f, fhat, xi: float, max_rounds: int = 0) -> FixResult:
    """One-shot correction loop (plan + msz_fix + copy of the results)."""
    plan = Plan(tuple(f.shape), f.dtype, max_rounds)
    try:
        return plan.fix(f, fhat, xi)
    finally:
        plan.close()


def apply(decomp, edit_idx, edit_val) -> None:
    """Writes the edits into ``decomp`` in place (msz_apply)."""
    torch = _torch()
    idx = edit_idx.to(device=decomp.device, dtype=torch.int32).contiguous()
    val = edit_val.to(device=decomp.device, dtype=decomp.dtype).contiguous()
    st = native.msz_apply(decomp.data_ptr(), tuple(decomp.shape), decomp.dtype, idx.data_ptr(),
                          val.data_ptr(), int(idx.numel()), torch.cuda.current_stream().cuda_stream)
    native.check(st, "msz_apply")


def field_metrics(f, g) -> dict:
    """Appendix B metrics of g against f (CUDA tensors of one shape and
    dtype): mse, value_range, psnr, wrong (vertices with a wrong maximum or
    minimum label) and right_labelled (msz_field_metrics)."""
    torch = _torch()
    if f.shape != g.shape or f.dtype != g.dtype:
        raise ValueError("f and g must have one shape and dtype")
    f, g = f.contiguous(), g.contiguous()
    st, m = native.msz_field_metrics(f.data_ptr(), g.data_ptr(), tuple(f.shape), f.dtype,
                                     torch.cuda.current_stream().cuda_stream)
    native.check(st, "msz_field_metrics")
    return {"mse": m.mse, "value_range": m.value_range, "psnr": m.psnr, "wrong": int(m.wrong),
            "right_labelled": m.right_labelled}


def encode_edits(edit_idx, edit_val, fhat):
    """Lossless coding of an edit list (Sec. 5.3; msz_encode_edits): a uint8
    CUDA tensor holding the encoded bytes. edit_idx ascending, edit_val the
    new values, fhat the field they replace (CUDA tensors)."""
    torch = _torch()
    idx = edit_idx.to(device=fhat.device, dtype=torch.int32).contiguous()
    val = edit_val.to(device=fhat.device, dtype=fhat.dtype).contiguous()
    fh = fhat.contiguous()
    n = int(idx.numel())
    cap = native.msz_edits_encoded_bound(n, fh.dtype)
    native.check(cap if cap < 0 else 0, "msz_edits_encoded_bound")
    out = torch.empty(cap, dtype=torch.uint8, device=fh.device)
    st, nb = native.msz_encode_edits(idx.data_ptr(), val.data_ptr(), n, fh.data_ptr(), tuple(fh.shape), fh.dtype,
                                     out.data_ptr(), cap, torch.cuda.current_stream().cuda_stream)
    native.check(st, "msz_encode_edits")
    return out[:nb]


def decode_edits(data, fhat, cap_edits=None):
    """(edit_idx int32, edit_val) of an encoded edit list (msz_decode_edits)."""
    torch = _torch()
    data = data.to(device=fhat.device, dtype=torch.uint8).contiguous()
    fh = fhat.contiguous()
    cap = fh.numel() if cap_edits is None else int(cap_edits)
    idx = torch.empty(cap, dtype=torch.int32, device=fh.device)
    val = torch.empty(cap, dtype=fh.dtype, device=fh.device)
    st, n = native.msz_decode_edits(data.data_ptr(), int(data.numel()), fh.data_ptr(), tuple(fh.shape), fh.dtype,
                                    idx.data_ptr(), val.data_ptr(), cap, torch.cuda.current_stream().cuda_stream)
    native.check(st, "msz_decode_edits")
    return idx[:n], val[:n]


def directions(field):
    """Direction byte per vertex (ascending slot | descending slot << 4)."""
    torch = _torch()
    out = torch.empty(field.shape, dtype=torch.uint8, device=field.device)
    st = native.msz_directions(field.contiguous().data_ptr(), tuple(field.shape), field.dtype,
                               out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    native.check(st, "msz_directions")
    return out
