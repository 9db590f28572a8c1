"""Seeded synthetic fields and the error-bounded quantiser.

The paper evaluates MSz on simulation outputs (Nyx cosmology, viscous
fingering, CESM, Red Sea, ...) compressed by SZ3 / ZFP (Sec. 6-7). Neither
the datasets nor the compressors are available here, so every input is a
seeded synthetic field with the shape and spectral character of those data,
and the compressor is replaced by a deterministic uniform quantiser
``xhat = round(x / 2xi) * 2xi`` that respects the absolute bound xi.

This module holds no part of the MSz method: it only makes inputs. Both the
CUDA path and the CPU oracle are fed from it. Arrays are numpy (or torch,
for the large 3D generators when a device is given) in C order with x the
fastest axis: 2D fields have shape (ny, nx), 3D fields (nz, ny, nx).
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

# ---------------------------------------------------------------------------
# Fields
# ---------------------------------------------------------------------------


def _gauss_sum_2d(nx, ny, cx, cy, sigma, amp):
    """sum_e amp_e * exp(-((x-cx_e)^2 + (y-cy_e)^2) / (2 sigma_e^2)) on the grid,
    evaluated separably (float64)."""
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    gx = np.exp(-((x[None, :] - cx[:, None]) ** 2) / (2.0 * sigma[:, None] ** 2))  # (E, nx)
    gy = np.exp(-((y[None, :] - cy[:, None]) ** 2) / (2.0 * sigma[:, None] ** 2))  # (E, ny)
    return (gy * amp[:, None]).T @ gx  # (ny, nx)


def bumps2d(nx=128, ny=128, seed=0, nbumps=16, noise=1e-3, dtype=np.float32):
    """Sum of Gaussian bumps plus white noise: centres uniform on the grid,
    sigma uniform in [4, 16] px, amplitudes uniform in [-1, 1]."""
    rng = np.random.default_rng(seed)
    cx = rng.uniform(0, nx, nbumps)
    cy = rng.uniform(0, ny, nbumps)
    sigma = rng.uniform(4, 16, nbumps)
    amp = rng.uniform(-1, 1, nbumps)
    f = _gauss_sum_2d(nx, ny, cx, cy, sigma, amp)
    f += rng.normal(0.0, noise, (ny, nx))
    return f.astype(dtype)


def lognormal3d(n=256, seed=1, dtype=np.float32, shape=None):
    """Cosmology-like density: Gaussian random field with power spectrum
    P(k) ~ k^-3 (amplitude k^-3/2, |k| in integer grid units, k = 0 removed),
    standardised to zero mean / unit variance, then exponentiated."""
    shape = tuple(shape) if shape is not None else (n, n, n)
    rng = np.random.default_rng(seed)
    white = rng.standard_normal(shape)
    F = np.fft.rfftn(white)
    kz = np.fft.fftfreq(shape[0]) * shape[0]
    ky = np.fft.fftfreq(shape[1]) * shape[1]
    kx = np.fft.rfftfreq(shape[2]) * shape[2]
    k = np.sqrt(kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2)
    with np.errstate(divide="ignore"):
        filt = np.where(k > 0, k ** -1.5, 0.0)
    g = np.fft.irfftn(F * filt, s=shape, axes=(0, 1, 2))
    g = (g - g.mean()) / g.std()
    return np.exp(g).astype(dtype)


def ocean2d(nx=3600, ny=2400, seed=2, neddies=400, dtype=np.float32):
    """Ocean-like field: meridional gradient y/(ny-1) plus Gaussian eddies
    (radius 10-60 px used as sigma, amplitude uniform in [-0.3, 0.3]) plus
    N(0, 1e-3) noise."""
    rng = np.random.default_rng(seed)
    cx = rng.uniform(0, nx, neddies)
    cy = rng.uniform(0, ny, neddies)
    radius = rng.uniform(10, 60, neddies)
    amp = rng.uniform(-0.3, 0.3, neddies)
    f = _gauss_sum_2d(nx, ny, cx, cy, radius, amp)
    f += (np.arange(ny, dtype=np.float64) / max(ny - 1, 1))[:, None]
    f += rng.normal(0.0, 1e-3, (ny, nx))
    return f.astype(dtype)


def _turbulence_modes(seed, nmodes, kmax):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((nmodes, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    kmag = np.exp(rng.uniform(0.0, math.log(kmax), nmodes))
    phase = rng.uniform(0.0, 2.0 * math.pi, nmodes)
    k = d * kmag[:, None]  # cycles per box, (kx, ky, kz)
    amp = kmag ** (-5.0 / 6.0)
    return k, amp, phase


def turbulence3d(n=512, seed=3, nmodes=256, kmax=64.0, dtype=np.float32, device=None,
                 shape=None):
    """Turbulence-like field: 256 random-phase sinusoidal modes,
    f = sum_m A_m sin(2 pi k_m . x / n + phi_m), directions uniform on the
    sphere, |k| log-uniform in [1, kmax] cycles per box, A = |k|^(-5/6)
    (a Kolmogorov -5/3 energy spectrum).

    Evaluated separably in complex128: for each z-plane the mode sum is a
    (ny x M) @ (M x nx) product. With ``device`` (a torch CUDA device) the
    products run on the GPU and a torch tensor is returned."""
    L = float(n if shape is None else max(shape))
    shape = tuple(shape) if shape is not None else (n, n, n)
    nz, ny, nx = shape
    k, amp, phase = _turbulence_modes(seed, nmodes, kmax)
    c = amp * np.exp(1j * phase)
    ex = np.exp(2j * math.pi * np.outer(np.arange(nx), k[:, 0]) / L)  # (nx, M)
    ey = np.exp(2j * math.pi * np.outer(np.arange(ny), k[:, 1]) / L)  # (ny, M)
    ez = np.exp(2j * math.pi * np.outer(np.arange(nz), k[:, 2]) / L)  # (nz, M)
    if device is None:
        out = np.empty(shape, dtype=dtype)
        exT = ex.T.copy()
        for z in range(nz):
            out[z] = ((ey * (c * ez[z])[None, :]) @ exT).imag.astype(dtype)
        return out
    import torch

    tdt = torch.float32 if dtype == np.float32 else torch.float64
    ex_t = torch.from_numpy(ex.T.copy()).to(device)
    ey_t = torch.from_numpy(ey).to(device)
    cz_t = torch.from_numpy(c[None, :] * ez).to(device)  # (nz, M)
    out = torch.empty(shape, dtype=tdt, device=device)
    step = 16
    for z0 in range(0, nz, step):
        z1 = min(nz, z0 + step)
        a = ey_t[None, :, :] * cz_t[z0:z1, None, :]  # (b, ny, M)
        out[z0:z1] = torch.matmul(a, ex_t).imag.to(tdt)
    return out


# ---------------------------------------------------------------------------
# Error bound and quantiser (stand-in for SZ3 / ZFP)
# ---------------------------------------------------------------------------


def value_range(f) -> float:
    """max - min of the field, in float64."""
    if hasattr(f, "detach"):
        return float(f.max().item()) - float(f.min().item())
    return float(np.max(f)) - float(np.min(f))


def xi_for(f, rel: float) -> float:
    """Absolute bound xi = rel * range, rounded once to the field's dtype."""
    dt = np.float32 if str(getattr(f, "dtype", "")).endswith("float32") else np.float64
    return float(dt(rel * value_range(f)))


def _exact_within(x: np.ndarray, q: np.ndarray, xi: float) -> np.ndarray:
    """Exact test |q - x| <= xi (elementwise) for float arrays of one dtype."""
    wide = np.float64 if x.dtype == np.float32 else np.longdouble
    d = np.abs(q.astype(wide) - x.astype(wide))
    ok = d <= wide(xi)
    near = np.abs(d - wide(xi)) <= wide(xi) * wide(1e-6)
    for i in np.flatnonzero(near):
        ok.flat[i] = abs(Fraction(float(q.flat[i])) - Fraction(float(x.flat[i]))) <= Fraction(xi)
    return ok


def quantise(f: np.ndarray, xi: float) -> np.ndarray:
    """xhat = RN_dtype(rint(x / 2xi) * 2xi) computed in float64 (ties to even),
    then moved one ulp at a time towards x until |xhat - x| <= xi exactly."""
    f = np.asarray(f)
    dt = f.dtype.type
    xi = float(dt(xi))
    if xi == 0.0:
        return f.copy()
    step = 2.0 * xi
    q = (np.rint(f.astype(np.float64) / step) * step).astype(f.dtype)
    for _ in range(64):
        bad = ~_exact_within(f, q, xi)
        if not bad.any():
            return q
        q[bad] = np.nextafter(q[bad], f[bad])
    raise RuntimeError("quantiser did not reach the bound")


def quantise_torch(f, xi: float):
    """GPU version of ``quantise`` for large torch fields (same definition;
    the bound test runs in float64, exact for float32 inputs)."""
    import torch

    xi = float(np.float32(xi)) if f.dtype == torch.float32 else float(xi)
    if xi == 0.0:
        return f.clone()
    step = 2.0 * xi
    q = (torch.round(f.double() / step) * step).to(f.dtype)
    if f.dtype != torch.float32:
        raise TypeError("quantise_torch handles float32 fields")
    for _ in range(64):
        bad = (q.double() - f.double()).abs() > xi
        if not bool(bad.any()):
            return q
        q = torch.where(bad, torch.nextafter(q, f), q)
    raise RuntimeError("quantiser did not reach the bound")


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------


def workload(name: str, rel: float | None = None, device=None):
    """Named workloads: returns (f, fhat, xi).

    bumps128   : 2D 128x128 f32 bumps, seed 0, xi = 1e-3 * range
    lognormal256 : 3D 256^3 f32 lognormal, seed 1
    ocean      : 2D 3600x2400 f32, seed 2
    turb512    : 3D 512^3 f32 turbulence, seed 3
    """
    if name == "bumps128":
        f = bumps2d(128, 128, 0)
        rel = 1e-3 if rel is None else rel
    elif name == "lognormal256":
        f = lognormal3d(256, 1)
        rel = 1e-3 if rel is None else rel
    elif name == "ocean":
        f = ocean2d(3600, 2400, 2)
        rel = 1e-3 if rel is None else rel
    elif name == "turb512":
        f = turbulence3d(512, 3, device=device)
        rel = 1e-3 if rel is None else rel
    else:
        raise KeyError(name)
    xi = xi_for(f, rel)
    if device is not None and hasattr(f, "detach"):
        return f, quantise_torch(f, xi), xi
    return f, quantise(f, xi), xi


def batch_fields(count=64, first_seed=100):
    """Mixed batch: fields i < count/2 are 2D (sides uniform in [64, 1024],
    bump count 16*ceil(area/128^2) capped at 1024), the rest 3D (sides uniform
    in [32, 192], lognormal for even i, turbulence with |k| <= side/8 for odd
    i). float32 for even i, float64 for odd i; xi = 10^U(-5,-3) * range.
    Yields (f, fhat, xi) per field."""
    half = count // 2
    for i in range(count):
        seed = first_seed + i
        rng = np.random.default_rng(seed)
        dt = np.float32 if i % 2 == 0 else np.float64
        if i < half:
            nx, ny = (int(v) for v in rng.integers(64, 1025, 2))
            nb = min(1024, 16 * math.ceil(nx * ny / 128 ** 2))
            f = bumps2d(nx, ny, seed, nbumps=nb, dtype=dt)
        else:
            sx, sy, sz = (int(v) for v in rng.integers(32, 193, 3))
            if i % 2 == 0:
                f = lognormal3d(seed=seed, dtype=dt, shape=(sz, sy, sx))
            else:
                side = max(sx, sy, sz)
                f = turbulence3d(side, seed, kmax=max(1.0, side / 8), dtype=dt, shape=(sz, sy, sx))
        rel = 10.0 ** rng.uniform(-5, -3)
        xi = xi_for(f, rel)
        yield f, quantise(f, xi), xi
