"""Seeded synthetic fields and the error-bounded quantiser.

The paper evaluates MSz on simulation outputs (Nyx cosmology, viscous
fingering, CESM, Red Sea, ...) compressed by SZ3 / ZFP (Sec. 6-7). Neither
the datasets nor the compressors are available here, so every input is a
seeded synthetic field with the shape and spectral character of those data,
and the compressor is replaced by a deterministic uniform quantiser
``xhat = round(x / 2xi) * 2xi`` that respects the absolute bound xi.

This module holds no part of the MSz method: it only makes inputs. Both the
CUDA path and the CPU oracle are fed from it. Arrays are numpy (or torch,
when a device is given) in C order with x the fastest axis: 2D fields have
shape (ny, nx), 3D fields (nz, ny, nx).

Bit-reproducible generation. A field must come out with the same bits on
every machine and in both array libraries, so that results stored on one
host (oracle outputs, hashes) can be checked against a run on another. So
every generator is built only from operations that IEEE 754 rounds exactly
once: +, -, *, / and sqrt on float64, elementwise, in a fixed order. No
library exp / log / sin / cos, no BLAS product and no library FFT (their last
bits differ between CPUs and libraries). Those are replaced by the
elementary functions below, restated from their series with argument
reduction (Cody and Waite's split of the reduction constant), a radix-2 FFT
written out as butterflies, and a reduction whose summation tree is fixed.
The random numbers are numpy's PCG64 stream read as uniform doubles
(``Generator.random``, an exact bit conversion), so normal deviates come
from the Box-Muller transform computed here.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

# ---------------------------------------------------------------------------
# Array backends: numpy on the host, torch on a device. The arithmetic is
# written once with Python operators; each operator is one elementwise
# IEEE-rounded operation in either library. On the torch side a division
# always has a tensor divisor (see _Torch.scalar).
# ---------------------------------------------------------------------------


class _Numpy:
    def zeros(self, shape):
        return np.zeros(shape, dtype=np.float64)

    def asarray(self, a):
        return np.asarray(a, dtype=np.float64)

    def rint(self, x):
        return np.rint(x)

    def where(self, c, a, b):
        return np.where(c, a, b)

    def sqrt(self, x):
        return np.sqrt(x)

    def bits(self, x):
        return x.view(np.int64)

    def from_bits(self, i):
        return i.view(np.float64)

    def to_int(self, x):
        return x.astype(np.int64)

    def to_float(self, i):
        return i.astype(np.float64)

    def cat(self, xs, axis=0):
        return np.concatenate(xs, axis=axis)

    def stack(self, xs, axis):
        return np.stack(xs, axis=axis)

    def moveaxis(self, x, a, b):
        return np.moveaxis(x, a, b)

    def contiguous(self, x):
        return np.ascontiguousarray(x)

    def take(self, x, idx, axis):
        return np.take(x, idx, axis=axis)

    def item(self, x):
        return float(x)

    def scalar(self, v):
        return np.float64(v)

    def out(self, x, dtype):
        return x.astype(dtype)


class _Torch:
    def __init__(self, device):
        import torch

        self.t = torch
        self.dev = torch.device(device)

    def zeros(self, shape):
        return self.t.zeros(shape, dtype=self.t.float64, device=self.dev)

    def asarray(self, a):
        return self.t.as_tensor(np.asarray(a, dtype=np.float64), device=self.dev)

    def rint(self, x):
        return self.t.round(x)  # ties to even, like numpy's rint

    def where(self, c, a, b):
        t = self.t
        a = a if isinstance(a, t.Tensor) else t.tensor(a, dtype=t.float64, device=self.dev)
        b = b if isinstance(b, t.Tensor) else t.tensor(b, dtype=t.float64, device=self.dev)
        return t.where(c, a, b)

    def sqrt(self, x):
        return self.t.sqrt(x)

    def bits(self, x):
        return x.contiguous().view(self.t.int64)

    def from_bits(self, i):
        return i.contiguous().view(self.t.float64)

    def to_int(self, x):
        return x.to(self.t.int64)

    def to_float(self, i):
        return i.to(self.t.float64)

    def cat(self, xs, axis=0):
        return self.t.cat(xs, dim=axis)

    def stack(self, xs, axis):
        return self.t.stack(xs, dim=axis)

    def moveaxis(self, x, a, b):
        return self.t.movedim(x, a, b)

    def contiguous(self, x):
        return x.contiguous()

    def take(self, x, idx, axis):
        return self.t.index_select(x, axis, self.t.as_tensor(idx, device=self.dev))

    def item(self, x):
        return float(x.item())

    def scalar(self, v):
        # a 0-dim tensor on the device: CUDA kernels divide by a host scalar
        # through its reciprocal (two roundings), by a device tensor exactly
        return self.t.tensor(float(v), dtype=self.t.float64, device=self.dev)

    def out(self, x, dtype):
        return x.to(self.t.float32 if dtype == np.float32 else self.t.float64)


def _backend(device):
    return _Numpy() if device is None else _Torch(device)


# ---------------------------------------------------------------------------
# Constants, derived from the mathematics with exact rational arithmetic
# ---------------------------------------------------------------------------

# pi and ln 2 to 60 decimal places (more than the 3 x 53 bits used below)
_PI = Fraction("3.141592653589793238462643383279502884197169399375105820974944")
_LN2 = Fraction("0.693147180559945309417232121458176568075500134360255254120680")


def _split(x: Fraction, bits: int, parts: int) -> list[float]:
    """x as a sum of `parts` doubles, each but the last rounded to `bits`
    significant bits, so that n * part is exact for |n| < 2^(53 - bits)."""
    out = []
    rest = x
    for k in range(parts):
        if k == parts - 1:
            out.append(float(rest))
            break
        e = math.floor(math.log2(abs(float(rest))))
        q = Fraction(2) ** (e - bits + 1)
        head = Fraction(round(rest / q)) * q
        out.append(float(head))
        rest -= head
    return out


_PIO2 = _split(_PI / 2, 33, 3)   # pi/2 in three parts (Cody-Waite reduction)
_LN2P = _split(_LN2, 32, 2)      # ln 2 in two parts
_TWO_OVER_PI = float(2 / _PI)
_INV_LN2 = float(1 / _LN2)
_TWO_PI = float(2 * _PI)
_LN2F = float(_LN2)
_SQRT2 = float(Fraction(math.isqrt(2 * 10 ** 60), 10 ** 30))
_EXP_C = [float(Fraction(1, math.factorial(k))) for k in range(15)]             # e^r, |r| <= ln2/2
_SIN_C = [float(Fraction((-1) ** j, math.factorial(2 * j + 1))) for j in range(10)]  # |r| <= pi/4
_COS_C = [float(Fraction((-1) ** j, math.factorial(2 * j))) for j in range(11)]
_ATANH_C = [float(Fraction(1, 2 * j + 1)) for j in range(13)]                    # |s| <= 0.172


def _horner(B, z, coef):
    p = B.zeros(z.shape) + coef[-1]
    for c in reversed(coef[:-1]):
        p = p * z + c
    return p


def _pow2(B, n):
    """2^n for integer-valued float64 n in [-1022, 1023] (exponent bits)."""
    return B.from_bits((B.to_int(n) + 1023) << 52)


def det_exp(x, B=None):
    """e^x: x = n ln2 + r with |r| <= ln2/2 (ln2 in two parts), e^r from its
    Taylor series to degree 14 (remainder below 1e-18 relative), times 2^n.
    Arguments below -708 give 0."""
    B = B or _Numpy()
    xc = B.where(x < -708.0, -708.0, B.where(x > 709.0, 709.0, x))
    n = B.rint(xc * _INV_LN2)
    r = (xc - n * _LN2P[0]) - n * _LN2P[1]
    y = _horner(B, r, _EXP_C) * _pow2(B, n)
    return B.where(x < -708.0, 0.0, y)


def det_log(x, B=None):
    """ln x for positive normal x: x = m 2^e with m in [sqrt(2)/2, sqrt(2)),
    ln m = 2 atanh(s) with s = (m - 1)/(m + 1), |s| <= 0.172, from its series
    to s^25 (remainder below 1e-20)."""
    B = B or _Numpy()
    bits = B.bits(x)
    e = (bits >> 52) - 1023
    m = B.from_bits((bits & ((1 << 52) - 1)) | (1023 << 52))  # [1, 2)
    big = m > _SQRT2
    m = B.where(big, m * 0.5, m)
    ef = B.to_float(e) + B.where(big, 1.0, 0.0)
    s = (m - 1.0) / (m + 1.0)
    lm = (s * 2.0) * _horner(B, s * s, _ATANH_C)
    return ef * _LN2F + lm


def det_sincos(x, B=None):
    """(sin x, cos x) for |x| < 2^19: n = nearest integer to x / (pi/2),
    r = x - n pi/2 with pi/2 in three parts (|r| <= pi/4 + tiny), Taylor
    series of sin r to r^19 and of cos r to r^20, then the quadrant n mod 4."""
    B = B or _Numpy()
    n = B.rint(x * _TWO_OVER_PI)
    r = ((x - n * _PIO2[0]) - n * _PIO2[1]) - n * _PIO2[2]
    z = r * r
    s = r * _horner(B, z, _SIN_C)
    c = _horner(B, z, _COS_C)
    q = B.to_int(n) & 3
    sin = B.where(q == 0, s, B.where(q == 1, c, B.where(q == 2, -s, -c)))
    cos = B.where(q == 0, c, B.where(q == 1, -s, B.where(q == 2, -c, s)))
    return sin, cos


def tree_sum(x, B=None):
    """Sum of all elements in a fixed pairwise order (halving the flattened
    array, zero-padded to even length at every level)."""
    B = B or _Numpy()
    x = x.reshape(-1)
    while x.shape[0] > 1:
        if x.shape[0] % 2:
            x = B.cat([x, B.zeros((1,))])
        x = x[0::2] + x[1::2]
    return B.item(x[0])


def _uniform(rng, lo, hi, n):
    """lo + (hi - lo) u for u = rng.random(n), in two roundings."""
    return lo + (hi - lo) * rng.random(n)


def _normals(rng, n, B=None):
    """n standard normal deviates by the Box-Muller transform of uniform pairs
    (u1, u2): sqrt(-2 ln(1 - u1)) cos(2 pi u2) and the same with sin,
    interleaved; all uniforms are drawn first (u1 block, then u2 block)."""
    B = B or _Numpy()
    h = (n + 1) // 2
    u1 = B.asarray(rng.random(h))
    u2 = B.asarray(rng.random(h))
    rad = B.sqrt(det_log(1.0 - u1, B) * -2.0)
    s, c = det_sincos(u2 * _TWO_PI, B)
    z = B.stack([rad * c, rad * s], 1).reshape(-1)
    return z[:n]


def ifft_axis(re, im, axis, B=None):
    """Unnormalised inverse DFT, x_n = sum_k X_k e^(+2 pi i k n / P), along
    one axis of length P = 2^q: decimation in time (bit-reversed input order,
    then q stages of butterflies), complex arithmetic on separate real and
    imaginary arrays."""
    B = B or _Numpy()
    P = re.shape[axis]
    q = P.bit_length() - 1
    if P != 1 << q:
        raise ValueError("power-of-two length")
    rev = np.array([int(format(i, f"0{q}b")[::-1], 2) if q else 0 for i in range(P)], dtype=np.int64)
    re = B.contiguous(B.moveaxis(B.take(re, rev, axis), axis, -1))
    im = B.contiguous(B.moveaxis(B.take(im, rev, axis), axis, -1))
    lead = re.shape[:-1]
    h = 1
    while h < P:
        ws, wc = det_sincos((np.arange(h, dtype=np.float64) * _TWO_PI) / float(2 * h))
        ws, wc = B.asarray(ws), B.asarray(wc)
        r4 = re.reshape(lead + (P // (2 * h), 2, h))
        i4 = im.reshape(lead + (P // (2 * h), 2, h))
        ar, ai, br, bi = r4[..., 0, :], i4[..., 0, :], r4[..., 1, :], i4[..., 1, :]
        tr = wc * br - ws * bi
        ti = wc * bi + ws * br
        re = B.stack([ar + tr, ar - tr], -2).reshape(lead + (P,))
        im = B.stack([ai + ti, ai - ti], -2).reshape(lead + (P,))
        h *= 2
    return B.contiguous(B.moveaxis(re, -1, axis)), B.contiguous(B.moveaxis(im, -1, axis))


# ---------------------------------------------------------------------------
# Fields
# ---------------------------------------------------------------------------


def _gauss_sum_2d(B, xs, ys, cx, cy, sigma, amp):
    """sum_e amp_e exp(-((x - cx_e)^2 + (y - cy_e)^2) / (2 sigma_e^2)) at the
    grid coordinates xs (nx,) and ys (ny,), summed over e in order
    (separable: amp_e gy_e(y) gx_e(x); the factors are tabulated on the
    host)."""
    den = ((sigma * sigma) * 2.0)[:, None]
    dx = xs[None, :] - cx[:, None]
    dy = ys[None, :] - cy[:, None]
    gx = B.asarray(det_exp(-((dx * dx) / den)))                   # (E, nx)
    gy = B.asarray(det_exp(-((dy * dy) / den)) * amp[:, None])    # (E, ny)
    f = B.zeros((ys.shape[0], xs.shape[0]))
    for e in range(len(cx)):
        f = f + gy[e].reshape(-1, 1) * gx[e].reshape(1, -1)
    return f


def bumps2d(nx=128, ny=128, seed=0, nbumps=16, noise=1e-3, dtype=np.float32, device=None):
    """Sum of Gaussian bumps plus white noise: centres uniform on the grid,
    sigma uniform in [4, 16] px, amplitudes uniform in [-1, 1], noise N(0,
    noise^2). Draws: cx, cy, sigma, amp (nbumps each), then the noise."""
    B = _backend(device)
    rng = np.random.default_rng(seed)
    cx = _uniform(rng, 0.0, float(nx), nbumps)
    cy = _uniform(rng, 0.0, float(ny), nbumps)
    sigma = _uniform(rng, 4.0, 16.0, nbumps)
    amp = _uniform(rng, -1.0, 1.0, nbumps)
    f = _gauss_sum_2d(B, np.arange(nx, dtype=np.float64), np.arange(ny, dtype=np.float64), cx, cy, sigma, amp)
    f = f + _normals(rng, nx * ny, B).reshape(ny, nx) * noise
    return B.out(f, dtype)


def ocean2d(nx=3600, ny=2400, seed=2, neddies=400, dtype=np.float32, device=None, window=None):
    """Ocean-like field: Gaussian eddies (radius 10-60 px used as sigma,
    amplitude uniform in [-0.3, 0.3]) plus a meridional gradient y/(ny-1)
    plus N(0, 1e-6) noise. window = (y0, y1, x0, x1) returns that part of the
    full field (the same bits as cropping it)."""
    B = _backend(device)
    rng = np.random.default_rng(seed)
    cx = _uniform(rng, 0.0, float(nx), neddies)
    cy = _uniform(rng, 0.0, float(ny), neddies)
    radius = _uniform(rng, 10.0, 60.0, neddies)
    amp = _uniform(rng, -0.3, 0.3, neddies)
    y0, y1, x0, x1 = window if window is not None else (0, ny, 0, nx)
    ys = np.arange(y0, y1, dtype=np.float64)
    f = _gauss_sum_2d(B, np.arange(x0, x1, dtype=np.float64), ys, cx, cy, radius, amp)
    f = f + B.asarray(ys / float(max(ny - 1, 1))).reshape(-1, 1)
    z = _normals(rng, nx * ny, B).reshape(ny, nx)[y0:y1, x0:x1]
    f = f + z * 1e-3
    return B.out(f, dtype)


def lognormal3d(n=256, seed=1, dtype=np.float32, shape=None, device=None):
    """Cosmology-like density: a Gaussian random field with power spectrum
    P(k) ~ k^-3, standardised to zero mean and unit variance, exponentiated.
    The field is the real part of the inverse DFT of complex white noise
    (Box-Muller, real parts then imaginary parts) times |k|^-3/2 (k in integer
    grid units, k = 0 removed) on a periodic grid whose sides are the powers
    of two at or above shape's; the result is its leading corner of shape."""
    B = _backend(device)
    shape = tuple(shape) if shape is not None else (n, n, n)
    P = tuple(1 << max(0, (s - 1).bit_length()) for s in shape)
    rng = np.random.default_rng(seed)
    cnt = P[0] * P[1] * P[2]
    re = _normals(rng, cnt, B).reshape(P)
    im = _normals(rng, cnt, B).reshape(P)
    k2 = None
    for ax, p in enumerate(P):
        k = np.arange(p, dtype=np.float64)
        k = np.where(k < p - k, k, k - p)  # signed frequency, |k| <= p/2
        sh = [1, 1, 1]
        sh[ax] = p
        term = B.asarray(k * k).reshape(sh)
        k2 = term if k2 is None else k2 + term
    k2 = k2 + B.zeros(P)
    safe = B.where(k2 > 0.0, k2, 1.0)
    filt = B.where(k2 > 0.0, det_exp(det_log(safe, B) * -0.75, B), 0.0)
    re, im = re * filt, im * filt
    for ax in range(3):
        re, im = ifft_axis(re, im, ax, B)
    g = B.contiguous(re[: shape[0], : shape[1], : shape[2]])
    N = float(g.shape[0] * g.shape[1] * g.shape[2])
    mean = tree_sum(g, B) / N
    d = g - mean
    std = math.sqrt(tree_sum(d * d, B) / N)
    return B.out(det_exp(d / B.scalar(std), B), dtype)


def _turbulence_modes(seed, nmodes, kmax):
    """Mode directions uniform on the sphere (z = 2u - 1, azimuth 2 pi u'),
    |k| log-uniform in [1, kmax], phases uniform in [0, 2 pi); amplitude
    |k|^(-5/6). Draws: z, azimuth, log|k|, phase (nmodes each)."""
    rng = np.random.default_rng(seed)
    zc = _uniform(rng, -1.0, 1.0, nmodes)
    az = rng.random(nmodes) * _TWO_PI
    lk = rng.random(nmodes) * float(det_log(np.array([float(kmax)]))[0])
    phase = rng.random(nmodes) * _TWO_PI
    s_az, c_az = det_sincos(az)
    rxy = np.sqrt(1.0 - zc * zc)
    kmag = det_exp(lk)
    k = np.stack([(rxy * c_az) * kmag, (rxy * s_az) * kmag, zc * kmag], 1)  # cycles per box, (kx, ky, kz)
    amp = det_exp(det_log(kmag) * (-5.0 / 6.0))
    return k, amp, phase


def turbulence3d(n=512, seed=3, nmodes=256, kmax=64.0, dtype=np.float32, device=None, shape=None):
    """Turbulence-like field: random-phase sinusoidal modes,
    f = sum_m A_m sin(2 pi k_m . x / L + phi_m) with L the largest side,
    directions uniform on the sphere, |k| log-uniform in [1, kmax] cycles per
    box, A = |k|^(-5/6) (a Kolmogorov -5/3 energy spectrum).

    Evaluated separably, mode by mode in order: sin(a + b + c + phi) is the
    imaginary part of the product c_m e^(ia) e^(ib) e^(ic), c_m = A_m
    e^(i phi_m), with the per-axis factors tabulated. With ``device`` (a torch
    device) the arithmetic runs there and a torch tensor is returned; the
    bits are the same either way."""
    shape = tuple(shape) if shape is not None else (n, n, n)
    L = float(max(shape))
    nz, ny, nx = shape
    B = _backend(device)
    k, amp, phase = _turbulence_modes(seed, nmodes, kmax)
    sp, cp = det_sincos(phase)
    cr, ci = amp * cp, amp * sp  # c_m

    def table(npts, kk):  # e^(2 pi i k x / L) for x < npts, per mode: (npts, M)
        w = (kk * _TWO_PI) / L
        s, c = det_sincos(np.arange(npts, dtype=np.float64)[:, None] * w[None, :])
        return c, s

    exr, exi = table(nx, k[:, 0])
    eyr, eyi = table(ny, k[:, 1])
    ezr, ezi = table(nz, k[:, 2])
    # c_m e^(ic): (nz, M)
    czr = cr[None, :] * ezr - ci[None, :] * ezi
    czi = cr[None, :] * ezi + ci[None, :] * ezr
    exr_b, exi_b = B.asarray(exr), B.asarray(exi)
    eyr_b, eyi_b = B.asarray(eyr), B.asarray(eyi)
    czr_b, czi_b = B.asarray(czr), B.asarray(czi)
    out = None
    # slabs of planes keep the working set small; every element still sees
    # the modes in order
    slab = max(1, min(nz, (1 << 21) // max(1, nx * ny))) if device is None else nz
    parts = []
    for z0 in range(0, nz, slab):
        z1 = min(nz, z0 + slab)
        acc = B.zeros((z1 - z0, ny, nx))
        for m in range(nmodes):
            # (c_m e^(ic)) e^(ib): (nz, ny)
            tr = czr_b[z0:z1, m].reshape(-1, 1) * eyr_b[:, m].reshape(1, -1) - \
                czi_b[z0:z1, m].reshape(-1, 1) * eyi_b[:, m].reshape(1, -1)
            ti = czr_b[z0:z1, m].reshape(-1, 1) * eyi_b[:, m].reshape(1, -1) + \
                czi_b[z0:z1, m].reshape(-1, 1) * eyr_b[:, m].reshape(1, -1)
            # imaginary part of that times e^(ia)
            acc = acc + (tr.reshape(z1 - z0, ny, 1) * exi_b[:, m].reshape(1, 1, nx) +
                         ti.reshape(z1 - z0, ny, 1) * exr_b[:, m].reshape(1, 1, nx))
        parts.append(B.out(acc, dtype))
    out = parts[0] if len(parts) == 1 else B.cat(parts, 0)
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
    """Device version of ``quantise`` for large float32 torch fields (the same
    definition and the same bits: the bound test runs in float64, exact for
    float32 inputs)."""
    import torch

    if f.dtype != torch.float32:
        raise TypeError("quantise_torch handles float32 fields")
    xi = float(np.float32(xi))
    if xi == 0.0:
        return f.clone()
    step = 2.0 * xi
    # divisor on the device: a host scalar would be applied as a reciprocal
    q = (torch.round(f.double() / torch.tensor(step, dtype=torch.float64, device=f.device)) * step).to(f.dtype)
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

    bumps128     : 2D 128x128 f32 bumps, seed 0
    lognormal256 : 3D 256^3 f32 lognormal, seed 1
    ocean        : 2D 3600x2400 f32, seed 2
    turb512      : 3D 512^3 f32 turbulence, seed 3
    xi = rel * range (default rel 1e-3). With device the field is a torch
    tensor there (same bits as the host form).
    """
    rel = 1e-3 if rel is None else rel
    if name == "bumps128":
        f = bumps2d(128, 128, 0, device=device)
    elif name == "lognormal256":
        f = lognormal3d(256, 1, device=device)
    elif name == "ocean":
        f = ocean2d(3600, 2400, 2, device=device)
    elif name == "turb512":
        f = turbulence3d(512, 3, device=device)
    else:
        raise KeyError(name)
    xi = xi_for(f, rel)
    if device is not None:
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
        rel = 10.0 ** float(_uniform(rng, -5.0, -3.0, 1)[0])
        xi = xi_for(f, rel)
        yield f, quantise(f, xi), xi
