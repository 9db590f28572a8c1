"""The input generator's uniform quantiser (the stand-in for the lossy
compressor): its result stays within the bound exactly, equals the rounded
lattice point 2 xi * rint(x / 2 xi) wherever that already fits, and the
torch version used for large fields agrees with the numpy one bit for bit."""
import numpy as np
import pytest

from paper_2406_09423_gb300 import synth
from tests.invariants import bits_of, within_bound


def _field(dtype, seed, shape=(37, 53)):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) * 10.0 ** rng.integers(-2, 3)).astype(dtype)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("rel", [1e-1, 1e-3, 1e-5, 1e-7])
def test_quantise_within_bound_and_on_the_lattice(dtype, rel):
    f = _field(dtype, 3)
    xi = synth.xi_for(f, rel)
    q = synth.quantise(f, xi)
    assert q.dtype == f.dtype and q.shape == f.shape
    assert within_bound(f, q, xi)
    X = float(f.dtype.type(xi))
    lattice = (np.rint(f.astype(np.float64) / (2 * X)) * (2 * X)).astype(f.dtype)
    fits = np.abs(lattice.astype(np.longdouble) - f.astype(np.longdouble)) <= np.longdouble(X)
    assert fits.mean() > 0.9
    assert np.array_equal(bits_of(q[fits]), bits_of(lattice[fits]))
    # a nudged value moved towards x from the lattice point, which did not fit
    moved = ~fits
    if moved.any():
        assert (np.abs(q[moved].astype(np.float64) - f[moved]) <= np.abs(lattice[moved].astype(np.float64) - f[moved])).all()


def test_quantise_zero_bound_is_a_copy():
    f = _field(np.float32, 4)
    q = synth.quantise(f, 0.0)
    assert np.array_equal(bits_of(q), bits_of(f)) and q is not f


@pytest.mark.parametrize("rel", [1e-2, 1e-4, 1e-6])
def test_quantise_torch_matches_numpy(rel):
    torch = pytest.importorskip("torch")
    f = _field(np.float32, 5, shape=(64, 65))
    xi = synth.xi_for(f, rel)
    qt = synth.quantise_torch(torch.from_numpy(f), xi).numpy()
    assert np.array_equal(bits_of(qt), bits_of(synth.quantise(f, xi)))


# ---------------------------------------------------------------------------
# Bit-reproducible generation: the restated elementary functions, the FFT and
# the fixed summation tree, and every generator giving the same bits through
# numpy and through torch.
# ---------------------------------------------------------------------------


def test_restated_elementary_functions_are_accurate():
    x = np.linspace(-700.0, 700.0, 100_001)
    assert np.max(np.abs(synth.det_exp(x) - np.exp(x)) / np.exp(x)) < 1e-15
    assert synth.det_exp(np.array([-800.0, 0.0]))[0] == 0.0 and synth.det_exp(np.array([0.0]))[0] == 1.0
    u = np.concatenate([np.geomspace(1e-300, 1e300, 50_001), np.linspace(1e-3, 10.0, 50_001)])
    assert np.max(np.abs(synth.det_log(u) - np.log(u)) / np.maximum(1.0, np.abs(np.log(u)))) < 1e-15
    assert synth.det_log(np.array([1.0]))[0] == 0.0
    t = np.linspace(-5000.0, 5000.0, 200_001)
    s, c = synth.det_sincos(t)
    assert np.max(np.abs(s - np.sin(t))) < 1e-15 and np.max(np.abs(c - np.cos(t))) < 1e-15
    assert np.max(np.abs(s * s + c * c - 1.0)) < 1e-15


def test_restated_fft_is_the_inverse_dft():
    rng = np.random.default_rng(0)
    re, im = rng.standard_normal((8, 16, 4)), rng.standard_normal((8, 16, 4))
    a, b = re, im
    for ax in range(3):
        a, b = synth.ifft_axis(a, b, ax)
    ref = np.fft.ifftn(re + 1j * im) * re.size
    assert np.max(np.abs(a + 1j * b - ref)) < 1e-12
    # a single mode comes out as the sampled exponential
    P = 32
    re1, im1 = np.zeros(P), np.zeros(P)
    re1[3] = 1.0
    a, b = synth.ifft_axis(re1, im1, 0)
    n = np.arange(P)
    assert np.max(np.abs(a - np.cos(2 * np.pi * 3 * n / P))) < 1e-14
    assert np.max(np.abs(b - np.sin(2 * np.pi * 3 * n / P))) < 1e-14


def test_tree_sum_is_exact_on_integers_and_fixed():
    x = np.arange(1, 1_000_002, dtype=np.float64)
    assert synth.tree_sum(x) == float(1_000_001 * 1_000_002 // 2)
    y = np.random.default_rng(1).standard_normal(12345)
    assert synth.tree_sum(y) == synth.tree_sum(y.copy())
    assert abs(synth.tree_sum(y) - np.sum(y)) < 1e-10


def test_box_muller_deviates_are_standard_normal():
    z = synth._normals(np.random.default_rng(7), 200_001)
    assert z.shape == (200_001,)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    assert abs(np.mean(np.abs(z) < 1.0) - 0.6827) < 0.005


GENERATORS = [
    ("bumps", lambda d: synth.bumps2d(64, 48, 1, device=d)),
    ("bumps-f64", lambda d: synth.bumps2d(33, 20, 5, dtype=np.float64, device=d)),
    ("ocean-window", lambda d: synth.ocean2d(3600, 2400, 2, window=(100, 140, 3000, 3064), device=d)),
    ("lognormal-ragged", lambda d: synth.lognormal3d(seed=1, shape=(20, 24, 33), device=d)),
    ("turbulence-f64", lambda d: synth.turbulence3d(32, 8, kmax=4.0, dtype=np.float64, shape=(16, 32, 32), device=d)),
    ("turbulence", lambda d: synth.turbulence3d(24, 3, kmax=6.0, device=d)),
]


@pytest.mark.parametrize("name,make", GENERATORS, ids=[g[0] for g in GENERATORS])
def test_generators_same_bits_in_numpy_and_torch(name, make):
    torch = pytest.importorskip("torch")
    a = make(None)
    b = make("cpu")
    assert isinstance(b, torch.Tensor) and b.dtype == (torch.float32 if a.dtype == np.float32 else torch.float64)
    assert np.array_equal(bits_of(a), bits_of(b.numpy()))


def test_ocean_window_is_the_crop_of_the_field():
    full = synth.ocean2d(400, 300, 9, neddies=40)
    part = synth.ocean2d(400, 300, 9, neddies=40, window=(50, 120, 200, 333))
    assert np.array_equal(bits_of(part), bits_of(full[50:120, 200:333]))


def test_fields_have_their_stated_statistics():
    ln = synth.lognormal3d(seed=1, shape=(32, 32, 32)).astype(np.float64)
    g = np.log(ln)
    assert abs(g.mean()) < 1e-5 and abs(g.std() - 1.0) < 1e-5  # exp of a standardised field
    t = synth.turbulence3d(32, 3, kmax=4.0).astype(np.float64)
    k, amp, _ = synth._turbulence_modes(3, 256, 4.0)
    kmag = np.linalg.norm(k, axis=1)
    assert np.all(kmag >= 1.0 - 1e-12) and np.all(kmag <= 4.0 + 1e-12)
    assert np.allclose(amp, kmag ** (-5.0 / 6.0), rtol=1e-14)
    assert abs(np.mean(t * t) - 0.5 * np.sum(amp * amp)) < 0.5 * np.sum(amp * amp)
    oc = synth.ocean2d(360, 240, 2, neddies=40).astype(np.float64)
    assert -1.0 < oc.min() and oc.max() < 2.0 and oc[-1].mean() > oc[0].mean()
