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
