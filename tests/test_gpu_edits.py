"""Edit-list coding on the device (msz_encode_edits / msz_decode_edits,
Sec. 5.3) against the oracle's restatement: identical bytes, exact round
trips."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import edits as oedits
from paper_2406_09423_gb300 import synth

pytestmark = pytest.mark.gpu


def _msz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2406_09423_gb300 as msz

    return msz


def _random_list(rng, n_field, n_steps, dtype):
    steps = rng.choice([1, 1, 1, 1, 2, 3, 17, 251, 252, 253, 300, 65788, 65789, 70000], size=n_steps)
    idx = np.cumsum(steps) - 1
    idx = idx[idx < n_field]
    fhat = rng.standard_normal(n_field).astype(dtype)
    val = (fhat[idx] * np.asarray(0.75, dtype=dtype) + np.asarray(1e-3, dtype=dtype)).astype(dtype)
    return idx, val, fhat


@pytest.mark.parametrize("dtype,seed,n_steps", [(np.float32, 0, 20000), (np.float64, 1, 9000),
                                                (np.float32, 2, 5), (np.float32, 3, 70000)])
def test_encode_matches_oracle_and_round_trips(dtype, seed, n_steps):
    msz = _msz()
    rng = np.random.default_rng(seed)
    shape = (300, 1000)
    idx, val, fhat = _random_list(rng, shape[0] * shape[1], n_steps, dtype)
    fh = torch.from_numpy(fhat.reshape(shape)).cuda()
    data = msz.encode_edits(torch.from_numpy(idx).cuda(), torch.from_numpy(val).cuda(), fh)
    ref = oedits.encode(idx, val, fhat)
    assert bytes(data.cpu().numpy()) == ref
    for src in (data, torch.frombuffer(bytearray(ref), dtype=torch.uint8)):
        i2, v2 = msz.decode_edits(src, fh)
        assert np.array_equal(i2.cpu().numpy(), idx)
        assert np.array_equal(v2.cpu().numpy().view(np.uint8), val.view(np.uint8))


@pytest.mark.parametrize("rel", [1e-2, 1e-3])
def test_edit_list_of_a_fix(rel):
    msz = _msz()
    f = synth.turbulence3d(48, 5, kmax=6.0, shape=(40, 44, 48))
    xi = synth.xi_for(f, rel)
    fhat = synth.quantise(f, xi)
    tf, th = torch.from_numpy(f).cuda(), torch.from_numpy(fhat).cuda()
    res = msz.fix(tf, th, xi)
    data = msz.encode_edits(res.edit_idx, res.edit_val, th)
    ref = oedits.encode(res.edit_idx.cpu().numpy(), res.edit_val.cpu().numpy(), fhat)
    assert bytes(data.cpu().numpy()) == ref
    i2, v2 = msz.decode_edits(data, th)
    g = th.clone()
    msz.apply(g, i2, v2)
    g_ref = th.clone()
    msz.apply(g_ref, res.edit_idx, res.edit_val)
    assert torch.equal(g.view(torch.int32), g_ref.view(torch.int32))
    # smaller than the raw list (4-byte index + 4-byte value per edit)
    assert data.numel() < 8 * res.edit_idx.numel()


def test_empty_and_invalid_lists():
    msz = _msz()
    from paper_2406_09423_gb300 import native

    fh = torch.zeros((8, 9), dtype=torch.float32, device="cuda")
    empty = msz.encode_edits(torch.zeros(0, dtype=torch.int32), torch.zeros(0), fh)
    assert bytes(empty.cpu().numpy()) == oedits.encode([], np.zeros(0, np.float32), fh.cpu().numpy())
    i2, v2 = msz.decode_edits(empty, fh)
    assert i2.numel() == 0 and v2.numel() == 0
    # indices not ascending, or outside the field: rejected before any output
    with pytest.raises(RuntimeError):
        msz.encode_edits(torch.tensor([3, 2], dtype=torch.int32), torch.zeros(2), fh)
    with pytest.raises(RuntimeError):
        msz.encode_edits(torch.tensor([3, 72], dtype=torch.int32), torch.zeros(2), fh)
    data = msz.encode_edits(torch.tensor([1, 2, 3, 40], dtype=torch.int32), torch.ones(4), fh)
    # a truncated stream, another type, too small a capacity: rejected from the header
    with pytest.raises(RuntimeError):
        msz.decode_edits(data[:-4], fh)
    with pytest.raises(RuntimeError):
        msz.decode_edits(data, fh.double())
    with pytest.raises(RuntimeError):
        msz.decode_edits(data, fh, cap_edits=3)
    st, _ = native.msz_decode_edits(data.data_ptr(), 10, fh.data_ptr(), tuple(fh.shape), fh.dtype, 0, 0, 4)
    assert st == -1
