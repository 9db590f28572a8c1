"""Pins of the oracle's edit-list coding (Sec. 5.3: sorted indices, their
differences, run-length and Huffman coding; values coded separately)."""
import heapq
import itertools

import numpy as np
import pytest

from oracle import edits


def test_index_tokens_hand_example():
    # deltas: 1 (idx 0), 1, 1, 1, 7 (idx 10), 1, 289 (idx 300), 70000
    idx = [0, 1, 2, 3, 10, 11, 300, 70300]
    assert edits.index_tokens(idx) == [
        (edits.RUN, 2, 5),           # a run of four deltas equal to 1
        (6, 0, 0),                   # delta 7
        (0, 0, 0),                   # a lone delta 1
        (edits.ESC16, 289 - 253, 16),
        (edits.ESC32, 70000, 32),
    ]


def test_runs_stop_at_the_group_boundary():
    idx = list(range(40))  # 40 deltas equal to 1: groups of 32 and 8
    assert edits.index_tokens(idx) == [(edits.RUN, 30, 5), (edits.RUN, 6, 5)]
    idx = list(range(33))  # 32 + a lone one
    assert edits.index_tokens(idx) == [(edits.RUN, 30, 5), (0, 0, 0)]


def _huffman_cost(freq):
    h = [f for f in freq if f > 0]
    if len(h) < 2:
        return sum(h)
    heapq.heapify(h)
    cost = 0
    while len(h) > 1:
        a, b = heapq.heappop(h), heapq.heappop(h)
        cost += a + b
        heapq.heappush(h, a + b)
    return cost


@pytest.mark.parametrize("seed", range(6))
def test_package_merge_is_an_optimal_prefix_code(seed):
    rng = np.random.default_rng(seed)
    freq = [int(x) for x in rng.integers(0, 50, size=40)]
    lens = edits.package_merge(freq)
    used = [l for f, l in zip(freq, lens) if f > 0]
    assert all(1 <= l <= edits.MAX_LEN for l in used)
    assert sum(2.0 ** -l for l in used) == 1.0  # complete (Kraft equality)
    # with no length limit binding it reaches the Huffman cost
    assert sum(f * l for f, l in zip(freq, lens)) == _huffman_cost(freq)


def test_package_merge_respects_the_length_limit():
    fib = [1, 1]
    while len(fib) < 24:
        fib.append(fib[-1] + fib[-2])  # unlimited Huffman would need 23 bits
    lens = edits.package_merge(fib)
    assert max(lens) == edits.MAX_LEN
    assert sum(2.0 ** -l for l in lens) <= 1.0
    assert sum(f * l for f, l in zip(fib, lens)) >= _huffman_cost(fib)


def test_canonical_codes_hand_example():
    lens = [2, 1, 3, 3]
    assert edits.canonical_codes(lens) == [0b10, 0b0, 0b110, 0b111]


def test_canonical_codes_are_prefix_free():
    lens = edits.package_merge([5, 9, 12, 13, 16, 45, 0, 3])
    codes = edits.canonical_codes(lens)
    words = [format(c, f"0{l}b") for c, l in zip(codes, lens) if l]
    for a, b in itertools.permutations(words, 2):
        assert not b.startswith(a)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_round_trip_with_runs_and_escapes(dtype):
    rng = np.random.default_rng(7)
    n = 30000
    fhat = rng.standard_normal(n * 3).astype(dtype)
    # runs of consecutive vertices, small gaps, gaps needing 16 and 32 raw bits
    steps = rng.choice([1, 1, 1, 2, 5, 40, 300, 70000], size=5000)
    idx = np.cumsum(steps)
    idx = idx[idx < fhat.size]
    val = (fhat[idx] * np.asarray(0.999, dtype=dtype)).astype(dtype)
    data = edits.encode(idx, val, fhat)
    i2, v2 = edits.decode(data, fhat)
    assert np.array_equal(i2, idx)
    assert np.array_equal(v2.view(np.uint8), val.view(np.uint8))


def test_payload_size_is_the_code_lengths_plus_raw_bits():
    rng = np.random.default_rng(8)
    fhat = rng.standard_normal(5000).astype(np.float32)
    idx = np.unique(rng.integers(0, 5000, size=900))
    val = fhat[idx] + np.float32(1e-3)
    data = edits.encode(idx, val, fhat)
    import struct

    h = struct.unpack_from("<4I Q 4I Q Q", data, 0)
    bits_i, bits_v = h[-2], h[-1]
    toks = edits.index_tokens(idx)
    freq = [0] * 256
    for s, _, _ in toks:
        freq[s] += 1
    lens = edits.package_merge(freq)
    assert bits_i == sum(lens[s] + rb for s, _, rb in toks)
    sv = edits.value_symbols(val, fhat, idx)
    fv = [0] * 256
    for s in sv:
        fv[s] += 1
    lv = edits.package_merge(fv)
    assert bits_v == sum(lv[s] for s in sv)


def test_empty_list():
    fhat = np.zeros(10, dtype=np.float32)
    data = edits.encode([], np.zeros(0, dtype=np.float32), fhat)
    i2, v2 = edits.decode(data, fhat)
    assert i2.size == 0 and v2.size == 0
