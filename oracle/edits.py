"""Lossless coding of an edit list (Sec. 5.3), plain Python: test
infrastructure only, like the rest of this package (it shares nothing with
the CUDA library).

The paper sorts the edited indices, takes their differences, and codes them
with run-length and Huffman coding before a general-purpose compressor; the
values are coded separately. This restatement fixes the unstated details:

* Index deltas: d_k = idx_k - idx_{k-1} with idx_{-1} = -1 (so d_k >= 1).
  Tokens, in edit order, within aligned groups of 32 edits (k // 32):
  a maximal run of L >= 2 deltas equal to 1 inside a group is one RUN token
  (symbol 252, 5 raw bits L - 2); any other delta d is a literal: symbol
  d - 1 for d <= 252; symbol 253 with 16 raw bits d - 253 for
  d <= 253 + 65535; symbol 254 with 32 raw bits d otherwise.
* Values: the bytes (little-endian) of bits(new value) XOR bits(fhat at the
  index), one symbol per byte.
* Each of the two symbol streams gets its own canonical Huffman code with at
  most 15 bits per code (package-merge); a symbol's code is followed by its
  raw bits. Bits are packed most significant first into 32-bit words. Every
  4096th symbol of a stream starts a chunk whose bit offset is stored.
* Layout (little-endian): 14 header words (magic 'MSZE', version 1, dtype,
  bytes per value, n_edits as u64, index tokens, index chunks, value
  chunks, 0, index bits as u64, value bits as u64); 256 index code lengths
  and 256 value code lengths (bytes); per index chunk (bit offset u64, first
  edit u32, index before it u32, 0xffffffff for none); per value chunk (bit
  offset u64); the index payload, then the value payload, in words.

Pins (tests/test_oracle_edits.py): tokenisations worked by hand (runs,
group boundaries, both escapes); package-merge lengths complete (Kraft
equality) and at the Huffman cost when the limit does not bind, within 15
bits when it does; canonical codes by hand and prefix-free; exact round
trips; payload bits equal to the code lengths plus raw bits.
"""
from __future__ import annotations

import heapq
import struct

import numpy as np

MAGIC = 0x45535A4D
VERSION = 1
MAX_LEN = 15
CHUNK = 4096
GROUP = 32
RUN, ESC16, ESC32 = 252, 253, 254


def index_tokens(idx) -> list[tuple[int, int, int]]:
    """(symbol, raw value, raw bits) per token of an ascending index list."""
    idx = [int(v) for v in idx]
    d = [v - (idx[k - 1] if k else -1) for k, v in enumerate(idx)]
    out = []
    k = 0
    while k < len(d):
        if d[k] == 1:
            end = min(len(d), (k // GROUP + 1) * GROUP)
            j = k
            while j < end and d[j] == 1:
                j += 1
            L = j - k
            out.append((RUN, L - 2, 5) if L >= 2 else (0, 0, 0))
            k = j
            continue
        v = d[k]
        if v <= 252:
            out.append((v - 1, 0, 0))
        elif v <= 253 + 65535:
            out.append((ESC16, v - 253, 16))
        else:
            out.append((ESC32, v, 32))
        k += 1
    return out


def value_symbols(val: np.ndarray, fhat: np.ndarray, idx) -> list[int]:
    """Bytes of bits(val) XOR bits(fhat[idx]), little-endian per value."""
    val = np.ascontiguousarray(val)
    ref = np.ascontiguousarray(fhat).ravel()[np.asarray(idx, dtype=np.int64)]
    u = np.uint32 if val.dtype == np.float32 else np.uint64
    x = val.view(u) ^ ref.astype(val.dtype).view(u)
    return list(x.astype(x.dtype.newbyteorder("<")).tobytes())


def package_merge(freq: list[int], max_len: int = MAX_LEN) -> list[int]:
    """Code lengths of a length-limited optimal prefix code (Larmore and
    Hirschberg's package-merge): 0 for unused symbols; a lone symbol gets 1."""
    used = [s for s, f in enumerate(freq) if f > 0]
    lens = [0] * len(freq)
    if not used:
        return lens
    if len(used) == 1:
        lens[used[0]] = 1
        return lens
    assert len(used) <= (1 << max_len)
    leaves = sorted((freq[s], s) for s in used)
    # items: (weight, tuple of symbols, each counted once per occurrence)
    level = [(w, (s,)) for w, s in leaves]
    for _ in range(max_len - 1):
        packages = [(level[i][0] + level[i + 1][0], level[i][1] + level[i + 1][1])
                    for i in range(0, len(level) - 1, 2)]
        level = sorted([(w, (s,)) for w, s in leaves] + packages, key=lambda t: t[0])
    for w, syms in level[: 2 * len(used) - 2]:
        for s in syms:
            lens[s] += 1
    return lens


def canonical_codes(lens: list[int]) -> list[int]:
    """Canonical codes: symbols ordered by (length, symbol), consecutive
    values, shifted left when the length grows."""
    codes = [0] * len(lens)
    code, prev = 0, 0
    for l, s in sorted((l, s) for s, l in enumerate(lens) if l > 0):
        code <<= l - prev
        codes[s] = code
        code += 1
        prev = l
    return codes


class _Bits:
    def __init__(self):
        self.words: list[int] = []
        self.n = 0

    def put(self, value: int, nbits: int):
        for b in range(nbits - 1, -1, -1):
            if self.n % 32 == 0:
                self.words.append(0)
            if (value >> b) & 1:
                self.words[-1] |= 1 << (31 - self.n % 32)
            self.n += 1


def _encode_stream(syms, raws, rbits, lens, codes):
    bits, offs = _Bits(), []
    for t, s in enumerate(syms):
        if t % CHUNK == 0:
            offs.append(bits.n)
        bits.put(codes[s], lens[s])
        if rbits[t]:
            bits.put(raws[t], rbits[t])
    return bits, offs


def encode(idx, val: np.ndarray, fhat: np.ndarray) -> bytes:
    idx = [int(v) for v in idx]
    val = np.ascontiguousarray(val)
    es = val.dtype.itemsize
    dtype = 0 if val.dtype == np.float32 else 1
    n = len(idx)
    toks = index_tokens(idx)
    si = [t[0] for t in toks]
    freq_i = [0] * 256
    for s in si:
        freq_i[s] += 1
    sv = value_symbols(val, fhat, idx) if n else []
    freq_v = [0] * 256
    for s in sv:
        freq_v[s] += 1
    len_i, len_v = package_merge(freq_i), package_merge(freq_v)
    bi, offs_i = _encode_stream(si, [t[1] for t in toks], [t[2] for t in toks], len_i, canonical_codes(len_i))
    bv, offs_v = _encode_stream(sv, [0] * len(sv), [0] * len(sv), len_v, canonical_codes(len_v))
    # edit position and previous index at each index chunk's first token
    first, k = [], 0
    for t, (s, r, rb) in enumerate(toks):
        if t % CHUNK == 0:
            first.append(k)
        k += (r + 2) if s == RUN else 1
    out = struct.pack("<4I Q 4I Q Q", MAGIC, VERSION, dtype, es, n, len(toks), len(offs_i), len(offs_v), 0,
                      bi.n, bv.n)
    out += bytes(len_i) + bytes(len_v)
    for o, k0 in zip(offs_i, first):
        out += struct.pack("<QII", o, k0, idx[k0 - 1] if k0 else 0xFFFFFFFF)
    for o in offs_v:
        out += struct.pack("<Q", o)
    out += struct.pack(f"<{len(bi.words)}I", *bi.words)
    out += struct.pack(f"<{len(bv.words)}I", *bv.words)
    return out


def _decoder(lens):
    codes = canonical_codes(lens)
    return {(lens[s], codes[s]): s for s in range(len(lens)) if lens[s] > 0}


def decode(data: bytes, fhat: np.ndarray):
    """(idx int64 array, val array) of an encoded edit list."""
    h = struct.unpack_from("<4I Q 4I Q Q", data, 0)
    magic, version, dtype, es, n, ntok, nci, ncv, _, bits_i, bits_v = h
    assert magic == MAGIC and version == VERSION
    pos = struct.calcsize("<4I Q 4I Q Q")
    len_i, len_v = list(data[pos:pos + 256]), list(data[pos + 256:pos + 512])
    pos += 512 + 16 * nci + 8 * ncv
    wi = (bits_i + 31) // 32
    words_i = struct.unpack_from(f"<{wi}I", data, pos)
    words_v = struct.unpack_from(f"<{(bits_v + 31) // 32}I", data, pos + 4 * wi)

    def bit(words, j):
        return (words[j // 32] >> (31 - j % 32)) & 1

    def read_stream(words, lens, count, raw_of):
        table, j, out = _decoder(lens), 0, []
        for _ in range(count):
            c, l = 0, 0
            while (l, c) not in table:
                c = (c << 1) | bit(words, j)
                l += 1
                j += 1
                assert l <= MAX_LEN
            s = table[(l, c)]
            rb = raw_of(s)
            r = 0
            for _ in range(rb):
                r = (r << 1) | bit(words, j)
                j += 1
            out.append((s, r))
        return out

    raw_bits = {RUN: 5, ESC16: 16, ESC32: 32}
    idx, prev = [], -1
    for s, r in read_stream(words_i, len_i, ntok, lambda s: raw_bits.get(s, 0)):
        if s == RUN:
            for _ in range(r + 2):
                prev += 1
                idx.append(prev)
            continue
        prev += (r + 253) if s == ESC16 else r if s == ESC32 else s + 1
        idx.append(prev)
    assert len(idx) == n
    dt = np.float32 if dtype == 0 else np.float64
    u = np.uint32 if dtype == 0 else np.uint64
    vb = bytes(s for s, _ in read_stream(words_v, len_v, n * es, lambda s: 0))
    x = np.frombuffer(vb, dtype=np.dtype(u).newbyteorder("<")).astype(u)
    ref = np.ascontiguousarray(fhat).ravel()[np.asarray(idx, dtype=np.int64)].astype(dt).view(u)
    return np.asarray(idx, dtype=np.int64), (x ^ ref).view(dt)
