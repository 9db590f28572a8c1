// Lossless coding of an edit list (Sec. 5.3): the sorted indices as
// differences with run-length tokens, and the values as the bytes of
// bits(new value) XOR bits(fhat), each stream with its own length-limited
// canonical Huffman code. The format is documented with msz_encode_edits in
// msz.h. Encoding and decoding run on the device; the host builds the codes
// (256 symbols) between the histogram and the packing.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "msz.h"
#include "msz_device.cuh"

namespace msz {
namespace {

constexpr uint32_t kMagic = 0x45535A4Du;  // 'MSZE'
constexpr uint32_t kVersion = 1;
constexpr int kMaxLen = 15;     // longest code
constexpr int kChunk = 4096;    // symbols per decoding chunk
constexpr int kGroup = 32;      // edits per run-length group (one warp)
constexpr int kRun = 252, kEsc16 = 253, kEsc32 = 254;
constexpr int kET = 256;        // threads per block
constexpr int kSeg = 4096;      // scan segment per block

struct Header {  // 56 bytes, little-endian (the device is)
  uint32_t magic, version, dtype, es;
  uint64_t n;
  uint32_t ntok, nci, ncv, zero;
  uint64_t bits_i, bits_v;
};
static_assert(sizeof(Header) == 56, "header layout");
constexpr size_t kTables = sizeof(Header) + 512;  // + code lengths of both streams

// ---- host: length-limited optimal code (package-merge), canonical codes ----

// Code lengths <= max_len of an optimal prefix code for freq (Larmore and
// Hirschberg's package-merge): leaves sorted by (weight, symbol); each level
// pairs the previous level's items into packages and merges them with the
// leaves, a leaf first among equal weights; a symbol's length is its count in
// the first 2n - 2 items of the last level. A lone symbol gets length 1.
void package_merge(const uint32_t* freq, int nsym, int max_len, uint8_t* len) {
  std::memset(len, 0, (size_t)nsym);
  struct Item {
    uint64_t w;
    std::vector<uint16_t> syms;
  };
  std::vector<Item> leaves;
  for (int s = 0; s < nsym; ++s)
    if (freq[s]) leaves.push_back({freq[s], {(uint16_t)s}});
  std::stable_sort(leaves.begin(), leaves.end(), [](const Item& a, const Item& b) { return a.w < b.w; });
  const size_t n = leaves.size();
  if (n == 0) return;
  if (n == 1) {
    len[leaves[0].syms[0]] = 1;
    return;
  }
  std::vector<Item> level = leaves;
  for (int it = 0; it < max_len - 1; ++it) {
    std::vector<Item> packages;
    for (size_t i = 0; i + 1 < level.size(); i += 2) {
      Item p{level[i].w + level[i + 1].w, level[i].syms};
      p.syms.insert(p.syms.end(), level[i + 1].syms.begin(), level[i + 1].syms.end());
      packages.push_back(std::move(p));
    }
    std::vector<Item> next;
    size_t a = 0, b = 0;
    while (a < leaves.size() || b < packages.size()) {
      if (b == packages.size() || (a < leaves.size() && leaves[a].w <= packages[b].w)) next.push_back(leaves[a++]);
      else next.push_back(std::move(packages[b++]));
    }
    level.swap(next);
  }
  for (size_t i = 0; i < 2 * n - 2 && i < level.size(); ++i)
    for (uint16_t s : level[i].syms) ++len[s];
}

// Canonical codes: symbols by (length, symbol), consecutive values, shifted
// left when the length grows.
void canonical(const uint8_t* len, int nsym, uint32_t* code) {
  std::vector<std::pair<int, int>> order;
  for (int s = 0; s < nsym; ++s)
    if (len[s]) order.push_back({len[s], s});
  std::sort(order.begin(), order.end());
  uint32_t c = 0;
  int prev = 0;
  for (auto& p : order) {
    c <<= (p.first - prev);
    code[p.second] = c++;
    prev = p.first;
  }
}

// 2^15-entry decoding table: the symbol and code length of every 15-bit
// window that starts with a code (0 for windows that start with none).
bool decode_table(const uint8_t* len, uint32_t* table) {
  uint32_t code[256] = {};
  double kraft = 0;
  for (int s = 0; s < 256; ++s) {
    if (len[s] > kMaxLen) return false;
    if (len[s]) kraft += 1.0 / (double)(1u << len[s]);
  }
  if (kraft > 1.0) return false;
  canonical(len, 256, code);
  std::memset(table, 0, sizeof(uint32_t) << kMaxLen);
  for (int s = 0; s < 256; ++s) {
    if (!len[s]) continue;
    const uint32_t lo = code[s] << (kMaxLen - len[s]), hi = (code[s] + 1) << (kMaxLen - len[s]);
    for (uint32_t v = lo; v < hi; ++v) table[v] = (uint32_t)s | ((uint32_t)len[s] << 16);
  }
  return true;
}

// ---- device helpers ----

// Bits [p, p + 32) of an MSB-first bit stream of nw words (zeros past the end).
__device__ __forceinline__ uint32_t bits32(const uint32_t* w, uint64_t nw, uint64_t p) {
  const uint64_t i = p >> 5;
  const int o = (int)(p & 31);
  const uint32_t a = i < nw ? w[i] : 0u, b = i + 1 < nw ? w[i + 1] : 0u;
  return o ? (a << o) | (b >> (32 - o)) : a;
}

// Writes the low nbits (<= 64) of v, most significant first, at bit p.
__device__ __forceinline__ void put_bits(uint32_t* w, uint64_t p, uint64_t v, int nbits) {
  while (nbits > 0) {
    const int off = (int)(p & 31), take = min(32 - off, nbits);
    const uint32_t piece = (uint32_t)((v >> (nbits - take)) & ((1ull << take) - 1ull));
    atomicOr(&w[p >> 5], piece << (32 - off - take));
    p += (uint64_t)take;
    nbits -= take;
  }
}

// ---- exclusive scan of u32 values into u64 offsets (3 passes) ----

__global__ void __launch_bounds__(kET) k_scan_sum(const uint32_t* in, uint64_t n, uint64_t* bsum) {
  __shared__ uint64_t s[kET / 32];
  const uint64_t b0 = (uint64_t)blockIdx.x * kSeg;
  uint64_t t = 0;
  for (uint64_t i = b0 + threadIdx.x; i < min(n, b0 + kSeg); i += kET) t += in[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t a = 0;
    for (int k = 0; k < kET / 32; ++k) a += s[k];
    bsum[blockIdx.x] = a;
  }
}

// One block: exclusive scan of the nb block sums in place; *total = their sum.
__global__ void __launch_bounds__(1024) k_scan_blocks(uint64_t* bsum, uint64_t nb, uint64_t* total) {
  __shared__ uint64_t s[1024];
  __shared__ uint64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint64_t c = 0; c < nb; c += 1024) {
    const uint64_t i = c + threadIdx.x;
    const uint64_t x = i < nb ? bsum[i] : 0;
    s[threadIdx.x] = x;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const uint64_t y = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0;
      __syncthreads();
      s[threadIdx.x] += y;
      __syncthreads();
    }
    const uint64_t c0 = carry;
    if (i < nb) bsum[i] = c0 + s[threadIdx.x] - x;
    __syncthreads();
    if (threadIdx.x == 1023) carry = c0 + s[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(kET) k_scan_apply(const uint32_t* in, uint64_t n, const uint64_t* boff,
                                                   uint64_t* out) {
  __shared__ uint64_t s[kET];
  __shared__ uint64_t carry;
  const uint64_t b0 = (uint64_t)blockIdx.x * kSeg;
  if (threadIdx.x == 0) carry = boff[blockIdx.x];
  __syncthreads();
  for (uint64_t c = b0; c < min(n, b0 + kSeg); c += kET) {
    const uint64_t i = c + threadIdx.x;
    const uint64_t x = i < n ? in[i] : 0;
    s[threadIdx.x] = x;
    __syncthreads();
    for (int o = 1; o < kET; o <<= 1) {
      const uint64_t y = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0;
      __syncthreads();
      s[threadIdx.x] += y;
      __syncthreads();
    }
    const uint64_t c0 = carry;
    if (i < n) out[i] = c0 + s[threadIdx.x] - x;
    __syncthreads();
    if (threadIdx.x == kET - 1) carry = c0 + s[kET - 1];
    __syncthreads();
  }
}

// Exclusive offsets of in[0 .. n) into out, and their total (host).
bool scan_u32(const uint32_t* in, uint64_t n, uint64_t* out, uint64_t* bsum, uint64_t* d_total, uint64_t* total,
              cudaStream_t s) {
  const uint64_t nb = std::max<uint64_t>(1, (n + kSeg - 1) / kSeg);
  k_scan_sum<<<(unsigned)nb, kET, 0, s>>>(in, n, bsum);
  k_scan_blocks<<<1, 1024, 0, s>>>(bsum, nb, d_total);
  k_scan_apply<<<(unsigned)nb, kET, 0, s>>>(in, n, bsum, out);
  return cudaMemcpyAsync(total, d_total, sizeof(uint64_t), cudaMemcpyDeviceToHost, s) == cudaSuccess;
}

// ---- encoding kernels ----

// Index tokens, one warp per group of 32 edits: a maximal run of L >= 2
// deltas equal to 1 inside the group is one RUN token at its first edit (5
// raw bits L - 2); any other delta d is a literal (symbol d - 1, or an
// escape with 16 / 32 raw bits). tsym[k] = -1 for an edit inside a run.
// Histogram of the symbols into hist[256]. *bad is set for indices that are
// not strictly ascending or not below n_field.
__global__ void __launch_bounds__(kET) k_index_tokens(const uint32_t* idx, uint64_t n, uint32_t n_field,
                                                      int32_t* tsym, uint32_t* traw, uint32_t* tlen_raw,
                                                      uint32_t* tflag, uint32_t* hist, int* bad) {
  __shared__ uint32_t h[256];
  for (int k = threadIdx.x; k < 256; k += blockDim.x) h[k] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
  for (uint64_t grp = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); grp * kGroup < n;
       grp += warps) {
    const uint64_t k = grp * kGroup + (uint64_t)lane;
    const bool in = k < n;
    uint32_t d = 0;
    if (in) {
      const uint32_t v = idx[k];
      const uint32_t prev = k ? idx[k - 1] : 0xffffffffu;  // idx_{-1} = -1
      d = v - prev;                                        // mod 2^32: v + 1 for the first
      if (v >= n_field || (k && v <= prev)) atomicExch(bad, 1);
    }
    const uint32_t ones = __ballot_sync(kFull, in && d == 1u);
    int32_t sym = -1;
    uint32_t raw = 0, rb = 0;
    if (in) {
      if (d == 1u) {
        const bool start = lane == 0 || !((ones >> (lane - 1)) & 1u);
        if (start) {
          const uint32_t L = (uint32_t)__ffs(~(ones >> lane)) - 1u;  // consecutive ones from this lane
          const uint32_t run = (lane + L > 32) ? 32u - lane : L;
          if (run >= 2) {
            sym = kRun;
            raw = run - 2;
            rb = 5;
          } else {
            sym = 0;
          }
        }
      } else if (d <= 252u) {
        sym = (int32_t)d - 1;
      } else if (d <= 253u + 65535u) {
        sym = kEsc16;
        raw = d - 253u;
        rb = 16;
      } else {
        sym = kEsc32;
        raw = d;
        rb = 32;
      }
      tsym[k] = sym;
      traw[k] = raw;
      tlen_raw[k] = rb;
      tflag[k] = sym >= 0 ? 1u : 0u;
      if (sym >= 0) atomicAdd(&h[sym], 1u);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 256; k += blockDim.x)
    if (h[k]) atomicAdd(&hist[k], h[k]);
}

// Value symbols: byte j of bits(val[k]) XOR bits(fhat[idx[k]]), k = j / es,
// little-endian; histogram into hist[256].
template <class U>
__global__ void __launch_bounds__(kET) k_value_symbols(const uint32_t* idx, const U* val, const U* fhat, uint64_t n,
                                                       uint32_t n_field, uint8_t* vsym, uint32_t* hist) {
  __shared__ uint32_t h[256];
  for (int k = threadIdx.x; k < 256; k += blockDim.x) h[k] = 0;
  __syncthreads();
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t i = idx[k];
    const U x = val[k] ^ (i < n_field ? fhat[i] : (U)0);
#pragma unroll
    for (int b = 0; b < (int)sizeof(U); ++b) {
      const uint8_t y = (uint8_t)(x >> (8 * b));
      vsym[k * sizeof(U) + b] = y;
      atomicAdd(&h[y], 1u);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 256; k += blockDim.x)
    if (h[k]) atomicAdd(&hist[k], h[k]);
}

// Bit length of every token (code + raw bits; 0 where there is none).
__global__ void __launch_bounds__(kET) k_index_bits(const int32_t* tsym, const uint32_t* tlen_raw, uint64_t n,
                                                    const uint8_t* len, uint32_t* nb) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x)
    nb[k] = tsym[k] >= 0 ? (uint32_t)len[tsym[k]] + tlen_raw[k] : 0u;
}

__global__ void __launch_bounds__(kET) k_value_bits(const uint8_t* vsym, uint64_t m, const uint8_t* len,
                                                    uint32_t* nb) {
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (uint64_t)gridDim.x * blockDim.x)
    nb[j] = len[vsym[j]];
}

// Packs the index tokens at their bit offsets; the first token of every
// chunk records (bit offset, edit, index before it).
struct IChunk {
  uint64_t bit;
  uint32_t first, prev;
};
__global__ void __launch_bounds__(kET) k_index_write(const uint32_t* idx, const int32_t* tsym, const uint32_t* traw,
                                                     const uint32_t* tlen_raw, const uint64_t* boff,
                                                     const uint64_t* tnum, uint64_t n, const uint8_t* len,
                                                     const uint32_t* code, uint32_t* words, IChunk* chunks) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) {
    const int32_t s = tsym[k];
    if (s < 0) continue;
    const int rb = (int)tlen_raw[k];
    const uint64_t v = ((uint64_t)code[s] << rb) | (uint64_t)traw[k];
    put_bits(words, boff[k], v, (int)len[s] + rb);
    if (tnum[k] % kChunk == 0) chunks[tnum[k] / kChunk] = {boff[k], (uint32_t)k, k ? idx[k - 1] : 0xffffffffu};
  }
}

__global__ void __launch_bounds__(kET) k_value_write(const uint8_t* vsym, const uint64_t* boff, uint64_t m,
                                                     const uint8_t* len, const uint32_t* code, uint32_t* words,
                                                     uint64_t* chunks) {
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (uint64_t)gridDim.x * blockDim.x) {
    const uint8_t s = vsym[j];
    put_bits(words, boff[j], code[s], len[s]);
    if (j % kChunk == 0) chunks[j / kChunk] = boff[j];
  }
}

// ---- decoding kernels ----

// One thread per index chunk: tokens [c * kChunk, min(ntok, (c + 1) * kChunk))
// from the chunk's bit offset, edits from its first edit on. Malformed input
// (no code, an index at or past n_field, more edits than n) sets *bad.
__global__ void __launch_bounds__(kET) k_index_decode(const uint32_t* words, uint64_t nw, const IChunk* chunks,
                                                      uint32_t nci, uint32_t ntok, uint64_t n, uint32_t n_field,
                                                      const uint32_t* table, uint32_t* idx, int* bad) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nci) return;
  const IChunk ch = chunks[c];
  uint64_t p = ch.bit, k = ch.first;
  uint32_t prev = ch.prev;  // 0xffffffff: before the first edit (idx_{-1} = -1)
  const uint32_t t1 = min(ntok, (c + 1) * (uint32_t)kChunk);
  for (uint32_t t = c * (uint32_t)kChunk; t < t1; ++t) {
    const uint32_t e = table[bits32(words, nw, p) >> (32 - kMaxLen)];
    const int l = (int)(e >> 16), s = (int)(e & 0xffffu);
    if (l == 0) {
      atomicExch(bad, 1);
      return;
    }
    p += (uint64_t)l;
    uint32_t cnt = 1, d = (uint32_t)s + 1u;
    if (s == kRun) {
      cnt = (bits32(words, nw, p) >> 27) + 2u;
      p += 5;
      d = 1;
    } else if (s == kEsc16) {
      d = (bits32(words, nw, p) >> 16) + 253u;
      p += 16;
    } else if (s == kEsc32) {
      d = bits32(words, nw, p);
      p += 32;
    }
    for (uint32_t r = 0; r < cnt; ++r) {
      prev += d;  // mod 2^32: the first edit's delta is its index + 1
      if (k >= n || prev >= n_field) {
        atomicExch(bad, 1);
        return;
      }
      idx[k++] = prev;
    }
  }
}

// One thread per value chunk of kChunk bytes (whole values: kChunk is a
// multiple of the value size): value = bytes XOR bits(fhat[idx]).
template <class U>
__global__ void __launch_bounds__(kET) k_value_decode(const uint32_t* words, uint64_t nw, const uint64_t* chunks,
                                                      uint32_t ncv, uint64_t m, const uint32_t* table,
                                                      const uint32_t* idx, const U* fhat, uint32_t n_field, U* val,
                                                      int* bad) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncv) return;
  uint64_t p = chunks[c];
  const uint64_t j0 = (uint64_t)c * kChunk, j1 = min(m, j0 + kChunk);
  U x = 0;
  for (uint64_t j = j0; j < j1; ++j) {
    const uint32_t e = table[bits32(words, nw, p) >> (32 - kMaxLen)];
    const int l = (int)(e >> 16);
    if (l == 0) {
      atomicExch(bad, 1);
      return;
    }
    p += (uint64_t)l;
    const int b = (int)(j % sizeof(U));
    x |= (U)(e & 0xffu) << (8 * b);
    if (b == (int)sizeof(U) - 1) {
      const uint64_t k = j / sizeof(U);
      const uint32_t i = idx[k];
      if (i >= n_field) {
        atomicExch(bad, 1);
        return;
      }
      val[k] = x ^ fhat[i];
      x = 0;
    }
  }
}

int grid_for(uint64_t items) {
  return (int)std::max<uint64_t>(1, std::min<uint64_t>((items + kET - 1) / kET, 152ull * 16));
}

}  // namespace
}  // namespace msz

using namespace msz;

namespace {
size_t value_size(int dtype) { return dtype == MSZ_F32 ? 4 : 8; }

// Geometry check shared by both entry points: the field's vertex count.
bool field_size(int ndim, const int64_t* dims, uint32_t& n_field) {
  if ((ndim != 2 && ndim != 3) || !dims) return false;
  const int64_t nx = dims[0], ny = dims[1], nz = ndim == 3 ? dims[2] : 1;
  if (nx < 1 || ny < 1 || nz < 1 || nx > 0x7fffffff || ny > 0x7fffffff || nz > 0x7fffffff) return false;
  const int64_t n = nx * ny * nz;
  if (n > 0x7fffffffLL) return false;
  n_field = (uint32_t)n;
  return true;
}

struct Layout {
  uint64_t ci, cv, pi, pv, end, nwi, nwv;
};
Layout layout_of(uint64_t nci, uint64_t ncv, uint64_t bits_i, uint64_t bits_v) {
  Layout L;
  L.ci = kTables;
  L.cv = L.ci + 16 * nci;
  L.pi = L.cv + 8 * ncv;
  L.nwi = (bits_i + 31) / 32;
  L.pv = L.pi + 4 * L.nwi;
  L.nwv = (bits_v + 31) / 32;
  L.end = L.pv + 4 * L.nwv;
  return L;
}
}  // namespace

int64_t msz_edits_encoded_bound(uint64_t n_edits, int dtype) {
  if (dtype != MSZ_F32 && dtype != MSZ_F64) return MSZ_ERR_DTYPE;
  const uint64_t es = value_size(dtype), m = n_edits * es;
  const Layout L = layout_of((n_edits + kChunk - 1) / kChunk, (m + kChunk - 1) / kChunk,
                             n_edits * (uint64_t)(kMaxLen + 32), m * (uint64_t)kMaxLen);
  return (int64_t)L.end;
}

int msz_encode_edits(const uint32_t* edit_idx_dev, const void* edit_val_dev, uint64_t n_edits, const void* fhat_dev,
                     int ndim, const int64_t dims[3], int dtype, void* out_dev, uint64_t out_cap,
                     uint64_t* out_bytes, void* stream) {
  uint32_t n_field = 0;
  if (!field_size(ndim, dims, n_field)) return MSZ_ERR_ARG;
  if (dtype != MSZ_F32 && dtype != MSZ_F64) return MSZ_ERR_DTYPE;
  if (!out_dev || !out_bytes || (n_edits && (!edit_idx_dev || !edit_val_dev || !fhat_dev))) return MSZ_ERR_ARG;
  if (n_edits > n_field) return MSZ_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint64_t n = n_edits, es = value_size(dtype), m = n * es;
  Header H{kMagic, kVersion, (uint32_t)dtype, (uint32_t)es, n, 0, 0, 0, 0, 0, 0};
  uint8_t lens[512] = {};
  if (n == 0) {
    if (out_cap < kTables) return MSZ_ERR_ARG;
    unsigned char host[kTables];
    std::memcpy(host, &H, sizeof(H));
    std::memcpy(host + sizeof(H), lens, 512);
    if (cudaMemcpyAsync(out_dev, host, kTables, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return MSZ_ERR_CUDA;
    *out_bytes = kTables;
    return MSZ_OK;
  }
  // scratch
  const uint64_t nb = (std::max(n, m) + kSeg - 1) / kSeg + 1;
  const size_t bytes = n * (4 * 5 + 8 * 2) + m * (1 + 4 + 8) + 512 * 4 + nb * 8 + 64 + 512 * 4 + 512;
  unsigned char* sc = nullptr;
  if (cudaMallocAsync(&sc, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return MSZ_ERR_OOM;
  }
  size_t o = 0;
  uint64_t* boff_i = reinterpret_cast<uint64_t*>(sc + o); o += 8 * n;
  uint64_t* tnum = reinterpret_cast<uint64_t*>(sc + o); o += 8 * n;
  uint64_t* boff_v = reinterpret_cast<uint64_t*>(sc + o); o += 8 * m;
  uint64_t* bsum = reinterpret_cast<uint64_t*>(sc + o); o += 8 * nb;
  uint64_t* d_tot = reinterpret_cast<uint64_t*>(sc + o); o += 32;
  int32_t* tsym = reinterpret_cast<int32_t*>(sc + o); o += 4 * n;
  uint32_t* traw = reinterpret_cast<uint32_t*>(sc + o); o += 4 * n;
  uint32_t* trb = reinterpret_cast<uint32_t*>(sc + o); o += 4 * n;
  uint32_t* tflag = reinterpret_cast<uint32_t*>(sc + o); o += 4 * n;
  uint32_t* nbi = reinterpret_cast<uint32_t*>(sc + o); o += 4 * n;
  uint32_t* nbv = reinterpret_cast<uint32_t*>(sc + o); o += 4 * m;
  uint32_t* hist = reinterpret_cast<uint32_t*>(sc + o); o += 4 * 512;
  uint32_t* dcode = reinterpret_cast<uint32_t*>(sc + o); o += 4 * 512;
  int* bad = reinterpret_cast<int*>(sc + o); o += 16;
  uint8_t* dlen = sc + o; o += 512;
  uint8_t* vsym = sc + o; o += m;
  int status = MSZ_OK;
  auto fail = [&](int st) {
    if (status == MSZ_OK) status = st;
  };
  auto ok = [&](cudaError_t e) {
    if (e != cudaSuccess) fail(MSZ_ERR_CUDA);
  };
  uint32_t hh[512];
  int hbad = 0;
  ok(cudaMemsetAsync(hist, 0, 4 * 512, s));
  ok(cudaMemsetAsync(bad, 0, sizeof(int), s));
  k_index_tokens<<<grid_for((n + kGroup - 1) / kGroup * kGroup), kET, 0, s>>>(edit_idx_dev, n, n_field, tsym, traw,
                                                                              trb, tflag, hist, bad);
  if (dtype == MSZ_F32)
    k_value_symbols<uint32_t><<<grid_for(n), kET, 0, s>>>(edit_idx_dev, static_cast<const uint32_t*>(edit_val_dev),
                                                          static_cast<const uint32_t*>(fhat_dev), n, n_field, vsym,
                                                          hist + 256);
  else
    k_value_symbols<uint64_t><<<grid_for(n), kET, 0, s>>>(edit_idx_dev, static_cast<const uint64_t*>(edit_val_dev),
                                                          static_cast<const uint64_t*>(fhat_dev), n, n_field, vsym,
                                                          hist + 256);
  ok(cudaMemcpyAsync(hh, hist, sizeof(hh), cudaMemcpyDeviceToHost, s));
  ok(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  ok(cudaStreamSynchronize(s));
  if (status == MSZ_OK && hbad) fail(MSZ_ERR_ARG);  // indices not ascending or not in the field
  uint32_t codes[512] = {};
  uint64_t tot[3] = {0, 0, 0};
  Layout L{};
  if (status == MSZ_OK) {
    package_merge(hh, 256, kMaxLen, lens);
    package_merge(hh + 256, 256, kMaxLen, lens + 256);
    canonical(lens, 256, codes);
    canonical(lens + 256, 256, codes + 256);
    ok(cudaMemcpyAsync(dcode, codes, sizeof(codes), cudaMemcpyHostToDevice, s));
    ok(cudaMemcpyAsync(dlen, lens, 512, cudaMemcpyHostToDevice, s));
    k_index_bits<<<grid_for(n), kET, 0, s>>>(tsym, trb, n, dlen, nbi);
    k_value_bits<<<grid_for(m), kET, 0, s>>>(vsym, m, dlen + 256, nbv);
    if (!scan_u32(nbi, n, boff_i, bsum, d_tot, &tot[0], s) || !scan_u32(tflag, n, tnum, bsum, d_tot + 1, &tot[1], s) ||
        !scan_u32(nbv, m, boff_v, bsum, d_tot + 2, &tot[2], s))
      fail(MSZ_ERR_CUDA);
    ok(cudaStreamSynchronize(s));
  }
  if (status == MSZ_OK) {
    H.ntok = (uint32_t)tot[1];
    H.nci = (uint32_t)((tot[1] + kChunk - 1) / kChunk);
    H.ncv = (uint32_t)((m + kChunk - 1) / kChunk);
    H.bits_i = tot[0];
    H.bits_v = tot[2];
    L = layout_of(H.nci, H.ncv, H.bits_i, H.bits_v);
    if (L.end > out_cap) fail(MSZ_ERR_ARG);
  }
  if (status == MSZ_OK) {
    unsigned char* out = static_cast<unsigned char*>(out_dev);
    ok(cudaMemsetAsync(out + L.pi, 0, L.end - L.pi, s));
    k_index_write<<<grid_for(n), kET, 0, s>>>(edit_idx_dev, tsym, traw, trb, boff_i, tnum, n, dlen, dcode,
                                               reinterpret_cast<uint32_t*>(out + L.pi),
                                               reinterpret_cast<IChunk*>(out + L.ci));
    k_value_write<<<grid_for(m), kET, 0, s>>>(vsym, boff_v, m, dlen + 256, dcode + 256,
                                               reinterpret_cast<uint32_t*>(out + L.pv),
                                               reinterpret_cast<uint64_t*>(out + L.cv));
    unsigned char host[kTables];
    std::memcpy(host, &H, sizeof(H));
    std::memcpy(host + sizeof(H), lens, 512);
    ok(cudaMemcpyAsync(out, host, kTables, cudaMemcpyHostToDevice, s));
    ok(cudaStreamSynchronize(s));
  }
  cudaFreeAsync(sc, s);
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) fail(MSZ_ERR_CUDA);
  if (status == MSZ_OK) *out_bytes = L.end;
  return status;
}

int msz_decode_edits(const void* in_dev, uint64_t in_bytes, const void* fhat_dev, int ndim, const int64_t dims[3],
                     int dtype, uint32_t* edit_idx_dev, void* edit_val_dev, uint64_t cap_edits, uint64_t* n_edits,
                     void* stream) {
  uint32_t n_field = 0;
  if (!field_size(ndim, dims, n_field)) return MSZ_ERR_ARG;
  if (dtype != MSZ_F32 && dtype != MSZ_F64) return MSZ_ERR_DTYPE;
  if (!in_dev || !n_edits || in_bytes < kTables) return MSZ_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char host[kTables];
  if (cudaMemcpyAsync(host, in_dev, kTables, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return MSZ_ERR_CUDA;
  Header H;
  std::memcpy(&H, host, sizeof(H));
  const uint8_t* lens = host + sizeof(H);
  const uint64_t es = value_size(dtype), n = H.n, m = n * es;
  // the header must describe a well-formed stream of this field's type
  if (H.magic != kMagic || H.version != kVersion || H.dtype != (uint32_t)dtype || H.es != es) return MSZ_ERR_ARG;
  if (n > cap_edits || n > n_field || H.ntok > n || H.nci != (H.ntok + kChunk - 1) / kChunk ||
      H.ncv != (m + kChunk - 1) / kChunk)
    return MSZ_ERR_ARG;
  const Layout L = layout_of(H.nci, H.ncv, H.bits_i, H.bits_v);
  if (L.end > in_bytes) return MSZ_ERR_ARG;
  if (n == 0) {
    *n_edits = 0;
    return MSZ_OK;
  }
  if (!fhat_dev || !edit_idx_dev || !edit_val_dev) return MSZ_ERR_ARG;
  std::vector<uint32_t> tab(2u << kMaxLen);
  if (!decode_table(lens, tab.data()) || !decode_table(lens + 256, tab.data() + (1u << kMaxLen))) return MSZ_ERR_ARG;
  unsigned char* sc = nullptr;
  if (cudaMallocAsync(&sc, tab.size() * 4 + 16, s) != cudaSuccess) {
    cudaGetLastError();
    return MSZ_ERR_OOM;
  }
  uint32_t* dtab = reinterpret_cast<uint32_t*>(sc);
  int* bad = reinterpret_cast<int*>(sc + tab.size() * 4);
  int status = MSZ_OK, hbad = 0;
  const unsigned char* in = static_cast<const unsigned char*>(in_dev);
  if (cudaMemcpyAsync(dtab, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(bad, 0, sizeof(int), s) != cudaSuccess)
    status = MSZ_ERR_CUDA;
  if (status == MSZ_OK) {
    k_index_decode<<<(H.nci + kET - 1) / kET, kET, 0, s>>>(reinterpret_cast<const uint32_t*>(in + L.pi), L.nwi,
                                                           reinterpret_cast<const IChunk*>(in + L.ci), H.nci,
                                                           H.ntok, n, n_field, dtab, edit_idx_dev, bad);
    if (cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      status = MSZ_ERR_CUDA;
    else if (hbad)
      status = MSZ_ERR_ARG;
  }
  if (status == MSZ_OK) {
    const uint32_t* wv = reinterpret_cast<const uint32_t*>(in + L.pv);
    const uint64_t* cv = reinterpret_cast<const uint64_t*>(in + L.cv);
    const uint32_t* tv = dtab + (1u << kMaxLen);
    if (dtype == MSZ_F32)
      k_value_decode<uint32_t><<<(H.ncv + kET - 1) / kET, kET, 0, s>>>(
          wv, L.nwv, cv, H.ncv, m, tv, edit_idx_dev, static_cast<const uint32_t*>(fhat_dev), n_field,
          static_cast<uint32_t*>(edit_val_dev), bad);
    else
      k_value_decode<uint64_t><<<(H.ncv + kET - 1) / kET, kET, 0, s>>>(
          wv, L.nwv, cv, H.ncv, m, tv, edit_idx_dev, static_cast<const uint64_t*>(fhat_dev), n_field,
          static_cast<uint64_t*>(edit_val_dev), bad);
    if (cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      status = MSZ_ERR_CUDA;
    else if (hbad)
      status = MSZ_ERR_ARG;
  }
  cudaFreeAsync(sc, s);
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) status = MSZ_ERR_CUDA;
  if (status == MSZ_OK) *n_edits = n;
  return status;
}
