// C ABI of the MSz correction library (include/msz.h): the host-side engine
// that runs one or many fields through the work-unit kernels of
// msz_kernels.cuh, and the entry points built on it (single-field plans,
// the allocation-free variant, batches, directions, apply).
//
// A step of the loop (Sec. 4 of the paper, control flow of Fig. 3) is the
// kernel sequence, per (dtype, dimension) group of fields:
//   sweep      - extremum flags of g + false critical points (Sec. 5.1)
//   mark_c     - C-loop edit requests of the current type (Eqs. 2-5)
//   label_tile - directions of g and in-tile path compression (Sec. 5.2)
//   jump x J   - pointer jumping across tiles
//   rcheck     - wrong labels + troublemaker requests (Sec. 4.2, Eq. 6)
//   apply      - applies the round's requests (iteration-synchronous)
// Kernels skip fields with nothing to do; the unit that completes a field's
// work advances that field's state machine on the device. The host captures
// a few steps in a CUDA graph once, replays it, and reads the fields' states
// once per chunk: it never synchronises per iteration.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "msz.h"
#include "msz_kernels.cuh"

namespace msz {
namespace {

// ---------------------------------------------------------------------------
// Small host utilities
// ---------------------------------------------------------------------------
std::mutex g_mu;

int num_sms() {
  static int sms = 0;
  std::lock_guard<std::mutex> lk(g_mu);
  if (sms == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    sms = v;
  }
  return sms;
}

bool geom_from(int ndim, const int64_t* dims, Geom& G) {
  if (ndim != 2 && ndim != 3) return false;
  if (!dims) return false;
  const int64_t nx = dims[0], ny = dims[1], nz = (ndim == 3) ? dims[2] : 1;
  if (nx < 1 || ny < 1 || nz < 1) return false;
  if (nx > 0x7fffffff || ny > 0x7fffffff || nz > 0x7fffffff) return false;
  const int64_t n = nx * ny * nz;
  if (n > 0x7fffffffLL) return false;
  G.nx = (int)nx;
  G.ny = (int)ny;
  G.nz = (int)nz;
  G.nxny = (int)(nx * ny);
  G.n = (int)n;
  G.nd = ndim;
  G.dx = fast_div((uint32_t)nx);
  G.dy = fast_div((uint32_t)ny);
  return true;
}

size_t esize(int dtype) { return dtype == MSZ_F32 ? 4 : 8; }
size_t round_up(size_t a, size_t b) { return (a + b - 1) / b * b; }

bool xi_ok(double xi, int dtype) {
  if (!(xi >= 0.0) || !std::isfinite(xi)) return false;
  if (dtype == MSZ_F32 && !std::isfinite((float)xi)) return false;
  return true;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!tried) {
    tried = true;
    void* q = nullptr;
    cudaDriverEntryPointQueryResult r;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &q, 12000, cudaEnableDefault, &r) ==
            cudaSuccess &&
        r == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(q);
    else
      cudaGetLastError();
  }
  return fn;
}

// Bump allocator over one device block (owned cudaMalloc block or the static
// scratch of msz_fix_noalloc). take() only computes offsets when base is null,
// which is how sizes are measured.
struct Bump {
  unsigned char* base;
  size_t off;
  void* take(size_t bytes, size_t align = 256) {
    off = round_up(off, align);
    void* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  }
};

// Host-side arena for an engine's bookkeeping arrays (a heap block for
// engines that own their memory, a stack buffer for msz_fix_noalloc).
struct HostArena {
  unsigned char* base;
  size_t cap, off;
  template <class U>
  U* take(size_t count, size_t align = alignof(U) < 64 ? 64 : alignof(U)) {
    off = round_up(off, align);
    U* p = (base && off + sizeof(U) * count <= cap) ? reinterpret_cast<U*>(base + off) : nullptr;
    off += sizeof(U) * count;
    return p;
  }
};

// Device buffers of one field.
struct FieldBufs {
  void* g = nullptr;
  uint8_t* fdir = nullptr;
  uint8_t* gdir = nullptr;
  uint8_t* flags = nullptr;
  uint32_t* term = nullptr;
  int32_t* Pup = nullptr;
  int32_t* Pdn = nullptr;
  uint32_t* lf[2] = {nullptr, nullptr};
  uint32_t* lw[2] = {nullptr, nullptr};
  uint8_t* xm[2] = {nullptr, nullptr};
  uint8_t* tdirty = nullptr;
  uint32_t* texit = nullptr;
  uint32_t* tsnap = nullptr;
  uint8_t* twrong = nullptr;
  uint8_t* cls = nullptr;
  uint32_t* cases = nullptr;
  uint32_t* epoch = nullptr;
  uint32_t* ccnt = nullptr;
  uint32_t* touched = nullptr;
  uint32_t* tile_cnt = nullptr;
  uint32_t* edit_idx = nullptr;
  void* edit_val = nullptr;
};

int emit_tiles(const Geom& G) { return (G.n + kEmitTile - 1) / kEmitTile; }

int label_tiles(const Geom& G) {
  if (G.nd == 3) {
    using LG = LabelGeom<3>;
    return ((G.nx + LG::TX - 1) / LG::TX) * ((G.ny + LG::TY - 1) / LG::TY) * ((G.nz + LG::TZ - 1) / LG::TZ);
  }
  using LG = LabelGeom<2>;
  return ((G.nx + LG::TX - 1) / LG::TX) * ((G.ny + LG::TY - 1) / LG::TY);
}

// Exit-table slots per direction: a slot per face cell of every label tile,
// rounded up to 16 (the marks are cleared by words).
size_t exit_slots(const Geom& G) {
  const size_t nf = (size_t)label_tiles(G) * (size_t)(G.nd == 3 ? LabelGeom<3>::NFACE : LabelGeom<2>::NFACE);
  return (nf + 15) / 16 * 16;
}

// Entries of lw[0]: its slots, and room for the freezes of a k_csmall launch
// (at most one per case it holds).
size_t freeze_cap(const Geom& G) {
  return std::max(exit_slots(G), std::min((size_t)G.n, (size_t)kSmallCases));
}

// Carves a field's buffers. Outputs (labels Pup/Pdn, edit list) are carved
// too unless the caller supplies them (with_outputs = false).
void carve_field(Bump& b, const Geom& G, int dtype, bool with_outputs, FieldBufs& B) {
  const size_t n = (size_t)G.n, es = esize(dtype), nt = (size_t)emit_tiles(G);
  B.g = b.take(n * es);
  B.fdir = (uint8_t*)b.take(n);
  B.gdir = (uint8_t*)b.take(n);
  B.flags = (uint8_t*)b.take(nt * kEmitTile);
  B.term = (uint32_t*)b.take(n * 4);
  const size_t nf = exit_slots(G);
  for (int d = 0; d < 2; ++d) {
    B.lf[d] = (uint32_t*)b.take(nf * 4);
    B.lw[d] = (uint32_t*)b.take((d == 0 ? freeze_cap(G) : nf) * 4);
    B.xm[d] = (uint8_t*)b.take(nf);
  }
  B.tdirty = (uint8_t*)b.take((size_t)label_tiles(G));
  B.texit = (uint32_t*)b.take((size_t)label_tiles(G) * 2 * (G.nd == 3 ? LabelGeom<3>::SHW : LabelGeom<2>::SHW) * 4);
  B.tsnap = (uint32_t*)b.take((size_t)label_tiles(G) * 2 * (G.nd == 3 ? LabelGeom<3>::SHELL : LabelGeom<2>::SHELL) * 4);
  B.twrong = (uint8_t*)b.take((size_t)label_tiles(G));
  B.cls = (uint8_t*)b.take(nt * kEmitTile);
  B.cases = (uint32_t*)b.take(n * 4);
  B.epoch = (uint32_t*)b.take(n * 4);
  B.ccnt = (uint32_t*)b.take(nt * 4 * 4);
  B.touched = (uint32_t*)b.take(n * 4);
  B.tile_cnt = (uint32_t*)b.take(nt * 4);
  if (with_outputs) {
    B.Pup = (int32_t*)b.take(n * 4);
    B.Pdn = (int32_t*)b.take(n * 4);
    B.edit_idx = (uint32_t*)b.take(n * 4);
    B.edit_val = b.take(n * es);
  }
}

// ---------------------------------------------------------------------------
// One (dtype, dimension) group of an engine's fields.
// ---------------------------------------------------------------------------
constexpr int kJumpsPerStep = 2;
// A step holds two C-loop rounds (gather, mark, apply, reclassify): most
// steps of a fix are C-loop rounds, and every launch of a stage that no field
// is in still costs a few microseconds.
constexpr int kStepSlots = 13 + kJumpsPerStep;  // launches per step
constexpr int kStepEvents = kStepSlots + 1;
static_assert(kStepSlots <= 32, "the step log holds one bit per launch slot");
// kernel of each launch slot of a step
constexpr int kSlotKernel[kStepSlots] = {KID_SWEEP, KID_GATHER, KID_CSMALL, KID_MARK,   KID_APPLY,
                                         KID_RECLASS, KID_GATHER, KID_MARK,  KID_LABEL,  KID_LABEL,
                                         KID_JUMP,  KID_JUMP,   KID_RCHECK, KID_APPLY, KID_RECLASS};
static_assert(kJumpsPerStep == 2, "slot table assumes two jump launches per step");
static_assert(NKID == MSZ_NUM_KERNELS, "kernel table and ABI disagree");
const char* const kKernelNames[NKID] = {"k_csweep", "k_gather", "k_mark",    "k_label_tile", "k_jump",
                                        "k_rcheck", "k_apply",  "k_reclass", "k_csmall"};

template <class T, int ND>
struct Group {
  using SG = SweepGeom<T, ND>;
  using LG = LabelGeom<ND>;
  int nf = 0;
  int* members = nullptr;  // engine field indices
  Field<T>* h_fields = nullptr;
  int* h_prefix = nullptr;
  CUtensorMap* h_maps = nullptr;
  Field<T>* d_fields = nullptr;
  int* d_prefix = nullptr;
  CUtensorMap* d_maps = nullptr;
  GroupArgs<T> args{};
  bool tma = false;
  int grid[NKIND] = {};
  bool small_ok[2] = {false, false};  // a k_csmall cluster of 16 / 4 blocks fits on the device
  bool small_has[2] = {false, false};  // some field's small rounds run in that cluster size
  size_t label_smem[2] = {0, 0};  // f's pass, g's passes
  int grid_label[2] = {0, 0};
  int grid_rcheck = 0;

  // Host arrays for nf fields (null pointers while measuring).
  void host_carve(HostArena& h) {
    if (nf == 0) return;  // an empty group is never set up or launched
    members = h.take<int>(std::max(nf, 1));
    h_fields = h.take<Field<T>>(std::max(nf, 1));
    h_prefix = h.take<int>(NKIND * (nf + 1));
    h_maps = h.take<CUtensorMap>(2 * std::max(nf, 1), 128);
  }
  bool empty() const { return nf == 0; }

  // Device bytes of the group's descriptor arrays.
  void carve(Bump& b) {
    if (nf == 0) return;
    d_fields = (Field<T>*)b.take(sizeof(Field<T>) * std::max(nf, 1), 64);
    d_prefix = (int*)b.take(sizeof(int) * NKIND * (nf + 1), 64);
    d_maps = (CUtensorMap*)b.take(sizeof(CUtensorMap) * 2 * std::max(nf, 1), 128);
  }

  static SweepTiling tiling(const Geom& G, int max_chunk) {
    SweepTiling TL;
    const int axis = (ND == 3) ? G.nz : G.ny;  // marching axis
    const int nchunks = (axis + max_chunk - 1) / max_chunk;
    TL.chunk = (axis + nchunks - 1) / nchunks;
    TL.chunks = (axis + TL.chunk - 1) / TL.chunk;
    TL.tiles_x = (G.nx + SG::TX - 1) / SG::TX;
    TL.tiles_y = (ND == 3) ? (G.ny + SG::TY - 1) / SG::TY : 1;
    TL.ntiles = TL.tiles_x * TL.tiles_y * TL.chunks;
    return TL;
  }

  static bool encode(CUtensorMap* maps, const Geom& G, void* g, void* fdir) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t es = sizeof(T);
    if (((cuuint64_t)G.nx * es) % 16 != 0 || (cuuint64_t)G.nx % 16 != 0) return false;
    const CUtensorMapDataType dt = (sizeof(T) == 4) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    cuuint64_t gdim[3] = {(cuuint64_t)G.nx, (cuuint64_t)G.ny, (cuuint64_t)G.nz};
    cuuint64_t gstride[2] = {(cuuint64_t)G.nx * es, (cuuint64_t)G.nx * (cuuint64_t)G.ny * es};
    cuuint32_t box[3] = {(cuuint32_t)SG::BX, (cuuint32_t)SG::BY, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    const cuuint32_t rank = (ND == 3) ? 3 : 2;
    CUresult r = enc(&maps[0], dt, rank, g, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NAN_REQUEST_ZERO_FMA);
    if (r != CUDA_SUCCESS) return false;
    cuuint64_t dstride[2] = {(cuuint64_t)G.nx, (cuuint64_t)G.nx * (cuuint64_t)G.ny};
    cuuint32_t dbox[3] = {(cuuint32_t)SG::TX, (cuuint32_t)((ND == 3) ? SG::TY : 1), 1};
    r = enc(&maps[1], CU_TENSOR_MAP_DATA_TYPE_UINT8, rank, fdir, gdim, dstride, dbox, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
  }

  // Builds descriptors, tensor maps, prefix sums and launch shapes.
  // engine_fields: the fields of the whole engine (all groups)
  int setup(const Geom* geoms, const FieldBufs* bufs, DevState* d_states, bool allow_tma, const msz_tuning& tn,
            int engine_fields) {
    std::memset(h_maps, 0, sizeof(CUtensorMap) * 2 * nf);
    std::memset(h_prefix, 0, sizeof(int) * NKIND * (nf + 1));
    tma = allow_tma;
    for (int j = 0; j < nf; ++j) {
      const int fi = members[j];
      const Geom& G = geoms[fi];
      const FieldBufs& B = bufs[fi];
      Field<T>& F = h_fields[j];
      std::memset(&F, 0, sizeof(F));
      F.g = (T*)B.g;
      F.fdir = B.fdir;
      F.gdir = B.gdir;
      F.flags = B.flags;
      // f's labels are resolved straight into the output arrays: the loop
      // ends only when g's labels equal them, so they are the final labels
      F.Mf = B.Pup;
      F.mf = B.Pdn;
      F.Pup = B.Pup;
      F.Pdn = B.Pdn;
      F.term = B.term;
      for (int d = 0; d < 2; ++d) {
        F.lf[d] = B.lf[d];
        F.lw[d] = B.lw[d];
        F.xm[d] = B.xm[d];
      }
      F.nface = (uint32_t)exit_slots(G);
      F.fz_cap = (uint32_t)freeze_cap(G);
      F.tdirty = B.tdirty;
      F.texit = B.texit;
      F.tsnap = B.tsnap;
      F.twrong = B.twrong;
      F.cls = B.cls;
      F.cases = B.cases;
      F.epoch = B.epoch;
      F.ccnt = B.ccnt;
      F.touched = B.touched;
      F.tile_cnt = B.tile_cnt;
      F.edit_idx = B.edit_idx;
      F.edit_val = (T*)B.edit_val;
      F.st = d_states + fi;
      F.G = G;
      F.TL = tiling(G, tn.sweep_chunk);
      F.units[K_DENSE] = (G.n + kDenseChunk - 1) / kDenseChunk;
      F.units[K_SWEEP] = F.TL.ntiles;
      F.units[K_LABEL] = label_tiles(G);
      F.units[K_SPARSE] = std::max(1, std::min(4096, G.n / 2048));
      F.units[K_EMIT] = emit_tiles(G);
      F.units[K_CASE] = (emit_tiles(G) + kCaseTiles - 1) / kCaseTiles;
      if (tma && !encode(&h_maps[2 * j], G, B.g, B.fdir)) tma = false;
    }
    for (int k = 0; k < NKIND; ++k)
      for (int j = 0; j < nf; ++j) h_prefix[k * (nf + 1) + j + 1] = h_prefix[k * (nf + 1) + j] + h_fields[j].units[k];
    args.fields = d_fields;
    args.prefix = d_prefix;
    args.maps = d_maps;
    args.nf = nf;
    for (int k = 0; k < NKIND; ++k) args.total[k] = h_prefix[k * (nf + 1) + nf];
    // launch shapes: persistent grids over units
    args.chase = tn.chase_steps;
    args.small_rounds = tn.small_rounds;
    args.small_cases = (uint32_t)tn.small_cases;
    const int sms = num_sms();
    // persistent grids: the kernel's occupancy (or fewer blocks per SM, as
    // the tuning asks) times the SMs, at most one block per unit
    auto occ_grid = [&](const void* fn, int threads, size_t smem, int units) {
      int occ = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem);
      if (occ < 1) occ = 1;
      if (tn.blocks_per_sm > 0) occ = std::min(occ, tn.blocks_per_sm);
      return std::max(1, std::min(units, occ * sms));
    };
    grid[K_DENSE] = occ_grid((const void*)k_jump<T>, kThreads, 0, args.total[K_DENSE]);
    grid[K_SPARSE] = occ_grid((const void*)k_apply<T>, kThreads, 0, args.total[K_SPARSE]);
    grid[K_EMIT] = occ_grid((const void*)k_emit_write<T>, kThreads, 0, args.total[K_EMIT]);
    grid[K_CASE] = occ_grid((const void*)k_gather<T, ND>, kThreads, 0, args.total[K_CASE]);
    grid[K_SWEEP] = tma ? occ_grid((const void*)k_csweep<T, ND, true>, SG::NTP, 0, args.total[K_SWEEP])
                        : occ_grid((const void*)k_csweep<T, ND, false>, SG::NT, 0, args.total[K_SWEEP]);
    label_smem[0] = label_smem_bytes<T, ND, false>();
    label_smem[1] = label_smem_bytes<T, ND, true>();
    if (cudaFuncSetAttribute(k_label_tile<T, ND, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)label_smem[0]) != cudaSuccess ||
        cudaFuncSetAttribute(k_label_tile<T, ND, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)label_smem[1]) != cudaSuccess)
      return MSZ_ERR_CUDA;
    grid_label[0] = occ_grid((const void*)k_label_tile<T, ND, false>, kThreads, label_smem[0], args.total[K_LABEL]);
    grid_label[1] = occ_grid((const void*)k_label_tile<T, ND, true>, kThreads, label_smem[1], args.total[K_LABEL]);
    grid_rcheck = occ_grid((const void*)k_rcheck<T, ND>, kThreads, 0, args.total[K_LABEL]);
    if (cudaGetLastError() != cudaSuccess) return MSZ_ERR_CUDA;
    // a device without clusters of a size runs those fields' rounds on the
    // grid kernels; ncl: how many clusters of the size fit at once
    auto cluster_fits = [&](const void* fn, int cs, int& ncl) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(cs);
      cfg.blockDim = dim3(kSmallThreads);
      cudaLaunchAttribute at;
      at.id = cudaLaunchAttributeClusterDimension;
      at.val.clusterDim.x = cs;
      at.val.clusterDim.y = at.val.clusterDim.z = 1;
      cfg.attrs = &at;
      cfg.numAttrs = 1;
      ncl = 0;
      if (cs > 8) cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      const bool ok = cudaOccupancyMaxActiveClusters(&ncl, fn, &cfg) == cudaSuccess && ncl > 0;
      cudaGetLastError();
      return ok;
    };
    int ncl16 = 0, ncl4 = 0;
    small_ok[0] = cluster_fits((const void*)k_csmall<T, ND, kSmallCluster>, kSmallCluster, ncl16);
    small_ok[1] = cluster_fits((const void*)k_csmall<T, ND, kSmallClusterLite>, kSmallClusterLite, ncl4);
    const bool lite = small_ok[1] && engine_fields > ncl16;  // more fields than 16-block clusters fit
    small_has[0] = small_has[1] = false;
    for (int j = 0; j < nf; ++j) {
      Field<T>& F = h_fields[j];
      F.small_cluster = (lite && F.G.n <= kSmallLiteVertices) ? kSmallClusterLite : kSmallCluster;
      small_has[F.small_cluster == kSmallCluster ? 0 : 1] = true;
    }
    return MSZ_OK;
  }

  // Uploads the descriptors with this run's inputs and bounds.
  int upload(const void* const* f, const void* const* fhat, const double* xi, cudaStream_t s) {
    for (int j = 0; j < nf; ++j) {
      const int fi = members[j];
      h_fields[j].f = (const T*)f[fi];
      h_fields[j].fhat = (const T*)fhat[fi];
      h_fields[j].xi = (T)xi[fi];
    }
    if (cudaMemcpyAsync(d_fields, h_fields, sizeof(Field<T>) * nf, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return MSZ_ERR_CUDA;
    if (cudaMemcpyAsync(d_prefix, h_prefix, sizeof(int) * NKIND * (nf + 1), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
      return MSZ_ERR_CUDA;
    if (cudaMemcpyAsync(d_maps, h_maps, sizeof(CUtensorMap) * 2 * nf, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return MSZ_ERR_CUDA;
    return MSZ_OK;
  }

  // csweep, (gather, csmall, mark, apply, reclass), gather, mark, label_tile
  // (f's, g's), jump x jumps, rcheck, apply, reclass
  int launches_per_step(int jumps) const { return empty() ? 0 : 13 + jumps; }

  void init(cudaStream_t s) {
    if (empty()) return;
    k_init<T><<<grid[K_DENSE], kThreads, 0, s>>>(args);
  }

  // One loop step, all kernels (each acts only on the fields in its stage).
  // Kernel timing (single-field plans with MSZ_OPT_TIME_KERNELS): e holds
  // kStepEvents events, one before each launch and one after the last; each
  // launch gets the step's log slot.
  void step(cudaStream_t s, int jumps, cudaEvent_t* e = nullptr, uint32_t* steplog = nullptr, int si = 0) {
    if (empty()) return;
    int slot = 0;
    auto a = [&]() {
      GroupArgs<T> x = args;
      if (e) {
        cudaEventRecord(e[slot], s);
        x.steplog = steplog;
        x.step = si;
        x.slot = slot;
      }
      ++slot;
      return x;
    };
    sweep(s, a());
    gather(s, a, true);
    tail(s, a);
    gather(s, a, false);
    labels(s, a, jumps);
    tail(s, a);
    if (e) cudaEventRecord(e[slot], s);
  }

  // Step pieces.
  void sweep(cudaStream_t s, const GroupArgs<T>& x) {
    if (tma) k_csweep<T, ND, true><<<grid[K_SWEEP], SG::NTP, 0, s>>>(x);
    else k_csweep<T, ND, false><<<grid[K_SWEEP], SG::NT, 0, s>>>(x);
  }
  // small: the listed round may run in k_csmall (with the rounds after it)
  template <class A>
  void gather(cudaStream_t s, A&& a, bool small) {
    k_gather<T, ND><<<grid[K_CASE], kThreads, 0, s>>>(a());
    if (small) {
      const GroupArgs<T> x = a();  // the slot counts even when the kernel is left out
      if (args.small_rounds > 0) {
        if (small_ok[0] && small_has[0])
          k_csmall<T, ND, kSmallCluster><<<nf * kSmallCluster, kSmallThreads, 0, s>>>(x);
        if (small_ok[1] && small_has[1])
          k_csmall<T, ND, kSmallClusterLite><<<nf * kSmallClusterLite, kSmallThreads, 0, s>>>(x);
      }
    }
    k_mark<T, ND><<<grid[K_SPARSE], kThreads, 0, s>>>(a());
  }
  template <class A>
  void labels(cudaStream_t s, A&& a, int jumps) {
    k_label_tile<T, ND, false><<<grid_label[0], kThreads, label_smem[0], s>>>(a());
    k_label_tile<T, ND, true><<<grid_label[1], kThreads, label_smem[1], s>>>(a());
    for (int j = 0; j < jumps; ++j) k_jump<T><<<grid[K_DENSE], kThreads, 0, s>>>(a());
    k_rcheck<T, ND><<<grid_rcheck, kThreads, 0, s>>>(a());
  }
  template <class A>
  void tail(cudaStream_t s, A&& a) {
    k_apply<T><<<grid[K_SPARSE], kThreads, 0, s>>>(a());
    k_reclass<T, ND><<<grid[K_SPARSE], kThreads, 0, s>>>(a());
  }

  void emit(cudaStream_t s) {
    if (empty()) return;
    k_emit_count<T><<<grid[K_EMIT], kThreads, 0, s>>>(args);
    k_emit_scan<T><<<args.nf, 1024, 0, s>>>(args);
    k_emit_write<T><<<grid[K_EMIT], kThreads, 0, s>>>(args);
  }
};

constexpr int kMaxChunk = 32;
// Groups per (dtype, dimension) class: a batch's fields of one class are
// dealt to these in turn, so that fields that need many rounds hold back only
// their own group's launches.
constexpr int kSubGroups = 2;
constexpr int kKinds = 4;

// Defaults and ranges of msz_tuning.
constexpr msz_tuning kDefaultTuning = {kJumpsPerStep, 32, 64, (int32_t)kSmallCases, 4, 64, 0, {0, 0, 0, 0, 0}};

bool tuning_ok(const msz_tuning& t) {
  for (int k = 0; k < 5; ++k)
    if (t.reserved[k] != 0) return false;
  return t.jumps_per_step >= 1 && t.jumps_per_step <= 4 && t.chase_steps >= 4 && t.chase_steps <= 256 &&
         t.small_rounds >= 0 && t.small_rounds <= 1024 && t.small_cases >= 1 && t.small_cases <= (int)kSmallCases &&
         t.graph_steps >= 1 && t.graph_steps <= 8 && t.sweep_chunk >= 4 && t.sweep_chunk <= 64 &&
         t.blocks_per_sm >= 0 && t.blocks_per_sm <= 64;
}

}  // namespace
}  // namespace msz

using namespace msz;

// ---------------------------------------------------------------------------
// Engine: a set of fields run together (a plan is an engine of one field).
// ---------------------------------------------------------------------------
struct msz_engine_s {
  int nf = 0;
  int device = 0;
  msz_options opt{};
  msz_tuning tune = kDefaultTuning;
  Geom* geoms = nullptr;
  int* dtypes = nullptr;
  FieldBufs* bufs = nullptr;
  unsigned char* host_mem = nullptr;  // heap block behind the host arrays (owned engines)
  DevState* d_states = nullptr;
  DevState* h_states = nullptr;  // pinned when owned, caller-provided otherwise
  bool h_states_pinned = false;
  // a class's fields are dealt in turn to kSubGroups groups, each of which
  // runs its steps on a stream of its own (issue_steps)
  Group<float, 2> gf2[kSubGroups];
  Group<float, 3> gf3[kSubGroups];
  Group<double, 2> gd2[kSubGroups];
  Group<double, 3> gd3[kSubGroups];
  void* block = nullptr;  // owned device block (null for the static scratch)
  size_t block_bytes = 0;
  cudaStream_t cap_stream = nullptr;
  // groups after the first run their steps on these streams, forked from
  // and joined back into the launching stream (engines with several groups)
  cudaStream_t grp_stream[4 * kSubGroups - 1] = {};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[4 * kSubGroups - 1] = {};
  cudaGraphExec_t graph = nullptr;
  bool use_graph = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEvent_t tev[kMaxChunk][kStepEvents] = {};
  bool tev_ready = false;
  double kernel_ms[kKinds] = {0, 0, 0, 0};
  // per-kernel statistics of the last timed run (single-field engines)
  uint32_t* d_steplog = nullptr;
  uint32_t h_steplog[kMaxChunk] = {};
  uint64_t ks_launches[NKID] = {}, ks_work[NKID] = {}, ks_units[NKID] = {};
  double ks_ms[NKID] = {}, ks_work_ms[NKID] = {};
  uint64_t launches = 0;
  // staging for msz_fix_host
  void* in_f = nullptr;
  void* in_fhat = nullptr;

  template <class Fn>
  void each_group(Fn&& fn) {
    for (int k = 0; k < kSubGroups; ++k) fn(gf2[k]);
    for (int k = 0; k < kSubGroups; ++k) fn(gf3[k]);
    for (int k = 0; k < kSubGroups; ++k) fn(gd2[k]);
    for (int k = 0; k < kSubGroups; ++k) fn(gd3[k]);
  }
  // Calls fn on the group that takes the k-th field (counted from 0) of a
  // class.
  template <class Fn>
  void class_group(int dtype, int nd, int k, Fn&& fn) {
    const int j = k % kSubGroups;
    if (dtype == MSZ_F32) {
      if (nd == 3) fn(gf3[j]);
      else fn(gf2[j]);
    } else {
      if (nd == 3) fn(gd3[j]);
      else fn(gd2[j]);
    }
  }
  int launches_per_step(int jumps) {
    int n = 0;
    each_group([&](auto& g) { n += g.launches_per_step(jumps); });
    return n;
  }
};

namespace msz {
namespace {

// Host bookkeeping arrays of an engine (h.base == null: measures). The
// group sizes must be known (assign_counts) before.
void host_layout(msz_engine_s* E, HostArena& h) {
  E->geoms = h.take<Geom>(E->nf);
  E->dtypes = h.take<int>(E->nf);
  E->bufs = h.take<FieldBufs>(E->nf);
  E->each_group([&](auto& g) { g.host_carve(h); });
}

// Lays out (base == null: measures) every device array of an engine.
size_t layout_engine(msz_engine_s* E, unsigned char* base, bool with_outputs) {
  Bump b{base, 0};
  for (int i = 0; i < E->nf; ++i) {
    FieldBufs tmp;
    carve_field(b, E->geoms[i], E->dtypes[i], with_outputs, base ? E->bufs[i] : tmp);
  }
  E->d_states = (DevState*)b.take(sizeof(DevState) * E->nf, 256);
  E->d_steplog = (uint32_t*)b.take(sizeof(uint32_t) * kMaxChunk, 256);
  E->each_group([&](auto& g) { g.carve(b); });
  return b.off;
}


// Group sizes from the fields' dtypes and dimensions.
void assign_counts(msz_engine_s* E, const int* ndim, const int* dtype) {
  E->each_group([](auto& g) { g.nf = 0; });
  int cls[4] = {0, 0, 0, 0};  // fields per class so far
  for (int i = 0; i < E->nf; ++i) {
    int& k = cls[(dtype[i] == MSZ_F32 ? 0 : 2) + (ndim[i] == 3 ? 1 : 0)];
    E->class_group(dtype[i], ndim[i], k++, [](auto& g) { ++g.nf; });
  }
}

// Fills the groups' member lists (host arrays must exist). fields: the
// engine fields to place, in order (all of them, or a server's running slots).
void assign_members(msz_engine_s* E, const int* fields, int n) {
  E->each_group([](auto& g) { g.nf = 0; });
  int cls[4] = {0, 0, 0, 0};
  for (int j = 0; j < n; ++j) {
    const int i = fields ? fields[j] : j;
    const int nd = E->geoms[i].nd;
    int& k = cls[(E->dtypes[i] == MSZ_F32 ? 0 : 2) + (nd == 3 ? 1 : 0)];
    E->class_group(E->dtypes[i], nd, k++, [&](auto& g) { g.members[g.nf++] = i; });
  }
}

int setup_groups(msz_engine_s* E) {
  int rc = MSZ_OK;
  const bool allow_tma = !(E->opt.flags & MSZ_OPT_NO_TMA);
  E->each_group([&](auto& g) {
    if (rc == MSZ_OK && !g.empty()) rc = g.setup(E->geoms, E->bufs, E->d_states, allow_tma, E->tune, E->nf);
  });
  return rc;
}

void free_engine(msz_engine_s* E) {
  if (E->graph) cudaGraphExecDestroy(E->graph);
  if (E->cap_stream) cudaStreamDestroy(E->cap_stream);
  for (int k = 0; k < 4 * kSubGroups - 1; ++k) {
    if (E->grp_stream[k]) cudaStreamDestroy(E->grp_stream[k]);
    if (E->join_ev[k]) cudaEventDestroy(E->join_ev[k]);
  }
  if (E->fork_ev) cudaEventDestroy(E->fork_ev);
  if (E->block) cudaFree(E->block);
  if (E->in_f) cudaFree(E->in_f);
  if (E->in_fhat) cudaFree(E->in_fhat);
  if (E->h_states_pinned && E->h_states) cudaFreeHost(E->h_states);
  if (E->ev0) cudaEventDestroy(E->ev0);
  if (E->ev1) cudaEventDestroy(E->ev1);
  if (E->tev_ready)
    for (int i = 0; i < kMaxChunk; ++i)
      for (int j = 0; j < kStepEvents; ++j) cudaEventDestroy(E->tev[i][j]);
  delete[] E->host_mem;
  delete E;
}

// Validates the field shapes and builds the host side of an engine of nf
// fields in the given host arena (measuring when h.base is null).
int host_engine(msz_engine_s* E, int nf, const int* ndim, const int64_t* dims, const int* dtype, HostArena& h) {
  E->nf = nf;
  assign_counts(E, ndim, dtype);
  host_layout(E, h);
  if (!h.base) return MSZ_OK;
  for (int i = 0; i < nf; ++i) {
    if (!geom_from(ndim[i], dims + 3 * i, E->geoms[i])) return MSZ_ERR_ARG;
    if (dtype[i] != MSZ_F32 && dtype[i] != MSZ_F64) return MSZ_ERR_DTYPE;
    E->dtypes[i] = dtype[i];
    E->bufs[i] = FieldBufs{};
  }
  assign_members(E, nullptr, E->nf);
  return MSZ_OK;
}

int check_shapes(int nf, const int* ndim, const int64_t* dims, const int* dtype) {
  if (nf < 1 || !ndim || !dims || !dtype) return MSZ_ERR_ARG;
  for (int i = 0; i < nf; ++i) {
    Geom G;
    if (!geom_from(ndim[i], dims + 3 * i, G)) return MSZ_ERR_ARG;
    if (dtype[i] != MSZ_F32 && dtype[i] != MSZ_F64) return MSZ_ERR_DTYPE;
  }
  return MSZ_OK;
}

// Creates an engine that owns its device memory (plans, batches).
int create_engine(msz_engine_s** out, int nf, const int* ndim, const int64_t* dims, const int* dtype,
                  const msz_options* opt) {
  *out = nullptr;
  int rc = check_shapes(nf, ndim, dims, dtype);
  if (rc != MSZ_OK) return rc;
  msz_engine_s* E = new (std::nothrow) msz_engine_s();
  if (!E) return MSZ_ERR_OOM;
  if (cudaGetDevice(&E->device) != cudaSuccess) {  // no device or driver: not a memory shortage
    cudaGetLastError();
    delete E;
    return MSZ_ERR_CUDA;
  }
  if (opt) E->opt = *opt;
  HostArena measure{nullptr, 0, 0};
  host_engine(E, nf, ndim, dims, dtype, measure);
  E->host_mem = new (std::nothrow) unsigned char[measure.off + 64];
  if (!E->host_mem) {
    delete E;
    return MSZ_ERR_OOM;
  }
  const size_t shift = (64 - (reinterpret_cast<uintptr_t>(E->host_mem) & 63)) & 63;
  HostArena h{E->host_mem + shift, measure.off, 0};
  rc = host_engine(E, nf, ndim, dims, dtype, h);
  if (rc != MSZ_OK) {
    free_engine(E);
    return rc;
  }
  E->block_bytes = layout_engine(E, nullptr, true);
  if (cudaMalloc(&E->block, E->block_bytes) != cudaSuccess) {
    cudaGetLastError();
    E->block = nullptr;
    free_engine(E);
    return MSZ_ERR_OOM;
  }
  layout_engine(E, static_cast<unsigned char*>(E->block), true);
  bool ok = cudaMallocHost((void**)&E->h_states, sizeof(DevState) * nf) == cudaSuccess;
  E->h_states_pinned = ok;
  ok = ok && cudaEventCreate(&E->ev0) == cudaSuccess && cudaEventCreate(&E->ev1) == cudaSuccess;
  // flags padding beyond N must be zero once (the kernels clear [0, N) each run)
  if (ok) {
    for (int i = 0; i < nf; ++i)
      if (cudaMemset(E->bufs[i].flags, 0, (size_t)emit_tiles(E->geoms[i]) * kEmitTile) != cudaSuccess) ok = false;
  }
  if (!ok) {
    cudaGetLastError();
    free_engine(E);
    return MSZ_ERR_OOM;
  }
  if (setup_groups(E) != MSZ_OK) {
    free_engine(E);
    return MSZ_ERR_CUDA;
  }
  E->use_graph = !(E->opt.flags & MSZ_OPT_TIME_KERNELS);
  *out = E;
  return MSZ_OK;
}

// Device bytes an engine of these fields allocates.
int64_t engine_bytes(int nf, const int* ndim, const int64_t* dims, const int* dtype) {
  const int rc = check_shapes(nf, ndim, dims, dtype);
  if (rc != MSZ_OK) return rc;
  msz_engine_s E;
  HostArena measure{nullptr, 0, 0};
  host_engine(&E, nf, ndim, dims, dtype, measure);
  unsigned char* mem = new (std::nothrow) unsigned char[measure.off + 64];
  if (!mem) return MSZ_ERR_OOM;
  const size_t shift = (64 - (reinterpret_cast<uintptr_t>(mem) & 63)) & 63;
  HostArena h{mem + shift, measure.off, 0};
  host_engine(&E, nf, ndim, dims, dtype, h);
  const int64_t bytes = (int64_t)layout_engine(&E, nullptr, true);
  delete[] mem;
  return bytes;
}

// Issues `steps` steps of every group on stream s (also inside a stream
// capture). The groups' fields are disjoint and every kernel touches only its
// own group's fields, so with several groups each runs its steps on a stream
// of its own, forked from s and joined back into it: one group's latency-bound
// rounds no longer wait behind another's.
int nonempty_groups(msz_engine_s* E) {
  int ng = 0;
  E->each_group([&](auto& g) { ng += g.empty() ? 0 : 1; });
  return ng;
}

// The streams and events that issue_steps forks onto (created outside any
// stream capture).
int ensure_group_streams(msz_engine_s* E) {
  const int ng = nonempty_groups(E);
  if (ng <= 1) return MSZ_OK;
  if (!E->fork_ev && cudaEventCreateWithFlags(&E->fork_ev, cudaEventDisableTiming) != cudaSuccess)
    return MSZ_ERR_CUDA;
  for (int k = 0; k < ng - 1; ++k) {
    if (!E->grp_stream[k] && cudaStreamCreateWithFlags(&E->grp_stream[k], cudaStreamNonBlocking) != cudaSuccess)
      return MSZ_ERR_CUDA;
    if (!E->join_ev[k] && cudaEventCreateWithFlags(&E->join_ev[k], cudaEventDisableTiming) != cudaSuccess)
      return MSZ_ERR_CUDA;
  }
  return MSZ_OK;
}

int issue_steps(msz_engine_s* E, cudaStream_t s, int steps, int jumps) {
  const int ng = nonempty_groups(E);
  if (ng <= 1) {
    for (int i = 0; i < steps; ++i) E->each_group([&](auto& g) { g.step(s, jumps); });
    return MSZ_OK;
  }
  if (!E->fork_ev) return MSZ_ERR_CUDA;  // ensure_group_streams not called
  if (cudaEventRecord(E->fork_ev, s) != cudaSuccess) return MSZ_ERR_CUDA;
  int k = 0, rc = MSZ_OK;
  E->each_group([&](auto& g) {
    if (g.empty() || rc != MSZ_OK) return;
    cudaStream_t gs = (k == 0) ? s : E->grp_stream[k - 1];
    if (k > 0 && cudaStreamWaitEvent(gs, E->fork_ev, 0) != cudaSuccess) rc = MSZ_ERR_CUDA;
    for (int i = 0; i < steps; ++i) g.step(gs, jumps);
    if (k > 0 && cudaEventRecord(E->join_ev[k - 1], gs) != cudaSuccess) rc = MSZ_ERR_CUDA;
    ++k;
  });
  for (int j = 0; j < k - 1 && rc == MSZ_OK; ++j)
    if (cudaStreamWaitEvent(s, E->join_ev[j], 0) != cudaSuccess) rc = MSZ_ERR_CUDA;
  return rc;
}

// Timed runs keep kJumpsPerStep jump launches per step (the slot table of
// the per-kernel statistics; single-field engines).
int launch_steps(msz_engine_s* E, cudaStream_t s, int steps, bool timed) {
  const int jumps = timed ? kJumpsPerStep : E->tune.jumps_per_step;
  E->launches += (uint64_t)steps * E->launches_per_step(jumps);
  if (!timed) return ensure_group_streams(E) == MSZ_OK ? issue_steps(E, s, steps, jumps) : MSZ_ERR_CUDA;
  for (int i = 0; i < steps; ++i) {
    cudaEvent_t* e = E->tev[i];
    E->each_group([&](auto& g) { g.step(s, jumps, e, E->d_steplog, i); });
  }
  return MSZ_OK;
}

// Per-launch device times of a timed chunk, split into launches that did work
// for the field (bit set in the step log) and the rest.
void collect_times(msz_engine_s* E, int steps) {
  for (int i = 0; i < steps; ++i) {
    cudaEvent_t* e = E->tev[i];
    for (int k = 0; k < kStepSlots; ++k) {
      float dt = 0.f;
      cudaEventElapsedTime(&dt, e[k], e[k + 1]);
      const int kid = kSlotKernel[k];
      E->ks_launches[kid]++;
      E->ks_ms[kid] += dt;
      if ((E->h_steplog[i] >> k) & 1u) {
        E->ks_work[kid]++;
        E->ks_work_ms[kid] += dt;
      }
      const int kind = (kid == KID_SWEEP || kid == KID_RECLASS)         ? 0
                       : (kid == KID_GATHER || kid == KID_MARK || kid == KID_APPLY || kid == KID_CSMALL) ? 3
                       : (kid == KID_RCHECK)                             ? 2
                                                                         : 1;  // label stages
      E->kernel_ms[kind] += dt;
    }
  }
}

// Captures tune.graph_steps steps of every group once (on a private stream). Each
// step launches every kernel; a kernel whose fields are all in other stages
// returns at once (about a microsecond in a graph).
int ensure_graph(msz_engine_s* E) {
  if (E->graph) return MSZ_OK;
  if (!E->cap_stream && cudaStreamCreateWithFlags(&E->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return MSZ_ERR_CUDA;
  cudaGraph_t gr = nullptr;
  if (ensure_group_streams(E) != MSZ_OK) return MSZ_ERR_CUDA;
  if (cudaStreamBeginCapture(E->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return MSZ_ERR_CUDA;
  const int irc = issue_steps(E, E->cap_stream, E->tune.graph_steps, E->tune.jumps_per_step);
  const cudaError_t ce = cudaStreamEndCapture(E->cap_stream, &gr);
  if (irc != MSZ_OK || ce != cudaSuccess) {
    if (gr) cudaGraphDestroy(gr);
    return MSZ_ERR_CUDA;
  }
  const cudaError_t r = cudaGraphInstantiate(&E->graph, gr, 0);
  cudaGraphDestroy(gr);
  return r == cudaSuccess ? MSZ_OK : MSZ_ERR_CUDA;
}

// Runs every field of the engine to completion. f / fhat / xi are indexed
// by engine field. Fills one msz_result per field (out may be null).
int run_engine(msz_engine_s* E, const void* const* f, const void* const* fhat, const double* xi, cudaStream_t s,
               msz_result* out) {
  const int nf = E->nf;
  for (int i = 0; i < nf; ++i) {
    if (!f[i] || !fhat[i] || !xi_ok(xi[i], E->dtypes[i])) return MSZ_ERR_ARG;
  }
  int rc = MSZ_OK;
  E->each_group([&](auto& g) {
    if (rc == MSZ_OK && !g.empty()) rc = g.upload(f, fhat, xi, s);
  });
  if (rc != MSZ_OK) return rc;
  DevState* H = E->h_states;
  const bool parked = (E->opt.flags & MSZ_OPT_TEST_STALL) != 0;
  for (int i = 0; i < nf; ++i) {
    std::memset(&H[i], 0, sizeof(DevState));
    H[i].phase = parked ? PH_PARKED : PH_INIT;
    H[i].max_rounds = E->opt.max_rounds ? E->opt.max_rounds : 10000000ull;
  }
  if (cudaMemcpyAsync(E->d_states, H, sizeof(DevState) * nf, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return MSZ_ERR_CUDA;
  if (E->ev0) cudaEventRecord(E->ev0, s);
  E->launches = 0;
  E->each_group([&](auto& g) { g.init(s); });
  E->each_group([&](auto& g) { E->launches += g.empty() ? 0 : 1; });
  const bool timed = (E->opt.flags & MSZ_OPT_TIME_KERNELS) != 0;
  if (timed && !E->tev_ready) {
    for (int i = 0; i < kMaxChunk; ++i)
      for (int j = 0; j < kStepEvents; ++j) cudaEventCreate(&E->tev[i][j]);
    E->tev_ready = true;
  }
  for (int k = 0; k < kKinds; ++k) E->kernel_ms[k] = 0.0;
  for (int k = 0; k < NKID; ++k) {
    E->ks_launches[k] = E->ks_work[k] = E->ks_units[k] = 0;
    E->ks_ms[k] = E->ks_work_ms[k] = 0.0;
  }
  if (timed && cudaMemsetAsync(E->d_steplog, 0, sizeof(uint32_t) * kMaxChunk, s) != cudaSuccess) return MSZ_ERR_CUDA;
  const bool graph = E->use_graph && !timed && ensure_graph(E) == MSZ_OK;
  // Steps in growing chunks; one state read per chunk. A chunk in which no
  // field's state machine moved means a stall.
  int chunk = 1;
  uint64_t last_ticks = ~0ull;
  const int gsteps = E->tune.graph_steps;
  for (;;) {
    if (graph) {
      for (int i = 0; i < chunk; ++i) cudaGraphLaunch(E->graph, s);
      E->launches += (uint64_t)chunk * gsteps * E->launches_per_step(E->tune.jumps_per_step);
    } else {
      if (launch_steps(E, s, std::min(chunk * gsteps, kMaxChunk), timed) != MSZ_OK) return MSZ_ERR_CUDA;
    }
    if (cudaMemcpyAsync(H, E->d_states, sizeof(DevState) * nf, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return MSZ_ERR_CUDA;
    if (timed && (cudaMemcpyAsync(E->h_steplog, E->d_steplog, sizeof(uint32_t) * kMaxChunk, cudaMemcpyDeviceToHost,
                                  s) != cudaSuccess ||
                  cudaMemsetAsync(E->d_steplog, 0, sizeof(uint32_t) * kMaxChunk, s) != cudaSuccess))
      return MSZ_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MSZ_ERR_CUDA;
    if (timed) collect_times(E, std::min(chunk * gsteps, kMaxChunk));
    bool all = true;
    uint64_t ticks = 0;
    for (int i = 0; i < nf; ++i) {
      all = all && (H[i].phase == PH_DONE || H[i].phase == PH_ERR);
      ticks += H[i].ticks;
    }
    if (all) break;
    if (ticks == last_ticks) {
      // no state machine moved in a whole chunk: report the stalled fields
      for (int i = 0; i < nf; ++i)
        if (H[i].phase != PH_DONE && H[i].phase != PH_ERR) {
          H[i].phase = PH_ERR;
          H[i].status = MSZ_ERR_TIMEOUT;
        }
      cudaMemcpyAsync(E->d_states, H, sizeof(DevState) * nf, cudaMemcpyHostToDevice, s);
      break;
    }
    last_ticks = ticks;
    chunk = std::max(1, std::min(chunk * 2, kMaxChunk / gsteps));
  }
  E->each_group([&](auto& g) { g.emit(s); });
  E->each_group([&](auto& g) { E->launches += g.empty() ? 0ull : 3ull; });
  if (E->ev1) cudaEventRecord(E->ev1, s);
  if (cudaMemcpyAsync(H, E->d_states, sizeof(DevState) * nf, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return MSZ_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MSZ_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess) return MSZ_ERR_CUDA;
  if (timed && nf == 1) {
    for (int k = 0; k < NKID; ++k) E->ks_units[k] = H[0].kunits[k];
    E->ks_units[KID_SWEEP] = (uint64_t)E->geoms[0].n * E->ks_work[KID_SWEEP];

  }
  float ms = 0.f;
  if (E->ev0 && E->ev1 && cudaEventElapsedTime(&ms, E->ev0, E->ev1) != cudaSuccess) ms = 0.f;
  int worst = MSZ_OK;
  for (int i = 0; i < nf; ++i) {
    int st = (H[i].phase == PH_DONE) ? MSZ_OK : (H[i].status ? H[i].status : MSZ_ERR_CUDA);
    if (H[i].err_bits & E_CHECK) st = MSZ_ERR_CHECK;  // a bounds check of the checked build fired
    if (st != MSZ_OK && worst == MSZ_OK) worst = st;
    if (!out) continue;
    msz_result& R = out[i];
    std::memset(&R, 0, sizeof(R));
    R.status = st;
    R.counts = H[i].cnt;
    if (st == MSZ_OK || (st == MSZ_ERR_NOCONVERGE && H[i].emitted)) {
      R.edit_idx = E->bufs[i].edit_idx;
      R.edit_val = E->bufs[i].edit_val;
      R.n_edits = H[i].n_edits;
    }
    if (st == MSZ_OK) {
      R.label_max = E->bufs[i].Pup;
      R.label_min = E->bufs[i].Pdn;
    }
    R.device_ms = ms;
    R.launches = E->launches;
    for (int k = 0; k < kKinds; ++k) R.kernel_ms[k] = (float)E->kernel_ms[k];
  }
  return worst;
}

// Applies launch parameters to an engine that owns its fields (plans,
// batches): group grids and sweep tiling are recomputed, and the step graph
// is captured again at the next fix.
int set_tuning(msz_engine_s* E, const msz_tuning& t) {
  if (!tuning_ok(t)) return MSZ_ERR_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return MSZ_ERR_CUDA;  // no fix of this engine in flight
  E->tune = t;
  if (E->graph) {
    cudaGraphExecDestroy(E->graph);
    E->graph = nullptr;
  }
  return setup_groups(E) == MSZ_OK ? MSZ_OK : MSZ_ERR_CUDA;
}

// Device time of one whole fix of every field under the engine's current
// launch parameters: the faster of two runs after one that captures the
// step graph (ev0 .. ev1 of run_engine).
int time_engine(msz_engine_s* E, const void* const* f, const void* const* fhat, const double* xi, cudaStream_t s,
                float* ms) {
  float best = 0.f;
  for (int r = 0; r < 3; ++r) {
    const int rc = run_engine(E, f, fhat, xi, s, nullptr);
    if (rc != MSZ_OK) return rc;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, E->ev0, E->ev1) != cudaSuccess) return MSZ_ERR_CUDA;
    if (r > 0 && (r == 1 || t < best)) best = t;
  }
  *ms = best;
  return MSZ_OK;
}

// Tuned settings of this process, by batch signature.
std::mutex g_tune_mu;
std::vector<std::pair<std::vector<int64_t>, msz_tuning>> g_tune_cache;

// Per field: dtype, dimension and log2 of the vertex count, sorted.
std::vector<int64_t> tune_signature(const msz_engine_s* E) {
  std::vector<int64_t> sig;
  for (int i = 0; i < E->nf; ++i) {
    int lg = 0;
    while ((1ll << (lg + 1)) <= (int64_t)E->geoms[i].n) ++lg;
    sig.push_back(((int64_t)E->dtypes[i] << 40) | ((int64_t)E->geoms[i].nd << 32) | lg);
  }
  std::sort(sig.begin(), sig.end());
  return sig;
}

// Coordinate descent over the launch parameters (see msz_batch_autotune).
int autotune(msz_engine_s* E, const void* const* f, const void* const* fhat, const double* xi, bool force,
             cudaStream_t s, msz_tuning* out, int* tried) {
  if (tried) *tried = 0;
  const std::vector<int64_t> sig = tune_signature(E);
  if (!force) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto& c : g_tune_cache)
      if (c.first == sig) {
        *out = c.second;
        return set_tuning(E, c.second);
      }
  }
  msz_tuning best = E->tune;
  float t_best = 0.f;
  int rc = time_engine(E, f, fhat, xi, s, &t_best);
  if (rc != MSZ_OK) return rc;
  int n = 1;
  struct Knob {
    int32_t msz_tuning::*field;
    std::vector<int32_t> values;
  };
  const std::vector<Knob> knobs = {
      {&msz_tuning::small_rounds, {0, 16, 64, 256}},
      {&msz_tuning::small_cases, {4096, 16384, (int32_t)kSmallCases}},
      {&msz_tuning::graph_steps, {2, 4, 8}},
      {&msz_tuning::jumps_per_step, {1, 2, 3}},
      {&msz_tuning::chase_steps, {16, 32, 64}},
      {&msz_tuning::sweep_chunk, {16, 32, 64}},
      {&msz_tuning::blocks_per_sm, {0, 2, 4}},
  };
  for (const Knob& k : knobs) {
    for (const int32_t v : k.values) {
      if (best.*(k.field) == v) continue;
      msz_tuning cand = best;
      cand.*(k.field) = v;
      if (!tuning_ok(cand)) continue;
      if ((rc = set_tuning(E, cand)) != MSZ_OK) return rc;
      float t = 0.f;
      if ((rc = time_engine(E, f, fhat, xi, s, &t)) != MSZ_OK) return rc;
      ++n;
      if (t < 0.98f * t_best) {
        best = cand;
        t_best = t;
      }
    }
  }
  if ((rc = set_tuning(E, best)) != MSZ_OK) return rc;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    bool found = false;
    for (auto& c : g_tune_cache)
      if (c.first == sig) {
        c.second = best;
        found = true;
      }
    if (!found) g_tune_cache.emplace_back(sig, best);
  }
  *out = best;
  if (tried) *tried = n;
  return MSZ_OK;
}

}  // namespace
}  // namespace msz

// A plan is an engine of one field.
struct msz_plan_s {
  msz_engine_s* E;
};
struct msz_batch_s {
  msz_engine_s* E;
  bool tuned = false;  // msz_batch_autotune has run on it
};

extern "C" {

int64_t msz_plan_bytes(int ndim, const int64_t dims[3], int dtype) {
  if (!dims) return MSZ_ERR_ARG;
  return engine_bytes(1, &ndim, dims, &dtype);
}

int msz_plan_create(msz_plan* out, int ndim, const int64_t dims[3], int dtype, const msz_options* opt) {
  if (!out) return MSZ_ERR_ARG;
  *out = nullptr;
  if (!dims) return MSZ_ERR_ARG;
  msz_engine_s* E = nullptr;
  const int rc = create_engine(&E, 1, &ndim, dims, &dtype, opt);
  if (rc != MSZ_OK) return rc;
  msz_plan_s* p = new (std::nothrow) msz_plan_s{E};
  if (!p) {
    free_engine(E);
    return MSZ_ERR_OOM;
  }
  *out = p;
  return MSZ_OK;
}

int msz_plan_destroy(msz_plan p) {
  if (!p) return MSZ_ERR_ARG;
  cudaDeviceSynchronize();
  free_engine(p->E);
  delete p;
  return MSZ_OK;
}

int msz_plan_kernel_stats(msz_plan p, msz_kernel_stat* out, int n) {
  if (!p || !out || n < 0 || !(p->E->opt.flags & MSZ_OPT_TIME_KERNELS)) return MSZ_ERR_ARG;
  const msz_engine_s* E = p->E;
  const int m = std::min(n, (int)NKID);
  for (int k = 0; k < m; ++k) {
    out[k].name = kKernelNames[k];
    out[k].launches = E->ks_launches[k];
    out[k].work_launches = E->ks_work[k];
    out[k].ms = E->ks_ms[k];
    out[k].work_ms = E->ks_work_ms[k];
    out[k].units = E->ks_units[k];
  }
  return m;
}

int msz_fix(msz_plan p, const void* orig_dev, const void* decomp_dev, double xi, void* stream, msz_result* out) {
  if (out) std::memset(out, 0, sizeof(*out));
  auto fail = [&](int code) {
    if (out) out->status = code;
    return code;
  };
  if (!p || !orig_dev || !decomp_dev) return fail(MSZ_ERR_ARG);
  if (!xi_ok(xi, p->E->dtypes[0])) return fail(MSZ_ERR_ARG);
  msz_result r;
  const int st = run_engine(p->E, &orig_dev, &decomp_dev, &xi, static_cast<cudaStream_t>(stream), &r);
  if (out) {
    *out = r;
    out->status = st;
  }
  return st;
}

int msz_fix_host(msz_plan p, const void* orig_host, const void* decomp_host, double xi, uint32_t* edit_idx_host,
                 void* edit_val_host, int32_t* label_max_host, int32_t* label_min_host, void* stream,
                 msz_result* out) {
  if (out) std::memset(out, 0, sizeof(*out));
  if (!p || !orig_host || !decomp_host || !edit_idx_host || !edit_val_host) return MSZ_ERR_ARG;
  msz_engine_s* E = p->E;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Geom& G = E->geoms[0];
  const size_t bytes = (size_t)G.n * esize(E->dtypes[0]);
  if (!E->in_f || !E->in_fhat) {
    if ((!E->in_f && cudaMalloc(&E->in_f, bytes) != cudaSuccess) ||
        (!E->in_fhat && cudaMalloc(&E->in_fhat, bytes) != cudaSuccess)) {
      cudaGetLastError();
      return MSZ_ERR_OOM;
    }
  }
  if (cudaMemcpyAsync(E->in_f, orig_host, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(E->in_fhat, decomp_host, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return MSZ_ERR_CUDA;
  msz_result r;
  const int st = msz_fix(p, E->in_f, E->in_fhat, xi, stream, &r);
  if (st != MSZ_OK) {
    if (out) *out = r;
    return st;
  }
  const size_t ne = (size_t)r.n_edits;
  if (ne) {
    if (cudaMemcpyAsync(edit_idx_host, r.edit_idx, ne * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(edit_val_host, r.edit_val, ne * esize(E->dtypes[0]), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess)
      return MSZ_ERR_CUDA;
  }
  if (label_max_host) cudaMemcpyAsync(label_max_host, r.label_max, (size_t)G.n * 4, cudaMemcpyDeviceToHost, s);
  if (label_min_host) cudaMemcpyAsync(label_min_host, r.label_min, (size_t)G.n * 4, cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return MSZ_ERR_CUDA;
  if (out) {
    *out = r;
    out->edit_idx = edit_idx_host;
    out->edit_val = edit_val_host;
    out->label_max = label_max_host;
    out->label_min = label_min_host;
  }
  return MSZ_OK;
}

// ---------------------------------------------------------------------------
// Batches
// ---------------------------------------------------------------------------
int64_t msz_batch_bytes(int n, const int* ndim, const int64_t* dims, const int* dtype) {
  return engine_bytes(n, ndim, dims, dtype);
}

int msz_batch_create(msz_batch* out, int n, const int* ndim, const int64_t* dims, const int* dtype,
                     const msz_options* opt) {
  if (!out || n < 1 || !ndim || !dims || !dtype) return MSZ_ERR_ARG;
  *out = nullptr;
  msz_engine_s* E = nullptr;
  const int rc = create_engine(&E, n, ndim, dims, dtype, opt);
  if (rc != MSZ_OK) return rc;
  msz_batch_s* b = new (std::nothrow) msz_batch_s{E, false};
  if (!b) {
    free_engine(E);
    return MSZ_ERR_OOM;
  }
  *out = b;
  return MSZ_OK;
}

int msz_batch_fix(msz_batch b, const void* const* orig_dev, const void* const* decomp_dev, const double* xi,
                  void* stream, msz_result* results) {
  if (!b || !orig_dev || !decomp_dev || !xi) return MSZ_ERR_ARG;
  if (b->E->opt.autotune && !b->tuned) {
    msz_tuning t;
    const int rc = msz_batch_autotune(b, orig_dev, decomp_dev, xi, 0, stream, &t, nullptr);
    if (rc != MSZ_OK) return rc;
  }
  return run_engine(b->E, orig_dev, decomp_dev, xi, static_cast<cudaStream_t>(stream), results);
}

void msz_tuning_default(msz_tuning* t) {
  if (t) *t = kDefaultTuning;
}

int msz_tuning_valid(const msz_tuning* t) { return (t && tuning_ok(*t)) ? MSZ_OK : MSZ_ERR_ARG; }

int msz_batch_set_tuning(msz_batch b, const msz_tuning* t) {
  if (!b || !t) return MSZ_ERR_ARG;
  return set_tuning(b->E, *t);
}

int msz_batch_get_tuning(msz_batch b, msz_tuning* t) {
  if (!b || !t) return MSZ_ERR_ARG;
  *t = b->E->tune;
  return MSZ_OK;
}

int msz_plan_set_tuning(msz_plan p, const msz_tuning* t) {
  if (!p || !t) return MSZ_ERR_ARG;
  return set_tuning(p->E, *t);
}

int msz_plan_get_tuning(msz_plan p, msz_tuning* t) {
  if (!p || !t) return MSZ_ERR_ARG;
  *t = p->E->tune;
  return MSZ_OK;
}

int msz_batch_autotune(msz_batch b, const void* const* orig_dev, const void* const* decomp_dev, const double* xi,
                       int force, void* stream, msz_tuning* out, int* tried) {
  if (!b || !orig_dev || !decomp_dev || !xi || !out) return MSZ_ERR_ARG;
  const int rc = autotune(b->E, orig_dev, decomp_dev, xi, force != 0, static_cast<cudaStream_t>(stream), out, tried);
  if (rc == MSZ_OK) b->tuned = true;
  return rc;
}

int msz_batch_destroy(msz_batch b) {
  if (!b) return MSZ_ERR_ARG;
  cudaDeviceSynchronize();
  free_engine(b->E);
  delete b;
  return MSZ_OK;
}

// ---------------------------------------------------------------------------
// Standalone kernels
// ---------------------------------------------------------------------------
int msz_apply(void* decomp_dev, int ndim, const int64_t dims[3], int dtype, const uint32_t* edit_idx_dev,
              const void* edit_val_dev, uint64_t n_edits, void* stream) {
  Geom G;
  if (!geom_from(ndim, dims, G)) return MSZ_ERR_ARG;
  if (dtype != MSZ_F32 && dtype != MSZ_F64) return MSZ_ERR_DTYPE;
  if (n_edits == 0) return MSZ_OK;
  if (!decomp_dev || !edit_idx_dev || !edit_val_dev) return MSZ_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t* bad = nullptr;
  if (cudaMallocAsync((void**)&bad, sizeof(uint32_t), s) != cudaSuccess) return MSZ_ERR_OOM;
  cudaMemsetAsync(bad, 0, sizeof(uint32_t), s);
  const int blocks =
      (int)std::max<uint64_t>(1, std::min<uint64_t>((n_edits + kThreads - 1) / kThreads, (uint64_t)num_sms() * 8));
  if (dtype == MSZ_F32)
    k_scatter<float><<<blocks, kThreads, 0, s>>>(static_cast<float*>(decomp_dev), G.n, edit_idx_dev,
                                                 static_cast<const float*>(edit_val_dev), n_edits, bad);
  else
    k_scatter<double><<<blocks, kThreads, 0, s>>>(static_cast<double*>(decomp_dev), G.n, edit_idx_dev,
                                                  static_cast<const double*>(edit_val_dev), n_edits, bad);
  uint32_t h = 0;
  cudaMemcpyAsync(&h, bad, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(bad, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return MSZ_ERR_CUDA;
  return h ? MSZ_ERR_ARG : MSZ_OK;
}

int msz_directions(const void* field_dev, int ndim, const int64_t dims[3], int dtype, uint8_t* dir_dev,
                   void* stream) {
  Geom G;
  if (!geom_from(ndim, dims, G)) return MSZ_ERR_ARG;
  if (dtype != MSZ_F32 && dtype != MSZ_F64) return MSZ_ERR_DTYPE;
  if (!field_dev || !dir_dev) return MSZ_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks =
      (int)std::max<int64_t>(1, std::min<int64_t>((G.n + kThreads - 1) / kThreads, (int64_t)num_sms() * 8));
  if (dtype == MSZ_F32) {
    if (ndim == 3) k_directions<float, 3><<<blocks, kThreads, 0, s>>>(static_cast<const float*>(field_dev), G, dir_dev);
    else k_directions<float, 2><<<blocks, kThreads, 0, s>>>(static_cast<const float*>(field_dev), G, dir_dev);
  } else {
    if (ndim == 3) k_directions<double, 3><<<blocks, kThreads, 0, s>>>(static_cast<const double*>(field_dev), G, dir_dev);
    else k_directions<double, 2><<<blocks, kThreads, 0, s>>>(static_cast<const double*>(field_dev), G, dir_dev);
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return MSZ_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? MSZ_OK : MSZ_ERR_CUDA;
}

const char* msz_strerror(int status) {
  switch (status) {
    case MSZ_OK: return "ok";
    case MSZ_ERR_ARG: return "invalid argument";
    case MSZ_ERR_DTYPE: return "unsupported dtype";
    case MSZ_ERR_NONFINITE: return "non-finite input value";
    case MSZ_ERR_BOUND: return "decompressed value outside the error bound";
    case MSZ_ERR_OOM: return "out of memory";
    case MSZ_ERR_NOCONVERGE: return "round cap reached";
    case MSZ_ERR_TIMEOUT: return "device-side wait gave up";
    case MSZ_ERR_CUDA: return "CUDA runtime error";
    case MSZ_ERR_BUSY: return "no free slot or request not ready";
    case MSZ_ERR_TOO_LARGE: return "field too large for the static scratch of msz_fix_noalloc";
    case MSZ_ERR_CANCELLED: return "request cancelled";
    case MSZ_ERR_CHECK: return "bounds check failed (checked build)";
    default: return "unknown status";
  }
}

const char* msz_version(void) { return "msz-gb300 0.2"; }

}  // extern "C"

// ---------------------------------------------------------------------------
// msz_fix_noalloc: the correction loop with no device allocation at all.
//
// Some callers cannot call cudaMalloc: code that runs where the allocator is
// owned by someone else (a framework's caching allocator or a memory pool
// that must not grow, a real-time loop where an allocation may block or fail,
// a plugin whose host forbids allocations during a call). For them this
// entry point keeps every intermediate array of the loop in one file-scope
// device array of fixed size, kNoAllocScratchBytes, which every GPU that
// loads the library holds until the process exits. Inputs and outputs are
// still the caller's buffers.
//
// In host code g_noalloc_scratch names a host-side stand-in, not the device
// array: its device address is obtained with cudaGetSymbolAddress, once per
// device, by the first call on that device (with that device current). That
// first call should therefore come before any stream capture.
//
// Every call shares the array and finds the previous call's contents in it;
// the loop clears what must start at zero (state, flags) itself. Calls whose
// work overlaps on the GPU (different streams, or different host threads on
// one device) race on the array and must be serialised by the caller.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;  // 64 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};
unsigned long long g_noalloc_ctx[kMaxDevices] = {};  // context the address belongs to

// Unique id of the current CUDA context (driver entry points, looked up
// once), so that an address set up in a context that was since destroyed
// (cudaDeviceReset) is not used in its successor. 0 if unavailable.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);
unsigned long long current_ctx_id() {
  static CtxGetCurrentFn get_cur = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* a = nullptr;
    void* b = nullptr;
    cudaDriverEntryPointQueryResult ra, rb;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &ra) == cudaSuccess &&
        ra == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &rb) == cudaSuccess &&
        rb == cudaDriverEntryPointSuccess) {
      get_cur = reinterpret_cast<CtxGetCurrentFn>(a);
      get_id = reinterpret_cast<CtxGetIdFn>(b);
    }
    cudaGetLastError();
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_cur && get_id && get_cur(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, &id) == CUDA_SUCCESS) return id;
  return 0;
}

// Device address of the scratch array on the current device, set up once per
// device and context.
int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return MSZ_ERR_CUDA;
  }
  // 0 while the runtime has not made a context current yet: then the set-up
  // below runs (the symbol lookup initialises the context) and records it
  const unsigned long long ctx = current_ctx_id();
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev] || ctx == 0 || g_noalloc_ctx[dev] != ctx) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      g_noalloc_ptr[dev] = nullptr;
      return MSZ_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = ptr;
    g_noalloc_ctx[dev] = current_ctx_id();
  }
  *out = g_noalloc_ptr[dev];
  return MSZ_OK;
}

}  // namespace

extern "C" int msz_fix_noalloc(int ndim, const int64_t dims[3], int dtype, const void* orig_dev,
                               const void* decomp_dev, double xi, uint32_t* edit_idx_dev, void* edit_val_dev,
                               int32_t* label_max_dev, int32_t* label_min_dev, void* stream, msz_result* out) {
  if (out) std::memset(out, 0, sizeof(*out));
  auto fail = [&](int code) {
    if (out) out->status = code;
    return code;
  };
  Geom G;
  if (!geom_from(ndim, dims, G)) return fail(MSZ_ERR_ARG);
  if (dtype != MSZ_F32 && dtype != MSZ_F64) return fail(MSZ_ERR_DTYPE);
  if (!orig_dev || !decomp_dev || !edit_idx_dev || !edit_val_dev || !label_max_dev || !label_min_dev)
    return fail(MSZ_ERR_ARG);
  if (!xi_ok(xi, dtype)) return fail(MSZ_ERR_ARG);
  void* base = nullptr;
  int rc = noalloc_scratch(&base);
  if (rc != MSZ_OK) return fail(rc);
  // An engine of one field whose arrays point into the static scratch and the
  // caller's outputs; its host-side arrays and state live on this stack frame.
  msz_engine_s E;
  if (cudaGetDevice(&E.device) != cudaSuccess) {
    cudaGetLastError();
    return fail(MSZ_ERR_CUDA);
  }
  alignas(128) unsigned char host_buf[8192];
  HostArena measure{nullptr, 0, 0};
  host_engine(&E, 1, &ndim, dims, &dtype, measure);
  // the host arrays of one field have a fixed size (no dependence on N):
  // this holds for every shape, and the scratch error is reported if not
  if (measure.off > sizeof(host_buf)) return fail(MSZ_ERR_TOO_LARGE);
  HostArena h{host_buf, sizeof(host_buf), 0};
  rc = host_engine(&E, 1, &ndim, dims, &dtype, h);
  if (rc != MSZ_OK) return fail(rc);
  if (layout_engine(&E, nullptr, false) > kNoAllocScratchBytes) return fail(MSZ_ERR_TOO_LARGE);
  layout_engine(&E, static_cast<unsigned char*>(base), false);
  E.bufs[0].Pup = label_max_dev;
  E.bufs[0].Pdn = label_min_dev;
  E.bufs[0].edit_idx = edit_idx_dev;
  E.bufs[0].edit_val = edit_val_dev;
  DevState host_state;
  E.h_states = &host_state;
  E.use_graph = false;
  if (setup_groups(&E) != MSZ_OK) return fail(MSZ_ERR_CUDA);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(E.bufs[0].flags, 0, (size_t)emit_tiles(G) * kEmitTile, s) != cudaSuccess)
    return fail(MSZ_ERR_CUDA);
  msz_result r;
  const int st = run_engine(&E, &orig_dev, &decomp_dev, &xi, s, &r);
  E.h_states = nullptr;  // the engine owns nothing here
  if (out) {
    *out = r;
    out->status = st;
  }
  return st;
}

// ---------------------------------------------------------------------------
// Serving: continuous batching of independent fields.
//
// A worker thread owns a CUDA stream and a table of slots. Submitted requests
// wait in a queue until a slot is free and their device memory fits the
// budget; they are then admitted into the running set while other fields are
// mid-correction: the group descriptors are rebuilt, the new field starts at
// its init phase, and every later step advances all resident fields together
// (each with its own state machine kept on the device until convergence).
// After each chunk of steps, converged fields get their edit lists emitted
// and leave the running set; their results stay in the slot until released.
// Because every field runs its own state machine on its own buffers, a
// field's result is the same alone and in any mix.
// ---------------------------------------------------------------------------
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>

namespace {

uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct SrvRequest {
  uint64_t id;
  int ndim;
  int64_t dims[3];
  int dtype;
  const void* f;
  const void* fhat;
  double xi;
  uint64_t submit_ns;
};

struct SrvSlot {
  int state = 0;  // 0 free, 1 running, 2 finished (result held), 3 release requested, 4 cancel requested
  uint64_t id = 0;
  void* block = nullptr;
  size_t bytes = 0;
  uint64_t submit_ns = 0, done_ns = 0;
  uint64_t last_ticks = ~0ull;
  int still = 0;  // chunks without a state transition
  msz_result result{};
};

struct SrvDone {  // requests that finished without a slot (rejected)
  int status;
  uint64_t done_ns;
};

}  // namespace

struct msz_server_s {
  msz_engine_s* E = nullptr;  // nf = slots; geoms/dtypes/bufs indexed by slot
  int slots_n = 0;
  int64_t budget = 0, used = 0;
  std::vector<SrvSlot> slots;
  std::vector<const void*> f, fhat;
  std::vector<double> xi;
  std::deque<SrvRequest> queue;
  std::unordered_map<uint64_t, int> where;  // id -> slot
  std::unordered_map<uint64_t, SrvDone> rejected;
  std::mutex mu;
  std::condition_variable cv;
  std::thread worker;
  bool stop = false;
  cudaStream_t stream = nullptr;
  uint64_t next_id = 1;
  unsigned char* dev_block = nullptr;  // states + group descriptors
  int steps_per_chunk = 8;
  uint64_t launches = 0;
};

namespace {

// Group membership from the running slots; re-uploads descriptors.
int srv_rebuild(msz_server_s* S) {
  msz_engine_s* E = S->E;
  std::vector<int> running;
  for (int i = 0; i < S->slots_n; ++i)
    if (S->slots[i].state == 1) running.push_back(i);
  assign_members(E, running.data(), (int)running.size());
  int rc = setup_groups(E);
  if (rc != MSZ_OK) return rc;
  E->each_group([&](auto& g) {
    if (rc == MSZ_OK && !g.empty()) rc = g.upload(S->f.data(), S->fhat.data(), S->xi.data(), S->stream);
  });
  return rc;
}

// Admits queued requests while slots and budget allow (caller holds mu).
bool srv_admit(msz_server_s* S) {
  msz_engine_s* E = S->E;
  bool changed = false;
  while (!S->queue.empty()) {
    const SrvRequest& R = S->queue.front();
    const int64_t need = engine_bytes(1, &R.ndim, R.dims, &R.dtype);
    if (need < 0 || need > S->budget) {  // can never fit
      S->rejected[R.id] = SrvDone{need < 0 ? (int)need : MSZ_ERR_OOM, now_ns()};
      S->queue.pop_front();
      S->cv.notify_all();
      continue;
    }
    if (S->used + need > S->budget) break;
    int slot = -1;
    for (int i = 0; i < S->slots_n; ++i)
      if (S->slots[i].state == 0) {
        slot = i;
        break;
      }
    if (slot < 0) break;
    SrvSlot& sl = S->slots[slot];
    void* block = nullptr;
    if (cudaMallocAsync(&block, (size_t)need, S->stream) != cudaSuccess) {
      cudaGetLastError();
      break;  // retry after other fields leave
    }
    Geom G;
    geom_from(R.ndim, R.dims, G);
    E->geoms[slot] = G;
    E->dtypes[slot] = R.dtype;
    Bump b{static_cast<unsigned char*>(block), 0};
    E->bufs[slot] = FieldBufs{};
    carve_field(b, G, R.dtype, true, E->bufs[slot]);
    cudaMemsetAsync(E->bufs[slot].flags, 0, (size_t)emit_tiles(G) * kEmitTile, S->stream);
    DevState& H = E->h_states[slot];
    std::memset(&H, 0, sizeof(DevState));
    H.phase = (E->opt.flags & MSZ_OPT_TEST_STALL) ? PH_PARKED : PH_INIT;
    H.max_rounds = E->opt.max_rounds ? E->opt.max_rounds : 10000000ull;
    cudaMemcpyAsync(E->d_states + slot, &H, sizeof(DevState), cudaMemcpyHostToDevice, S->stream);
    S->f[slot] = R.f;
    S->fhat[slot] = R.fhat;
    S->xi[slot] = R.xi;
    sl.state = 1;
    sl.id = R.id;
    sl.block = block;
    sl.bytes = (size_t)need;
    sl.submit_ns = R.submit_ns;
    sl.last_ticks = ~0ull;
    sl.still = 0;
    S->used += need;
    S->where[R.id] = slot;
    S->queue.pop_front();
    changed = true;
  }
  return changed;
}

void srv_worker(msz_server_s* S) {
  cudaSetDevice(S->E->device);
  msz_engine_s* E = S->E;
  bool changed = false;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(S->mu);
      // cancelled running fields leave the running set (no kernel is in
      // flight here: every chunk ends with a stream synchronisation)
      for (int i = 0; i < S->slots_n; ++i) {
        SrvSlot& sl = S->slots[i];
        if (sl.state == 4) {
          std::memset(&sl.result, 0, sizeof(sl.result));
          sl.result.status = MSZ_ERR_CANCELLED;
          sl.done_ns = now_ns();
          sl.result.device_ms = (float)((sl.done_ns - sl.submit_ns) * 1e-6);
          sl.state = 2;
          changed = true;
          S->cv.notify_all();
        }
      }
      // free released slots
      for (int i = 0; i < S->slots_n; ++i) {
        SrvSlot& sl = S->slots[i];
        if (sl.state == 3) {
          cudaFreeAsync(sl.block, S->stream);
          S->used -= (int64_t)sl.bytes;
          S->where.erase(sl.id);
          sl = SrvSlot{};
        }
      }
      if (srv_admit(S)) changed = true;
      bool running = false;
      for (int i = 0; i < S->slots_n; ++i) running = running || S->slots[i].state == 1;
      if (!running) {
        if (S->stop) break;
        if (!changed) {
          S->cv.wait_for(lk, std::chrono::milliseconds(2));
          continue;
        }
      }
      if (S->stop && !running) break;
    }
    if (changed) {
      if (srv_rebuild(S) != MSZ_OK) {
        std::lock_guard<std::mutex> lk(S->mu);
        for (int i = 0; i < S->slots_n; ++i)
          if (S->slots[i].state == 1) {
            S->slots[i].state = 2;
            S->slots[i].result.status = MSZ_ERR_CUDA;
            S->slots[i].done_ns = now_ns();
          }
        S->cv.notify_all();
        changed = true;
        continue;
      }
      changed = false;
    }
    // one chunk: init of newly admitted fields, steps, emission of converged ones
    E->each_group([&](auto& g) { g.init(S->stream); });
    const bool issued = ensure_group_streams(E) == MSZ_OK &&
                        issue_steps(E, S->stream, S->steps_per_chunk, E->tune.jumps_per_step) == MSZ_OK;
    E->each_group([&](auto& g) { g.emit(S->stream); });
    S->launches += (uint64_t)S->steps_per_chunk * E->launches_per_step(E->tune.jumps_per_step);
    cudaMemcpyAsync(E->h_states, E->d_states, sizeof(DevState) * S->slots_n, cudaMemcpyDeviceToHost, S->stream);
    const bool ok = cudaStreamSynchronize(S->stream) == cudaSuccess && issued;
    const uint64_t t = now_ns();
    std::lock_guard<std::mutex> lk(S->mu);
    for (int i = 0; i < S->slots_n; ++i) {
      SrvSlot& sl = S->slots[i];
      if (sl.state != 1) continue;
      const DevState& H = E->h_states[i];
      int st = 1;  // still running
      if (!ok) st = MSZ_ERR_CUDA;
      else if (H.phase == PH_DONE && H.emitted) st = MSZ_OK;
      else if (H.phase == PH_ERR) st = H.status ? H.status : MSZ_ERR_CUDA;
      else if (H.ticks == sl.last_ticks && ++sl.still >= 2) st = MSZ_ERR_TIMEOUT;
      if (st != 1 && (H.err_bits & E_CHECK)) st = MSZ_ERR_CHECK;
      if (H.ticks != sl.last_ticks) sl.still = 0;
      sl.last_ticks = H.ticks;
      if (st == 1) continue;
      msz_result& R = sl.result;
      std::memset(&R, 0, sizeof(R));
      R.status = st;
      R.counts = H.cnt;
      if (st == MSZ_OK || (st == MSZ_ERR_NOCONVERGE && H.emitted)) {
        R.edit_idx = E->bufs[i].edit_idx;
        R.edit_val = E->bufs[i].edit_val;
        R.n_edits = H.n_edits;
      }
      if (st == MSZ_OK) {
        R.label_max = E->bufs[i].Pup;
        R.label_min = E->bufs[i].Pdn;
      }
      R.device_ms = (float)((t - sl.submit_ns) * 1e-6);  // submit-to-result latency
      R.launches = S->launches;
      sl.done_ns = t;
      sl.state = 2;
      changed = true;
    }
    S->cv.notify_all();
  }
  // shutdown: free every slot
  for (int i = 0; i < S->slots_n; ++i)
    if (S->slots[i].block) cudaFreeAsync(S->slots[i].block, S->stream);
  cudaStreamSynchronize(S->stream);
}

}  // namespace

extern "C" {

int msz_server_create(msz_server* out, int64_t budget_bytes, int max_slots, const msz_options* opt) {
  if (!out || budget_bytes <= 0 || max_slots < 1 || max_slots > 4096) return MSZ_ERR_ARG;
  *out = nullptr;
  msz_server_s* S = new (std::nothrow) msz_server_s();
  if (!S) return MSZ_ERR_OOM;
  msz_engine_s* E = new (std::nothrow) msz_engine_s();
  if (!E) {
    delete S;
    return MSZ_ERR_OOM;
  }
  S->E = E;
  S->slots_n = max_slots;
  S->budget = budget_bytes;
  S->slots.resize(max_slots);
  S->f.assign(max_slots, nullptr);
  S->fhat.assign(max_slots, nullptr);
  S->xi.assign(max_slots, 0.0);
  cudaGetDevice(&E->device);
  if (opt) E->opt = *opt;
  E->opt.flags &= ~MSZ_OPT_TIME_KERNELS;
  E->nf = max_slots;
  // host arrays with every group sized for all slots
  E->each_group([&](auto& g) { g.nf = max_slots; });
  HostArena measure{nullptr, 0, 0};
  host_layout(E, measure);
  E->host_mem = new (std::nothrow) unsigned char[measure.off + 64];
  int rc = E->host_mem ? MSZ_OK : MSZ_ERR_OOM;
  if (rc == MSZ_OK) {
    const size_t shift = (64 - (reinterpret_cast<uintptr_t>(E->host_mem) & 63)) & 63;
    HostArena h{E->host_mem + shift, measure.off, 0};
    host_layout(E, h);
    for (int i = 0; i < max_slots; ++i) E->bufs[i] = FieldBufs{};
    // device: states and group descriptor arrays for all slots
    Bump mb{nullptr, 0};
    mb.take(sizeof(DevState) * max_slots, 256);
    E->each_group([&](auto& g) { g.carve(mb); });
    if (cudaMalloc((void**)&S->dev_block, mb.off) != cudaSuccess) rc = MSZ_ERR_OOM;
    if (rc == MSZ_OK) {
      Bump b{S->dev_block, 0};
      E->d_states = (DevState*)b.take(sizeof(DevState) * max_slots, 256);
      E->each_group([&](auto& g) { g.carve(b); });
      if (cudaMallocHost((void**)&E->h_states, sizeof(DevState) * max_slots) != cudaSuccess) rc = MSZ_ERR_OOM;
      else E->h_states_pinned = true;
      cudaMemset(E->d_states, 0, sizeof(DevState) * max_slots);
    }
    if (rc == MSZ_OK && cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess) rc = MSZ_ERR_CUDA;
  }
  E->each_group([&](auto& g) { g.nf = 0; });
  if (rc != MSZ_OK) {
    cudaGetLastError();
    if (S->dev_block) cudaFree(S->dev_block);
    if (S->stream) cudaStreamDestroy(S->stream);
    free_engine(E);
    delete S;
    return rc;
  }
  S->worker = std::thread(srv_worker, S);
  *out = S;
  return MSZ_OK;
}

int msz_server_submit(msz_server S, int ndim, const int64_t dims[3], int dtype, const void* orig_dev,
                      const void* decomp_dev, double xi, uint64_t* request_id) {
  if (!S || !dims || !orig_dev || !decomp_dev || !request_id) return MSZ_ERR_ARG;
  Geom G;
  if (!geom_from(ndim, dims, G)) return MSZ_ERR_ARG;
  if (dtype != MSZ_F32 && dtype != MSZ_F64) return MSZ_ERR_DTYPE;
  if (!xi_ok(xi, dtype)) return MSZ_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) return MSZ_ERR_ARG;
  SrvRequest R;
  R.id = S->next_id++;
  R.ndim = ndim;
  R.dims[0] = dims[0];
  R.dims[1] = dims[1];
  R.dims[2] = (ndim == 3) ? dims[2] : 1;
  R.dtype = dtype;
  R.f = orig_dev;
  R.fhat = decomp_dev;
  R.xi = xi;
  R.submit_ns = now_ns();
  S->queue.push_back(R);
  *request_id = R.id;
  S->cv.notify_all();
  return MSZ_OK;
}

int msz_server_poll(msz_server S, uint64_t request_id, int wait_ms, msz_result* out) {
  if (!S || !out) return MSZ_ERR_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  auto ready = [&]() -> int {
    auto rj = S->rejected.find(request_id);
    if (rj != S->rejected.end()) return 1;
    auto it = S->where.find(request_id);
    if (it == S->where.end()) {
      for (const SrvRequest& q : S->queue)
        if (q.id == request_id) return 0;
      return -1;
    }
    return S->slots[it->second].state == 2 ? 1 : 0;
  };
  int r = ready();
  if (r == 0 && wait_ms > 0)
    S->cv.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return ready() != 0; }), r = ready();
  if (r < 0) return MSZ_ERR_ARG;
  if (r == 0) return MSZ_ERR_BUSY;
  auto rj = S->rejected.find(request_id);
  if (rj != S->rejected.end()) {
    std::memset(out, 0, sizeof(*out));
    out->status = rj->second.status;
    return MSZ_OK;
  }
  *out = S->slots[S->where[request_id]].result;
  return MSZ_OK;
}

int msz_server_release(msz_server S, uint64_t request_id) {
  if (!S) return MSZ_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->rejected.erase(request_id)) return MSZ_OK;
  auto it = S->where.find(request_id);
  if (it == S->where.end() || S->slots[it->second].state != 2) return MSZ_ERR_BUSY;
  S->slots[it->second].state = 3;
  S->cv.notify_all();
  return MSZ_OK;
}

int msz_server_cancel(msz_server S, uint64_t request_id) {
  if (!S) return MSZ_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  for (auto q = S->queue.begin(); q != S->queue.end(); ++q)
    if (q->id == request_id) {
      S->queue.erase(q);
      S->rejected[request_id] = SrvDone{MSZ_ERR_CANCELLED, now_ns()};
      S->cv.notify_all();
      return MSZ_OK;
    }
  auto it = S->where.find(request_id);
  if (it == S->where.end()) return S->rejected.count(request_id) ? MSZ_ERR_BUSY : MSZ_ERR_ARG;
  SrvSlot& sl = S->slots[it->second];
  if (sl.state != 1) return MSZ_ERR_BUSY;
  sl.state = 4;
  S->cv.notify_all();
  return MSZ_OK;
}

int msz_server_destroy(msz_server S) {
  if (!S) return MSZ_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->queue.clear();
    for (SrvSlot& sl : S->slots)
      if (sl.state == 1) sl.state = 2;  // abandon running fields
  }
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  if (S->dev_block) cudaFree(S->dev_block);
  if (S->stream) cudaStreamDestroy(S->stream);
  free_engine(S->E);
  delete S;
  return MSZ_OK;
}

}  // extern "C"
