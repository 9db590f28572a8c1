// Work-unit kernels of the MSz correction loop (see msz_engine.cuh).
#pragma once

#include <cooperative_groups.h>
#include "msz_engine.cuh"

namespace msz {

// Asynchronous copy of one element global -> shared (cp.async, cached in
// L1 and L2), and the wait for all of the thread's copies.
template <class T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "element of 4 or 8 bytes");
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  if (sizeof(T) == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int ND>
struct LabelGeom {
  static constexpr int TX = (ND == 3) ? 16 : 64;
  static constexpr int TY = (ND == 3) ? 16 : 32;
  static constexpr int TZ = (ND == 3) ? 16 : 1;
  static constexpr int TV = TX * TY * TZ;  // 4096 (3D) / 2048 (2D) vertices
  static constexpr int SX = TX + 2, SY = TY + 2, SZ = (ND == 3) ? TZ + 2 : 1;
  static constexpr int HALO = SX * SY * SZ;  // < 32768: a pointer and a flag fit in 16 bits
  static constexpr int PER_THREAD = TV / kThreads;
  static constexpr int ROWS = SY * SZ;
  // The halo shell: the halo cells outside the tile (the only cells a path
  // can leave the tile through). In 3D the two end planes (SX * SY cells
  // each), then per inner plane a ring of 2 SX + 2 (SY - 2) cells; in 2D one
  // ring.
  static constexpr int RING = 2 * SX + 2 * (SY - 2);
  static constexpr int SHELL = (ND == 3) ? 2 * SX * SY + TZ * RING : RING;
  static constexpr int SHW = (SHELL + 31) / 32;  // 32-bit words of a shell bitmap
  // The tile's face cells (the tile cells with a neighbour in another tile;
  // every tile exit is one): in 3D the two end planes (TX * TY cells each),
  // then per inner plane a ring of 2 TX + 2 (TY - 2) cells; in 2D one ring.
  static constexpr int PLANE = TX * TY;
  static constexpr int RINGF = 2 * TX + 2 * (TY - 2);
  static constexpr int NFACE = (ND == 3) ? 2 * PLANE + (TZ - 2) * RINGF : RINGF;
  static_assert(HALO <= 0x4000 && TV <= 0x4000, "pointers, indices and the terminal flags share 16 bits");
};

// Face index of the face cell at tile coordinates (lx, ly, lz).
template <int ND>
__host__ __device__ __forceinline__ int face_index(int lx, int ly, int lz) {
  using LG = LabelGeom<ND>;
  int base = 0;
  if (ND == 3) {
    if (lz == 0) return ly * LG::TX + lx;
    if (lz == LG::TZ - 1) return LG::PLANE + ly * LG::TX + lx;
    base = 2 * LG::PLANE + (lz - 1) * LG::RINGF;
  }
  if (ly == 0) return base + lx;
  if (ly == LG::TY - 1) return base + LG::TX + lx;
  return base + 2 * LG::TX + 2 * (ly - 1) + (lx != 0);
}

// Tile coordinates of face cell f (the inverse of face_index).
template <int ND>
__host__ __device__ __forceinline__ void face_cell(int f, int& lx, int& ly, int& lz) {
  using LG = LabelGeom<ND>;
  int q = f;
  lz = 0;
  if (ND == 3) {
    if (f < 2 * LG::PLANE) {
      lz = (f < LG::PLANE) ? 0 : LG::TZ - 1;
      const int r = f - (f < LG::PLANE ? 0 : LG::PLANE);
      ly = r / LG::TX;
      lx = r % LG::TX;
      return;
    }
    const int r = f - 2 * LG::PLANE;
    lz = 1 + r / LG::RINGF;
    q = r - (lz - 1) * LG::RINGF;
  }
  if (q < LG::TX) {
    ly = 0;
    lx = q;
  } else if (q < 2 * LG::TX) {
    ly = LG::TY - 1;
    lx = q - LG::TX;
  } else {
    const int w = q - 2 * LG::TX;
    ly = 1 + (w >> 1);
    lx = (w & 1) * (LG::TX - 1);
  }
}

// Slot of a face vertex in its field's exit tables: its tile's index times
// NFACE plus its face index. A slot depends only on the vertex, so a tile's
// entries stay where they are while other tiles are recomputed.
template <int ND>
__host__ __device__ __forceinline__ uint32_t exit_slot(const Geom& G, int x, int y, int z) {
  using LG = LabelGeom<ND>;
  static_assert((LG::TX & (LG::TX - 1)) == 0 && (LG::TY & (LG::TY - 1)) == 0 && (LG::TZ & (LG::TZ - 1)) == 0,
                "power-of-two tile sides");
  const uint32_t ux = (uint32_t)x, uy = (uint32_t)y, uz = (uint32_t)z;
  const uint32_t tx = ((uint32_t)G.nx + LG::TX - 1) / LG::TX, ty = ((uint32_t)G.ny + LG::TY - 1) / LG::TY;
  const uint32_t tile = ux / LG::TX + tx * (uy / LG::TY + ty * (ND == 3 ? uz / LG::TZ : 0u));
  return tile * (uint32_t)LG::NFACE +
         (uint32_t)face_index<ND>((int)(ux % LG::TX), (int)(uy % LG::TY), ND == 3 ? (int)(uz % LG::TZ) : 0);
}

// The cells of a label tile that one thread owns: cell i = threadIdx.x +
// k kThreads for k < PER_THREAD. kThreads is a multiple of TX, so the thread
// keeps its x and each step moves it by RS = kThreads / TX rows (in 3D a
// whole plane, RS = TY): its halo index is c0 + k HSTEP, its vertex index
// v0 + k VSTEP, with no per-cell index arithmetic.
template <int ND>
struct CellWalk {
  using LG = LabelGeom<ND>;
  static constexpr int RS = kThreads / LG::TX;
  static_assert(kThreads % LG::TX == 0 && (ND == 3 ? RS == LG::TY : RS * LG::PER_THREAD == LG::TY),
                "a thread's cells are whole rows or planes apart");
  static constexpr int HSTEP = (ND == 3) ? LG::SX * LG::SY : RS * LG::SX;
  int lx, r0;  // the thread's x in the tile, its first row
  __device__ __forceinline__ CellWalk() : lx((int)threadIdx.x % LG::TX), r0((int)threadIdx.x / LG::TX) {}
  __device__ __forceinline__ int ly(int k) const { return (ND == 3) ? r0 : r0 + k * RS; }
  __device__ __forceinline__ int lz(int k) const { return (ND == 3) ? k : 0; }
  __device__ __forceinline__ int c0() const { return (lx + 1) + LG::SX * (r0 + 1) + ((ND == 3) ? LG::SX * LG::SY : 0); }
  // vertex index step between the thread's cells
  __device__ __forceinline__ int vstep(const Geom& G) const { return (ND == 3) ? G.nxny : RS * G.nx; }
  // whether step k of the tile at (x0, y0, z0) lies inside the grid
  __device__ __forceinline__ bool inside(const Geom& G, int x0, int y0, int z0, int k) const {
    return x0 + lx < G.nx && y0 + ly(k) < G.ny && z0 + lz(k) < G.nz;
  }
};

// Tile terminals (k_label_tile's output, one 32-bit word per vertex): the
// ascending terminal in the low 16 bits, the descending one in the high 16.
// Every terminal half has kTermFlag set. With kTermExtr also set, the low 14
// bits are the tile cell index (lx + TX (ly + TY lz)) of the extremum inside
// the tile where the vertex's integral line ends; otherwise they are the
// shell index of the halo cell where the line leaves its tile (a tile exit).
// During the pointer doubling an unflagged half is a pointer (halo index).
constexpr uint32_t kTermFlag = 0x8000u;
constexpr uint32_t kTermExtr = 0x4000u;
constexpr uint32_t kTermIdx = 0x3fffu;

// Halo coordinates of shell cell s.
template <int ND>
__host__ __device__ __forceinline__ void shell_cell(int s, int& hx, int& hy, int& hz) {
  using LG = LabelGeom<ND>;
  int q = s;
  hz = 0;
  if (ND == 3) {
    constexpr int P = LG::SX * LG::SY;
    if (s < 2 * P) {
      hz = (s < P) ? 0 : LG::SZ - 1;
      const int r = s - (s < P ? 0 : P);
      hy = r / LG::SX;
      hx = r - hy * LG::SX;
      return;
    }
    const int r = s - 2 * P;
    hz = 1 + r / LG::RING;
    q = r - (hz - 1) * LG::RING;
  }
  if (q < LG::SX) {
    hy = 0;
    hx = q;
  } else if (q < 2 * LG::SX) {
    hy = LG::SY - 1;
    hx = q - LG::SX;
  } else {
    const int w = q - 2 * LG::SX;
    hy = 1 + (w >> 1);
    hx = (w & 1) * (LG::SX - 1);
  }
}

// Shell index of the shell cell at halo coordinates (hx, hy, hz) (the
// inverse of shell_cell).
template <int ND>
__host__ __device__ __forceinline__ int shell_index(int hx, int hy, int hz) {
  using LG = LabelGeom<ND>;
  int base = 0;
  if (ND == 3) {
    constexpr int P = LG::SX * LG::SY;
    if (hz == 0) return hy * LG::SX + hx;
    if (hz == LG::SZ - 1) return P + hy * LG::SX + hx;
    base = 2 * P + (hz - 1) * LG::RING;
  }
  if (hy == 0) return base + hx;
  if (hy == LG::SY - 1) return base + LG::SX + hx;
  return base + 2 * LG::SX + 2 * (hy - 1) + (hx != 0);
}

// Halo coordinates of halo index h.
template <int ND>
__device__ __forceinline__ void halo_cell(int h, int& hx, int& hy, int& hz) {
  using LG = LabelGeom<ND>;
  hx = h % LG::SX;
  const int t = h / LG::SX;
  hy = t % LG::SY;
  hz = t / LG::SY;
}

// Origin (first vertex) of the label tile holding vertex (x, y, z).
template <int ND>
__device__ __forceinline__ void tile_origin_of(int x, int y, int z, int& x0, int& y0, int& z0) {
  using LG = LabelGeom<ND>;
  x0 = x - x % LG::TX;
  y0 = y - y % LG::TY;
  z0 = z - z % LG::TZ;
}

// Global index of the extremum of terminal half t (kTermExtr set) of a
// vertex whose tile starts at (x0, y0, z0): the tile cell index decoded with
// shifts (the tile sides are powers of two).
template <int ND>
__device__ __forceinline__ int extremum_vertex(const Geom& G, uint32_t t, int x0, int y0, int z0) {
  using LG = LabelGeom<ND>;
  static_assert((LG::TX & (LG::TX - 1)) == 0 && (LG::TY & (LG::TY - 1)) == 0, "power-of-two tile sides");
  const int ci = (int)(t & kTermIdx);
  return (x0 + ci % LG::TX) + G.nx * ((y0 + (ci / LG::TX) % LG::TY) + G.ny * (z0 + ci / (LG::TX * LG::TY)));
}

// Exit-table slot of shell cell s of a tile, less the tile's own first slot
// (tile index times NFACE), in a field of tx by ty (by any) label tiles: the
// cell lies in the neighbouring tile a fixed index step away, at a fixed face
// cell of it. Valid for shell cells inside the grid.
template <int ND>
__host__ __device__ __forceinline__ int shell_slot_delta(int s, int tx, int ty) {
  using LG = LabelGeom<ND>;
  int hx, hy, hz;
  shell_cell<ND>(s, hx, hy, hz);
  // halo coordinate h: tile step -1 (h = 0), 0 (1 .. side), +1 (side + 1),
  // and the coordinate within that tile
  auto split = [](int h, int side, int& step, int& l) {
    step = (h == 0) ? -1 : (h == side + 1 ? 1 : 0);
    l = h - 1 - step * side;
  };
  int sx, lx, sy, ly, sz = 0, lz = 0;
  split(hx, LG::TX, sx, lx);
  split(hy, LG::TY, sy, ly);
  if (ND == 3) split(hz, LG::TZ, sz, lz);
  return (sx + tx * (sy + ty * sz)) * LG::NFACE + face_index<ND>(lx, ly, lz);
}

// A block's table of shell_slot_delta for the field of geometry G (filled by
// every thread, then synchronised).
template <int ND>
__device__ __forceinline__ void fill_slot_table(int* tab, const Geom& G) {
  using LG = LabelGeom<ND>;
  const int tx = (G.nx + LG::TX - 1) / LG::TX, ty = (G.ny + LG::TY - 1) / LG::TY;
  for (int s = threadIdx.x; s < LG::SHELL; s += blockDim.x) tab[s] = shell_slot_delta<ND>(s, tx, ty);
}

// Marks every label tile whose tile or one-vertex halo contains vertex u:
// the tiles of u + d for d in {-1,0,1}^d (their terminals must be redone).
template <int ND>
__device__ __forceinline__ void mark_dirty_tiles(uint8_t* tdirty, const Geom& G, int u) {
  using LG = LabelGeom<ND>;
  int x, y, z;
  coords(G, u, x, y, z);
  const int tx = (G.nx + LG::TX - 1) / LG::TX, ty = (G.ny + LG::TY - 1) / LG::TY;
  const int zlo = (ND == 3) ? -1 : 0, zhi = (ND == 3) ? 1 : 0;
  for (int dz = zlo; dz <= zhi; ++dz) {
    const int Z = z + dz;
    if (Z < 0 || Z >= G.nz) continue;
    if (dz != 0 && (Z / LG::TZ) == (z / LG::TZ)) continue;  // same tile row as dz = 0
    for (int dy = -1; dy <= 1; ++dy) {
      const int Y = y + dy;
      if (Y < 0 || Y >= G.ny) continue;
      if (dy != 0 && (Y / LG::TY) == (y / LG::TY)) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        const int X = x + dx;
        if (X < 0 || X >= G.nx) continue;
        if (dx != 0 && (X / LG::TX) == (x / LG::TX)) continue;
        tdirty[(X / LG::TX) + tx * ((Y / LG::TY) + ty * (Z / LG::TZ))] = 1;
      }
    }
  }
}

// Next unit of this block (u, u + gridDim.x, ...) whose field satisfies
// active(field); the units of an inactive field are skipped in O(1), so a
// kernel with nothing to do costs one lookup per field and block. fi holds
// the field of the block's previous unit, known active: a field's state only
// changes once all of its units of the launch are done, so while the block
// has units of it left it needs no new check.
template <class T, class Pred>
__device__ __forceinline__ int next_active_unit(const GroupArgs<T>& A, const int* pre, int total, int u, Pred active,
                                                int& fi) {
  while (u < total) {
    const int i = field_of_unit(pre, A.nf, u);
    if (i == fi || active(A.fields[i])) {
      fi = i;
      return u;
    }
    const int end = __ldg(pre + i + 1);
    u += ((end - u + (int)gridDim.x - 1) / (int)gridDim.x) * (int)gridDim.x;
  }
  return total;
}

#define MSZ_ACTIVE_UNITS(A, KIND, PRE, FI, PRED)                                                      \
  for (int FI = -1, u_ = next_active_unit((A), (PRE), (A).total[KIND], (int)blockIdx.x, (PRED), FI); \
       u_ < (A).total[KIND]; u_ = next_active_unit((A), (PRE), (A).total[KIND], u_ + (int)gridDim.x, (PRED), FI))

// ---------------------------------------------------------------------------
// Init (Sec. 3 constraint): validate f and fhat (finite, |fhat - f| <= xi via
// the tightest representable bounds), g = fhat, clear flags.
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(kThreads) k_init(GroupArgs<T> A) {
  const int* pre = A.prefix + K_DENSE * (A.nf + 1);
  auto active = [](const Field<T>& F) { return F.st->phase == PH_INIT; };
  auto none = [](DevState*) {};
  auto done = [](DevState* st) { ctrl_after_init(st); };
  UnitTally tl;
  MSZ_ACTIVE_UNITS(A, K_DENSE, pre, i, active) {
    tl.enter(A, K_DENSE, i, none, done);
    const Field<T>& F = A.fields[i];
    DevState* st = F.st;
    const int v0 = (u_ - pre[i]) * kDenseChunk;
    const int v1 = min(F.G.n, v0 + kDenseChunk);
    uint32_t err = 0;
    for (int v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
      const T fv = F.f[v], hv = F.fhat[v];
      if (!finite(fv) || !finite(hv)) {
        err |= E_NONFINITE;
      } else {
        const T lb = lower_bound_of(fv, F.xi);
        const T ub = upper_bound_of(fv, F.xi);
        if (!finite(lb)) err |= E_ARG;
        else if (hv < lb || hv > ub) err |= E_BOUND;
      }
      F.g[v] = hv;
      F.flags[v] = 0;
      F.cls[v] = 0;
      F.epoch[v] = 0;
    }
    if (err) atomicOr(&st->err_bits, err);
    {
      const int ntl = F.units[K_LABEL], nu = F.units[K_DENSE], lu = u_ - pre[i];
      // no exit is marked yet (the marks' words, shared out over the units)
      const int nxw = (int)(F.nface / 4u), pw = (nxw + nu - 1) / nu;
      for (int w = lu * pw + threadIdx.x; w < min(nxw, (lu + 1) * pw); w += blockDim.x) {
        reinterpret_cast<uint32_t*>(F.xm[0])[w] = 0u;
        reinterpret_cast<uint32_t*>(F.xm[1])[w] = 0u;
      }
      // every label tile starts dirty
      const int per = (ntl + nu - 1) / nu;
      for (int t = lu * per + threadIdx.x; t < min(ntl, (lu + 1) * per); t += blockDim.x) {
        F.tdirty[t] = 1;
        F.twrong[t] = 0;
      }
      const int ncc = 4 * F.units[K_EMIT], pc = (ncc + nu - 1) / nu;
      for (int t = lu * pc + threadIdx.x; t < min(ncc, (lu + 1) * pc); t += blockDim.x) F.ccnt[t] = 0;
    }
  }
  tl.flush(A, K_DENSE, none, done);
}

// ---------------------------------------------------------------------------
// C-loop sweep (msz_sweep.cuh): extremum flags of g per vertex; the false
// critical points get their class bits, and their counts per type go to the
// field and to the per-tile counts (one warp reduction of byte-packed counts
// per warp and plane that holds any). Units are tiles (x-y tile by a chunk of
// planes). With kTMA a producer warp streams the planes of the block's
// active tiles through a ring of TMA stages (full/empty mbarriers, bounded
// waits); otherwise the consumers fill one stage with plain loads. A thread
// owns VX vertices of one row (16 bytes of g: one vector load per staged
// row) and carries from plane to plane what the next plane needs (centre
// values, LLL extrema) and the extremum tests already decided, so each
// plane is read from shared memory once.
// ---------------------------------------------------------------------------
template <class T, int ND, bool kTMA>
__global__ void __launch_bounds__(kTMA ? SweepGeom<T, ND>::NTP : SweepGeom<T, ND>::NT)
    k_csweep(GroupArgs<T> A) {
  using SG = SweepGeom<T, ND>;
  constexpr int VX = SG::VX;
  constexpr int NCW = SG::NT / 32;  // consumer warps
  using PV = Partials<T, VX>;
  static_assert((SG::STAGES & (SG::STAGES - 1)) == 0, "power-of-two stages");
  constexpr int SM1 = SG::STAGES - 1;
  __shared__ alignas(128) unsigned char smem[(kTMA ? SG::STAGES : 1) * SG::STAGE_BYTES];
  __shared__ alignas(8) uint64_t full[SG::STAGES];
  __shared__ alignas(8) uint64_t empty[SG::STAGES];
  __shared__ int s_abort;
  __shared__ unsigned s_tiles;
  const int* pre = A.prefix + K_SWEEP * (A.nf + 1);
  const int tid = threadIdx.x;
  const bool producer = kTMA && tid >= SG::NT;
  // the thread's first column in the tile and its row
  const int tx = (tid % SG::TPR) * VX, w = (tid / SG::TPR) % SG::TY;
  const int lane = tid & 31;

  // Next active tile of this block at or after global unit u: field index,
  // tile origin and planes per tile; false when the block's units are done.
  struct Tile {
    int u, i, x0, y0, c0, ppt;
  };
  auto next_tile = [&](Tile& t, int u) -> bool {
    int i = -1;  // no cached field: the producer warp and the consumers decide alike
    u = next_active_unit(
        A, pre, A.total[K_SWEEP], u,
        [](const Field<T>& F) { return F.st->phase == PH_C && F.st->action == ACT_NONE; }, i);
    if (u < A.total[K_SWEEP]) {
      const Field<T>& F = A.fields[i];
      const SweepTiling& TL = F.TL;
      const int lt = u - pre[i];
      const int bx = lt % TL.tiles_x;
      const int r = lt / TL.tiles_x;
      t.u = u;
      t.i = i;
      t.x0 = bx * SG::TX;
      t.y0 = (r % TL.tiles_y) * SG::TY;
      t.c0 = (r / TL.tiles_y) * TL.chunk;
      t.ppt = TL.chunk + 2;
      return true;
    }
    return false;
  };

  if (tid == 0) {
    if (kTMA) {
      for (int s = 0; s < SG::STAGES; ++s) {
        mbar_init(&full[s], 1);
        mbar_init(&empty[s], NCW);
      }
      mbar_fence_init();
    }
    s_abort = 0;
    s_tiles = 0;
  }
  __syncthreads();

  if (producer) {
    if (lane == 0) {
      int q = 0;
      Tile t;
      bool more = next_tile(t, blockIdx.x);
      int fenced = -1;  // field whose maps this thread has acquired
      while (more && !*(volatile int*)&s_abort) {
        const CUtensorMap* gm = A.maps + 2 * t.i;
        if (t.i != fenced) {
          tensormap_acquire(gm);
          tensormap_acquire(gm + 1);
          fenced = t.i;
        }
        for (int p = 0; p < t.ppt; ++p, ++q) {
          const int s = q & SM1;
          if (q >= SG::STAGES &&
              !mbar_wait_or_abort(&empty[s], (uint32_t)(((q - SG::STAGES) / SG::STAGES) & 1), &s_abort)) {
            atomicExch(&s_abort, 1);
            break;
          }
          const int pc = t.c0 - 1 + p;
          unsigned char* sp = smem + s * SG::STAGE_BYTES;
          mbar_expect_tx(&full[s], (uint32_t)(SG::STAGE_ELEMS * sizeof(T) + SG::TX * SG::TY));
          if (ND == 3) {
            tma_load_3d(sp, gm, &full[s], t.x0 - SG::PADX, t.y0 - 1, pc);
            tma_load_3d(sp + SG::G_BYTES, gm + 1, &full[s], t.x0, t.y0, pc);
          } else {
            tma_load_2d(sp, gm, &full[s], t.x0 - SG::PADX, pc);
            tma_load_2d(sp + SG::G_BYTES, gm + 1, &full[s], t.x0, pc);
          }
        }
        more = next_tile(t, t.u + gridDim.x);
      }
      if (*(volatile int*)&s_abort) {
        // wait (bounded) for the copies still in flight before leaving
        const int first = (q > SG::STAGES) ? q - SG::STAGES : 0;
        for (int k = first; k < q; ++k) mbar_wait(&full[k & SM1], (uint32_t)((k / SG::STAGES) & 1));
      }
    }
  } else {
    int q = 0;
    Tile t;
    bool more = next_tile(t, blockIdx.x);
    bool ok = true;
    while (more && ok) {
      const Field<T>& F = A.fields[t.i];
      DevState* st = F.st;
      const Geom G = F.G;
      const int chunk = t.ppt - 2;
      const int axis_n = (ND == 3) ? G.nz : G.ny;
      const int x = t.x0 + tx;  // the thread's first vertex
      const int y = (ND == 3) ? t.y0 + w : 0;
      uint32_t vmask = 0;  // bits 8k, 8k + 4: vertex k is inside the grid in x and y
#pragma unroll
      for (int k = 0; k < VX; ++k)
        if (x + k < G.nx && y < G.ny) vmask |= 0x11u << (8 * k);
      // vertex range of the warp's row segment (contiguous indices), for the
      // per-tile type counts
      const int wx0 = t.x0 + ((tid % SG::TPR) & ~31) * VX;
      const int wx1 = min(G.nx, wx0 + 32 * VX) - 1;
      uint32_t cnt[4] = {0, 0, 0, 0};
      // What a plane carries to the next (two register sets that alternate,
      // no copies): its centre values and LLL extrema (for the next plane's
      // L*(v)), and per vertex k the part of its extremum tests already
      // decided at bits 8k (maximum) and 8k + 4 (minimum): every L*(v)
      // neighbour and its own LUR corner compared with g. The tests against
      // the next plane's centre and LUR corner complete them. A comparison
      // with a max / min of several values is the conjunction of the
      // comparisons with each (NaN halo values compare false and are never
      // the max or min of a set with a number).
      struct PlaneState {
        T a0[VX], lM[VX], lm[VX];
        uint32_t pre;  // decided tests
        uint32_t fd;   // f's direction bytes of the thread's vertices
      };
      PlaneState S[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) S[h].pre = S[h].fd = 0;
      for (int p0 = 0; p0 < t.ppt && ok; p0 += 2) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int p = p0 + h;
          if (p >= t.ppt || !ok) continue;
          PlaneState& cur = S[h];
          const PlaneState& prv = S[h ^ 1];
          const int pcoord = t.c0 - 1 + p;  // plane coordinate (z in 3D, y in 2D)
          unsigned char* sp = smem + (kTMA ? (q & SM1) * SG::STAGE_BYTES : 0);
          const T* stage = reinterpret_cast<const T*>(sp);
          PV n;  // the plane's partials
          uint32_t fd = 0;
          if (kTMA) {
            // every lane waits for the stage (one decision for the warp)
            const bool got =
                __all_sync(kFull, mbar_wait_or_abort(&full[q & SM1], (uint32_t)((q / SG::STAGES) & 1), &s_abort));
            if (!got) {
              if (lane == 0) atomicExch(&s_abort, 1);
              ok = false;
              continue;
            }
            plane_partials<T, ND>(stage, SG::PADX + tx, w, n);
            const unsigned char* dp = sp + SG::G_BYTES + w * SG::TX + tx;
            if constexpr (VX == 4) fd = *reinterpret_cast<const uint32_t*>(dp);
            else if constexpr (VX == 2) fd = *reinterpret_cast<const uint16_t*>(dp);
            else fd = *dp;
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[q & SM1]);
          } else {
            __syncthreads();
            T* wst = reinterpret_cast<T*>(sp);
            for (int k = tid; k < SG::STAGE_ELEMS; k += SG::NT) {
              const int col = k % SG::BX, row = k / SG::BX;
              const int gx = t.x0 - SG::PADX + col;
              const int gy = (ND == 3) ? t.y0 - 1 + row : pcoord;
              const int gz = (ND == 3) ? pcoord : 0;
              const bool in = gx >= 0 && gx < G.nx && gy >= 0 && gy < G.ny && gz >= 0 && gz < G.nz;
              wst[k] = in ? F.g[gx + G.nx * (gy + G.ny * gz)] : qnan<T>();
            }
            __syncthreads();
            plane_partials<T, ND>(stage, SG::PADX + tx, w, n);
            const int vy = (ND == 3) ? y : pcoord, vz = (ND == 3) ? pcoord : 0;
#pragma unroll
            for (int k = 0; k < VX; ++k)
              if (x + k < G.nx && vy >= 0 && vy < G.ny && vz >= 0 && vz < G.nz)
                fd |= (uint32_t)F.fdir[(x + k) + G.nx * (vy + G.ny * vz)] << (8 * k);
          }
          ++q;
          if (p >= 2 && p - 2 < chunk) {
            // The previous plane's extremum flags (g's, completed with this
            // plane's centre and LUR corner; f's from its direction bytes)
            // at bits 8k (max) and 8k + 4 (min) of vertex k, and the false
            // types from their differences, word-parallel.
            uint32_t gb = 0;
#pragma unroll
            for (int k = 0; k < VX; ++k) {
              const T g = prv.a0[k];
              gb |= ((uint32_t)!(vmax(n.a0[k], n.uM[k]) >= g) << (8 * k)) |
                    ((uint32_t)!(vmin(n.a0[k], n.um[k]) < g) << (8 * k + 4));
            }
            gb &= prv.pre;
            const uint32_t fa = prv.fd;
            const uint32_t fb = fa & (fa >> 1) & (fa >> 2) & (fa >> 3) & 0x11111111u;  // nibble == 15
            const uint32_t valid = (pcoord - 1 < axis_n) ? vmask : 0u;
            const uint32_t Pm = gb & ~fb & valid;  // g's extremum, not f's: FPmax (bit 8k), FPmin (8k + 4)
            const uint32_t Nm = fb & ~gb & valid;  // f's extremum, not g's: FNmax, FNmin
            if (__any_sync(kFull, (Pm | Nm) != 0u)) {
              // byte k: the type bits of vertex k (FPmax, FPmin, FNmax, FNmin)
              const uint32_t codes = (Pm & 0x01010101u) | ((Pm >> 3) & 0x02020202u) |
                                     ((Nm << 2) & 0x04040404u) | ((Nm >> 1) & 0x08080808u);
              // the thread's count of each type, one per byte, for one warp reduction
              const uint32_t packed =
                  (uint32_t)__popc(Pm & 0x01010101u) | ((uint32_t)__popc(Pm & 0x10101010u) << 8) |
                  ((uint32_t)__popc(Nm & 0x01010101u) << 16) | ((uint32_t)__popc(Nm & 0x10101010u) << 24);
              const int z = (ND == 3) ? pcoord - 1 : 0;
              const int yy = (ND == 3) ? y : pcoord - 1;
              const int v0 = x + G.nx * (yy + G.ny * z);
              // class bits of the false vertices (cls starts zeroed and each
              // vertex has one owner): one store of the thread's bytes where
              // the row pitch keeps it aligned
              if (codes) {
                if constexpr (kTMA && VX == 4) {
                  *reinterpret_cast<uint32_t*>(F.cls + v0) = codes;
                } else if constexpr (kTMA && VX == 2) {
                  *reinterpret_cast<uint16_t*>(F.cls + v0) = (uint16_t)codes;
                } else {
#pragma unroll
                  for (int k = 0; k < VX; ++k)
                    if ((codes >> (8 * k)) & 15u) F.cls[v0 + k] = (uint8_t)((codes >> (8 * k)) & 15u);
                }
              }
              const uint32_t tot = __reduce_add_sync(kFull, packed);
              // per-tile type counts: one atomic per type when the warp's row
              // segment lies in one count tile, else one per vertex
              const int wv0 = wx0 + G.nx * (yy + G.ny * z), wv1 = wx1 + G.nx * (yy + G.ny * z);
              const int ct = wv0 / kEmitTile;
              if (ct == wv1 / kEmitTile) {
                if (lane == 0) {
#pragma unroll
                  for (int c = 0; c < 4; ++c) {
                    const uint32_t nc = (tot >> (8 * c)) & 0xffu;
                    if (nc) atomicAdd(&F.ccnt[ct * 4 + c], nc);
                  }
                }
              } else {
#pragma unroll
                for (int k = 0; k < VX; ++k) {
                  const uint32_t bits = (codes >> (8 * k)) & 15u;
#pragma unroll
                  for (int c = 0; c < 4; ++c)
                    if ((bits >> c) & 1u) atomicAdd(&F.ccnt[((v0 + k) / kEmitTile) * 4 + c], 1u);
                }
              }
              if (lane == 0) {
#pragma unroll
                for (int c = 0; c < 4; ++c) cnt[c] += (tot >> (8 * c)) & 0xffu;
              }
            }
          }
          // This plane's decided tests: its own LUR corner, and L*(v) (its
          // LLL corner, the previous plane's centre and LLL corner).
          uint32_t pre = 0;
#pragma unroll
          for (int k = 0; k < VX; ++k) {
            const T g = n.a0[k];
            const T LM = vmax3(n.lM[k], prv.a0[k], prv.lM[k]);
            const T Lm = vmin3(n.lm[k], prv.a0[k], prv.lm[k]);
            pre |= ((uint32_t)(!(n.uM[k] >= g) && !(LM > g)) << (8 * k)) |
                   ((uint32_t)(!(n.um[k] < g) && !(Lm <= g)) << (8 * k + 4));
          }
          cur.pre = pre;
#pragma unroll
          for (int k = 0; k < VX; ++k) {
            cur.a0[k] = n.a0[k];
            cur.lM[k] = n.lM[k];
            cur.lm[k] = n.lm[k];
          }
          cur.fd = fd;
        }
      }
      if (!ok) break;
      // Tile done by this warp: flush its counts; the last consumer warp to
      // finish the tile counts the unit for the field.
      if (lane == 0) {
        for (int c = 0; c < 4; ++c)
          if (cnt[c]) atomicAdd(&st->counts[c], cnt[c]);
        __threadfence();
        const unsigned old = atomicAdd(&s_tiles, 1u);
        if ((old + 1) % NCW == 0) {
          __threadfence();
          if (atomicAdd(&st->units_done, 1u) == (uint32_t)(F.units[K_SWEEP] - 1)) {
            __threadfence();
            ctrl_after_classify(st);
            log_work(A);
            st->units_done = 0;
          }
        }
      }
      __syncwarp();
      more = next_tile(t, t.u + gridDim.x);
    }
    if (!ok && lane == 0) {
      // gave up on a bounded wait: the tile is not counted, so the field's
      // state machine stalls and the host reports MSZ_ERR_TIMEOUT
      atomicOr(&A.fields[t.i].st->err_bits, E_TIMEOUT);
    }
  }
}

// The round's cases of the field's current type, listed from the per-vertex
// false-type bits; only tiles that hold cases of the type are read. A unit
// is kCaseTiles case-count tiles, kTilesPerWarp per warp (their counts read
// together); each 512-byte chunk of a tile appends its cases with one atomic
// per warp.
template <class T, int ND>
__global__ void __launch_bounds__(kThreads) k_gather(GroupArgs<T> A) {
  const int* pre = A.prefix + K_CASE * (A.nf + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto active = [](const Field<T>& F) { return F.st->action == ACT_GATHER; };
  uint32_t ncases = 0;
  auto pre_flush = [&](DevState* st) {
    log_units_warp(A, st, KID_GATHER, ncases);
    ncases = 0;
  };
  auto done = [&](DevState* st) {
    st->action = ACT_REQUEST;
    st->ticks++;
    log_work(A);
  };
  UnitTally tl;
  MSZ_ACTIVE_UNITS(A, K_CASE, pre, i, active) {
    tl.enter(A, K_CASE, i, pre_flush, done);
    const Field<T>& F = A.fields[i];
    const uint32_t type = F.st->T;
    // the warp's kTilesPerWarp tiles: their counts in one go, then the tiles with cases
    const int t0 = (u_ - pre[i]) * kCaseTiles + warp * kTilesPerWarp;
    const int tl_lane = t0 + lane;
    const bool has = lane < kTilesPerWarp && tl_lane * kEmitTile < F.G.n && F.ccnt[tl_lane * 4 + type] != 0;
    for (uint32_t hm = __ballot_sync(kFull, has); hm; hm &= hm - 1) {
      const int tile = t0 + __ffs(hm) - 1;
#pragma unroll 1
      for (int r = 0; r < kEmitTile / (32 * 16); ++r) {
        const int base = tile * kEmitTile + (r * 32 + lane) * 16;
        const uint4 q = *reinterpret_cast<const uint4*>(F.cls + base);
        const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
        uint32_t hits = 0;  // bit k: byte k holds a case of the type
#pragma unroll
        for (int k = 0; k < 16; ++k) hits |= ((w4[k >> 2] >> (8 * (k & 3) + type)) & 1u) << k;
        if (F.G.n - base < 16) hits &= (F.G.n - base > 0) ? (1u << (F.G.n - base)) - 1u : 0u;  // padding
        const uint32_t c = __popc(hits);
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += y;
        }
        const uint32_t total = __shfl_sync(kFull, incl, 31);
        if (!total) continue;
        uint32_t at = 0;
        if (lane == 31) at = atomicAdd(&F.st->ncase, total);
        at = __shfl_sync(kFull, at, 31) + incl - c;
        for (; hits; hits &= hits - 1, ++at)
          if (MSZ_IN(F.st, at, F.G.n)) F.cases[at] = (uint32_t)(base + __ffs(hits) - 1);
        ncases += c;
      }
    }
  }
  tl.flush(A, K_CASE, pre_flush, done);
}

// C-loop requests for the listed cases (Eqs. 2-5), one case per thread over
// the whole grid: FPmax and FNmin edit the false vertex itself; FPmin and
// FNmax edit its neighbour that is maximal in g, which is its steepest ascent
// since it is not a maximum of g's ring. A decrease is one flag mark; a
// request that freezes its anchor's closed ring lists the anchor in shared
// memory, and the block's warps mark the listed rings after its cases, a
// lane per ring vertex. All requests read the same snapshot (nothing they
// write is read by another request), so the order does not matter.
template <class T, int ND>
__global__ void __launch_bounds__(kThreads) k_mark(GroupArgs<T> A) {
  const int* pre = A.prefix + K_SPARSE * (A.nf + 1);
  auto active = [](const Field<T>& F) { return F.st->action == ACT_REQUEST; };
  auto none = [](DevState*) {};
  auto done = [&](DevState* st) {
    st->action = ACT_MARK_C;
    st->ticks++;
    log_work(A);
  };
  constexpr uint32_t kMFreeze = 1024;
  __shared__ uint32_t s_fz[kMFreeze];
  __shared__ uint32_t s_nfz;
  if (threadIdx.x == 0) s_nfz = 0;
  UnitTally tl;
  MSZ_ACTIVE_UNITS(A, K_SPARSE, pre, i, active) {
    const Field<T>& F = A.fields[i];
    DevState* st = F.st;
    uint64_t b, e;
    const uint32_t act = sparse_slice(st->ncase, F.units[K_SPARSE], u_ - pre[i], b, e);
    if ((uint32_t)(u_ - pre[i]) >= act) continue;  // left out: not counted
    tl.enter(A, K_SPARSE, i, none, done);
    tl.target = act;
    const uint32_t type = st->T;
    if (threadIdx.x == 0) log_units(A, st, KID_MARK, e - b);
    __syncthreads();  // the freeze list is empty
    for (uint64_t j = b + threadIdx.x; j < e; j += kThreads) {
      const int v = (int)F.cases[j];
      if (!MSZ_IN(st, v, F.G.n)) continue;
      const uint8_t d = F.gdir[v];  // exact: reclassified after every apply
      const int t = (type == FPMAX || type == FNMIN) ? v : v + slot_offset(d & 15, ND, F.G.nx, F.G.nxny);
      if (!MSZ_IN(st, t, F.G.n)) continue;
      const int cause = request_cause(F, t);
      if (cause == RQ_DEC) {
        mark(F, t, FL_DEC);
        continue;
      }
      count_freeze_req(st, (int)type, cause);
      const uint32_t q = atomicAdd(&s_nfz, 1u);
      if (q < kMFreeze) s_fz[q] = (uint32_t)v;
      else request<T, ND>(F, v, t);  // list full: the same freeze, vertex by vertex
    }
    __syncthreads();
    const uint32_t nfz = min(s_nfz, kMFreeze);
    for (uint32_t q = threadIdx.x >> 5; q < nfz; q += kThreads / 32)
      freeze_ring_warp<T, ND>(F, (int)s_fz[q], (int)(threadIdx.x & 31));
    __syncthreads();  // every thread has read the list and its count
    if (threadIdx.x == 0) s_nfz = 0;
  }
  tl.flush(A, K_SPARSE, none, done);
}

template <class T>
__device__ __forceinline__ uint32_t reclass_update(const Field<T>& F, int v, uint8_t dv, uint8_t fd, unsigned ob,
                                                   uint32_t (&acc)[4], int& vc);

// One reclassification item: ring slot s of touched vertex u (slot 2 * NPOS:
// u itself). The first item to reach a vertex in the round claims it (epoch
// stamp) and recomputes its false-type bits and its direction byte in g; the
// tile counts and acc move by the difference. The claimer gets
// 0x10000 | (old << 8) | new and vc = the vertex; any other item gets 0.
template <class T, int ND>
__device__ __forceinline__ uint32_t reclass_item(const Field<T>& F, int u, int s, uint32_t stamp, uint32_t (&acc)[4],
                                                 int& vc) {
  constexpr int NPOS = Slots<ND>::NPOS;
  const Geom& G = F.G;
  int x, y, z;
  coords(G, u, x, y, z);
  int v = u;
  if (s < 2 * NPOS) {
    const int sg = (s < NPOS) ? 1 : -1;
    const int m = (int)((Slots<ND>::MASKS >> (4 * (s < NPOS ? s : s - NPOS))) & 7u);
    const int dx = sg * (m & 1), dy = sg * ((m >> 1) & 1), dz = sg * ((m >> 2) & 1);
    x += dx;
    y += dy;
    z += dz;
    if (x < 0 || x >= G.nx || y < 0 || y >= G.ny || z < 0 || z >= G.nz) return 0;
    v = u + dx + dy * G.nx + dz * G.nxny;
  }
  // Only the claimer loads the class inputs: in a round whose rings
  // overlap, most items lose the claim.
  if (atomicExch(&F.epoch[v], stamp) == stamp) return 0;
  return reclass_update(F, v, direction_of<T, ND>(F.g, G, v, x, y, z), F.fdir[v], F.cls[v], acc, vc);
}

// The same for vertex v at (x, y, z) without a claim (a pass over every vertex).
template <class T, int ND>
__device__ __forceinline__ uint32_t reclass_vertex(const Field<T>& F, int v, int x, int y, int z, uint32_t (&acc)[4],
                                                   int& vc) {
  return reclass_update(F, v, direction_of<T, ND>(F.g, F.G, v, x, y, z), F.fdir[v], F.cls[v], acc, vc);
}

// Vertex v's new direction byte dv in g, f's direction byte fd and its old
// false-type bits ob: the byte and the bits are stored, the counts move.
// Returns 0x10000 | (ob << 8) | nb and sets vc = v.
template <class T>
__device__ __forceinline__ uint32_t reclass_update(const Field<T>& F, int v, uint8_t dv, uint8_t fd, unsigned ob,
                                                   uint32_t (&acc)[4], int& vc) {
  F.gdir[v] = dv;  // g's direction bytes stay exact for the requests and the labels
  const unsigned nb = case_bits(dv, fd);
  vc = v;
  if (nb == ob) return 0x10000u | (ob << 8) | nb;
  F.cls[v] = (uint8_t)nb;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const uint32_t d = ((nb >> c) & 1u) - ((ob >> c) & 1u);  // +1, 0 or -1 (mod 2^32)
    if (d) {
      atomicAdd(&F.ccnt[(v / kEmitTile) * 4 + c], d);
      acc[c] += d;
    }
  }
  return 0x10000u | (ob << 8) | nb;
}

// Incremental classification after an apply. A vertex's false-type bits
// depend only on g over its closed 1-ring, so only the closed 1-rings of the
// vertices the apply touched can change: the result equals a full sweep of
// the new g. Items are (touched vertex, ring slot) pairs; the first item to
// reach a vertex in this round claims it (epoch stamp = round number) and
// recomputes its bits and its direction byte in g; the field and tile type
// counts move by the difference. Units are slices of the items.
template <class T, int ND>
__global__ void __launch_bounds__(kThreads) k_reclass(GroupArgs<T> A) {
  const int* pre = A.prefix + K_SPARSE * (A.nf + 1);
  constexpr int NPOS = Slots<ND>::NPOS;
  constexpr int R = 2 * NPOS + 1;
  auto active = [](const Field<T>& F) { return F.st->action == ACT_RECLASS; };
  uint32_t acc[4] = {0, 0, 0, 0};
  auto pre_flush = [&](DevState* st) {
    block_add_striped<4>(acc, st);
    acc[0] = acc[1] = acc[2] = acc[3] = 0;
  };
  auto done = [&](DevState* st) {
    ctrl_after_classify(st);
    log_work(A);
  };
  UnitTally tl;
  MSZ_ACTIVE_UNITS(A, K_SPARSE, pre, i, active) {
    const Field<T>& F = A.fields[i];
    DevState* st = F.st;
    // more ring items than vertices: every vertex once, in order, unclaimed
    const bool dense = (uint64_t)st->ntouch * R > (uint64_t)F.G.n;
    uint64_t b, e;
    const uint32_t act =
        sparse_slice(dense ? (uint64_t)F.G.n : (uint64_t)st->ntouch * R, F.units[K_SPARSE], u_ - pre[i], b, e);
    if ((uint32_t)(u_ - pre[i]) >= act) continue;  // left out: not counted
    tl.enter(A, K_SPARSE, i, pre_flush, done);
    tl.target = act;
    const uint32_t stamp = (uint32_t)st->rounds;
    if (threadIdx.x == 0) log_units(A, st, KID_RECLASS, e - b);
    int vc;
    if (dense) {
      for (uint64_t j = b + threadIdx.x; j < e; j += blockDim.x) {
        int x, y, z;
        coords(F.G, (int)j, x, y, z);
        reclass_vertex<T, ND>(F, (int)j, x, y, z, acc, vc);
      }
    } else {
      for (uint64_t j = b + threadIdx.x; j < e; j += blockDim.x) {
        const uint32_t u = F.touched[j / R];
        if (MSZ_IN(st, u, F.G.n)) reclass_item<T, ND>(F, (int)u, (int)(j % R), stamp, acc, vc);
      }
    }
  }
  tl.flush(A, K_SPARSE, pre_flush, done);
}

// ---------------------------------------------------------------------------
// Labels, first level (Sec. 5.2 path compression): a block loads a tile plus
// a one-vertex halo into shared memory, computes every tile vertex's
// steepest ascending / descending neighbour (candidates in ascending index
// order: ties go to the larger index for the maximum and to the smaller for
// the minimum; NaN halo cells never win), and follows the pointers inside the
// tile by pointer doubling. Each vertex leaves with its tile terminal in each
// direction (one 32-bit word, see kTermFlag): the shell cell where its
// integral line leaves the tile, or the extremum inside the tile where it
// ends. Job 0: f (fdir, terminals), job 1: g (terminals from gdir).
// ---------------------------------------------------------------------------
// Dynamic shared memory of k_label_tile: f's pass holds the halo values and
// the pointers, g's passes the pointers only.
template <class T, int ND, bool JOB>
size_t label_smem_bytes() {
  using LG = LabelGeom<ND>;
  return (JOB ? 0 : ((LG::HALO * sizeof(T) + 15) / 16) * 16) + (size_t)LG::HALO * sizeof(uint32_t);
}

// A tile's values with a one-cell halo: every in-grid cell by an
// asynchronous global -> shared copy (all of the block's copies in flight at
// once), the others NaN.
template <class T, int ND>
__device__ __forceinline__ void load_halo(T* val, const T* src, const Geom& G, int x0, int y0, int z0) {
  using LG = LabelGeom<ND>;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int row = warp; row < LG::ROWS; row += kThreads / 32) {
    const int hy = row % LG::SY, hz = row / LG::SY;
    const int gy = y0 - 1 + hy, gz = (ND == 3) ? z0 - 1 + hz : 0;
    const bool rin = gy >= 0 && gy < G.ny && gz >= 0 && gz < G.nz;
    const size_t rbase = rin ? (size_t)G.nx * ((size_t)gy + (size_t)G.ny * gz) : 0;
    for (int hx = lane; hx < LG::SX; hx += 32) {
      const int gx = x0 - 1 + hx;
      const int h = hx + LG::SX * row;
      if (rin && gx >= 0 && gx < G.nx) cp_async_elem(&val[h], src + rbase + gx);
      else val[h] = qnan<T>();
    }
  }
}

// Direction byte (ascending slot | descending slot << 4) of tile cell c from
// the halo values: candidates in ascending index order, so ties go to the
// larger index for the maximum and to the smaller for the minimum (Sec. 3
// SoS); NaN cells never win.
template <class T, int ND>
__device__ __forceinline__ uint32_t halo_dir(const T* val, int c) {
  using LG = LabelGeom<ND>;
  constexpr int HS = LG::SX, HSS = LG::SX * LG::SY;
  constexpr int NC = (ND == 3) ? 15 : 7;
  T hv = -INFINITY, lv = INFINITY;
  int hs = kSelf, ls = kSelf;
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    int o, slot;
    if (ND == 3) {
      constexpr int tab[15][2] = {{-1 - HS - HSS, 13}, {-HS - HSS, 12}, {-1 - HSS, 11}, {-HSS, 9},
                                  {-1 - HS, 10},       {-HS, 8},        {-1, 7},        {0, kSelf},
                                  {1, 0},              {HS, 1},         {1 + HS, 3},    {HSS, 2},
                                  {1 + HSS, 4},        {HS + HSS, 5},   {1 + HS + HSS, 6}};
      o = tab[j][0];
      slot = tab[j][1];
    } else {
      constexpr int tab[7][2] = {{-1 - HS, 5}, {-HS, 4}, {-1, 3}, {0, kSelf}, {1, 0}, {HS, 1}, {1 + HS, 2}};
      o = tab[j][0];
      slot = tab[j][1];
    }
    const T u = val[c + o];
    if (u >= hv) { hv = u; hs = slot; }
    if (u < lv) { lv = u; ls = slot; }
  }
  return (uint32_t)hs | ((uint32_t)ls << 4);
}

// Whether the neighbour in slot s of a tile cell lies outside the tile. bhi /
// blo: the cell's axes (bit 0 x, 1 y, 2 z) on the tile's upper / lower face.
template <int ND>
__device__ __forceinline__ bool leaves_tile(int s, uint32_t bhi, uint32_t blo) {
  if (s == kSelf) return false;
  constexpr int npos = Slots<ND>::NPOS;
  const bool neg = s >= npos;
  const uint32_t m = (uint32_t)slot_mask(ND, neg ? s - npos : s);
  return (m & (neg ? blo : bhi)) != 0u;
}

// One pointer-doubling step of a 16-bit half a (lo: the low half of the
// words in PP, else the high half): a flagged half is a final terminal value
// and stays; a pointer moves to the pointed cell's half. The load is made in
// either case (a flagged half's low bits index a valid cell) so that both
// halves' loads issue together.
__device__ __forceinline__ uint32_t double_half(const uint32_t* PP, uint32_t a, bool lo) {
  const uint32_t w = PP[a & kTermIdx];
  const uint32_t q = lo ? (w & 0xffffu) : (w >> 16);
  return (a & kTermFlag) ? a : q;
}

// JOB: the fields in f's pass (false) or in g's (true); the two are launched
// side by side, each doing nothing for the other's fields.
template <class T, int ND, bool JOB>
__global__ void __launch_bounds__(kThreads, JOB ? 6 : 4) k_label_tile(GroupArgs<T> A) {
  using LG = LabelGeom<ND>;
  extern __shared__ __align__(16) unsigned char lsm[];
  T* val = reinterpret_cast<T*>(lsm);
  // Per halo cell, the ascending (low 16 bits) and descending (high 16 bits)
  // halves: a tile cell's halves point to its steepest neighbours (halo
  // indices), or hold its own terminal value kTermFlag | kTermExtr | cell
  // index if it is the extremum; a shell cell's halves hold its terminal
  // value kTermFlag | shell index.
  uint32_t* PP = reinterpret_cast<uint32_t*>(lsm + (JOB ? 0 : ((LG::HALO * sizeof(T) + 15) / 16) * 16));
  const int* pre = A.prefix + K_LABEL * (A.nf + 1);
  constexpr int HS = LG::SX, HSS = LG::SX * LG::SY;
  // the tile's exits by shell index (ascending, descending lines): the
  // tile's record for the label lookups
  constexpr int kShW = LabelGeom<ND>::SHW;
  __shared__ uint32_t shx[2][kShW];
  // halo-index offset of each stencil slot (slot 15: the cell itself)
  __shared__ int s_off[16];
  if (threadIdx.x < 16) s_off[threadIdx.x] = slot_offset((int)threadIdx.x, ND, HS, HSS);
  __shared__ int s_slotd[LG::SHELL];  // shell cells' exit-table slots, relative (shell_slot_delta)
  int slot_field = -1;                // the field s_slotd was filled for
  auto active = [](const Field<T>& F) {
    return F.st->action == ACT_LABELS && F.st->lstate == L_INIT && (F.st->ljob != 0) == JOB;
  };
  auto none = [](DevState*) {};
  auto done = [&](DevState* st) {
    st->lstate = L_JUMP;
    st->jump_rounds = 0;
    st->ticks++;
    log_work(A);
  };
  UnitTally tl;
  MSZ_ACTIVE_UNITS(A, K_LABEL, pre, fi, active) {
    tl.enter(A, K_LABEL, fi, none, done);
    const Field<T>& F = A.fields[fi];
    DevState* st = F.st;
    constexpr bool job = JOB;
    const Geom G = F.G;
    const int tiles_x = (G.nx + LG::TX - 1) / LG::TX;
    const int tiles_y = (G.ny + LG::TY - 1) / LG::TY;
    const int tile = u_ - pre[fi];
    // g's terminals only change in tiles whose tile or halo was edited
    const bool redo = !job || (F.tdirty[tile] & 1);
    __syncthreads();  // the block's previous tile is done with the shared arrays
    if (!redo) {
      // A tile that keeps its terminals keeps its first-level exit-table
      // entries; the working table restarts from them (16-byte copies: a
      // tile's block of slots is a multiple of 16 bytes).
      constexpr int kQ = LG::NFACE / 4;
      static_assert(LG::NFACE % 4 == 0, "whole 16-byte groups per tile");
      for (int k = threadIdx.x; k < 2 * kQ; k += kThreads) {
        const int d = k / kQ, q = k - d * kQ;
        reinterpret_cast<uint4*>(F.lw[d] + (size_t)tile * LG::NFACE)[q] =
            reinterpret_cast<const uint4*>(F.lf[d] + (size_t)tile * LG::NFACE)[q];
      }
      // algorithmic bytes (kernel timing runs): both tables' slots of the tile
      if (threadIdx.x == 0) log_units(A, st, KID_LABEL, 16ull * LG::NFACE);
      continue;
    }
    if (fi != slot_field) {  // the same for every thread of the block
      fill_slot_table<ND>(s_slotd, G);
      slot_field = fi;
    }
    const int x0 = (tile % tiles_x) * LG::TX;
    const int y0 = ((tile / tiles_x) % tiles_y) * LG::TY;
    const int z0 = (tile / (tiles_x * tiles_y)) * LG::TZ;
    for (int k = threadIdx.x; k < 2 * kShW; k += kThreads) shx[k / kShW][k % kShW] = 0u;
    // Job 0 reads f's values with the halo; job 1 needs no values: g's
    // direction bytes are kept exact by the classification that follows
    // every apply. The shell cells get their terminal values.
    if (!job) load_halo<T, ND>(val, F.f, G, x0, y0, z0);
    for (int s = threadIdx.x; s < LG::SHELL; s += kThreads) {
      int hx, hy, hz;
      shell_cell<ND>(s, hx, hy, hz);
      const uint32_t t = kTermFlag | (uint32_t)s;
      PP[hx + HS * (hy + LG::SY * hz)] = t | (t << 16);
    }
    cp_async_wait_all();
    __syncthreads();
    // Pointers of the tile cells inside the grid (the others are never
    // reached and stay out of the doubling). A pointer that leaves the tile
    // marks its shell cell as a tile exit: the first halo cell on an
    // integral line is the steepest neighbour of the line's last tile cell,
    // so the marked cells are exactly the exits of the tile's lines.
    uint32_t live = 0;
    const CellWalk<ND> cw;
    const int hc0 = cw.c0(), vs = cw.vstep(G);
    const int v0 = (x0 + cw.lx) + G.nx * ((y0 + cw.ly(0)) + G.ny * (z0 + cw.lz(0)));
#pragma unroll
    for (int k = 0; k < LG::PER_THREAD; ++k) {
      if (!cw.inside(G, x0, y0, z0, k)) continue;
      live |= 1u << k;
      const int i = threadIdx.x + k * kThreads;
      const int lx = cw.lx, ly = cw.ly(k), lz = cw.lz(k);
      const int c = hc0 + k * CellWalk<ND>::HSTEP;
      const int v = v0 + k * vs;
      uint32_t db;
      if (!job) {
        db = halo_dir<T, ND>(val, c);
        F.fdir[v] = (uint8_t)db;
      } else {
        db = F.gdir[v];
      }
      const int sa = (int)(db & 15u), sd = (int)(db >> 4);
      int ca = c + s_off[sa], cd = c + s_off[sd];
      if (!MSZ_IN(st, ca, LG::HALO)) ca = c;
      if (!MSZ_IN(st, cd, LG::HALO)) cd = c;
      const uint32_t self = kTermFlag | kTermExtr | (uint32_t)i;  // i: the tile cell index
      PP[c] = (sa == kSelf ? self : (uint32_t)ca) | ((sd == kSelf ? self : (uint32_t)cd) << 16);
      const uint32_t bhi = (uint32_t)(lx == LG::TX - 1) | ((uint32_t)(ly == LG::TY - 1) << 1) |
                           ((uint32_t)(ND == 3 && lz == LG::TZ - 1) << 2);
      const uint32_t blo = (uint32_t)(lx == 0) | ((uint32_t)(ly == 0) << 1) | ((uint32_t)(ND == 3 && lz == 0) << 2);
      if (bhi | blo) {
        // the exit's halo coordinates from the cell's and the slot's
        auto mark_exit = [&](int d, int sl) {
          constexpr int npos = Slots<ND>::NPOS;
          const bool neg = sl >= npos;
          const int m = slot_mask(ND, neg ? sl - npos : sl), sg = neg ? -1 : 1;
          const int sh = shell_index<ND>(lx + 1 + sg * (m & 1), ly + 1 + sg * ((m >> 1) & 1),
                                         (ND == 3) ? lz + 1 + sg * ((m >> 2) & 1) : 0);
          atomicOr(&shx[d][sh >> 5], 1u << (sh & 31));
        };
        if (leaves_tile<ND>(sa, bhi, blo)) mark_exit(0, sa);
        if (leaves_tile<ND>(sd, bhi, blo)) mark_exit(1, sd);
      }
    }
    if (!job) {
      // g's values (f-hat at this point) for g's first direction bytes,
      // copied in while the pointers double
      __syncthreads();
      load_halo<T, ND>(val, F.g, G, x0, y0, z0);
    }
    __syncthreads();
    // pointer doubling until every cell of the tile holds its two terminals
    for (int round = 0; round < 2 * LG::TV && __syncthreads_or(live != 0u); ++round) {
      // the thread's live cells only
      for (uint32_t lm = live; lm; lm &= lm - 1) {
        const int k = __ffs(lm) - 1;
        const int c = hc0 + k * CellWalk<ND>::HSTEP;
        const uint32_t p = PP[c];
        uint32_t a = p & 0xffffu, b = p >> 16;
        if (!MSZ_IN(st, a & kTermIdx, LG::HALO)) a = kTermFlag;
        if (!MSZ_IN(st, b & kTermIdx, LG::HALO)) b = kTermFlag;
        const uint32_t a2 = double_half(PP, a, true);
        const uint32_t b2 = double_half(PP, b, false);
        PP[c] = a2 | (b2 << 16);  // stored even when unchanged: fewer instructions than the test
        if (a2 & b2 & kTermFlag) live &= ~(1u << k);
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < LG::PER_THREAD; ++k) {
      if (cw.inside(G, x0, y0, z0, k)) {
        const int lx = cw.lx, ly = cw.ly(k), lz = cw.lz(k);
        const int v = v0 + k * vs;
        const uint32_t p = PP[hc0 + k * CellWalk<ND>::HSTEP];
        F.term[v] = p;
      }
    }
    // the tile's exit record
    for (int k = threadIdx.x; k < 2 * kShW; k += kThreads)
      F.texit[(size_t)tile * 2 * kShW + k] = shx[k / kShW][k % kShW];
    // First-level exit-table entries of the tile's face cells (a slot per
    // face cell, see exit_slot): a line that ends inside the tile gives its
    // label (kRes), one that leaves it the slot of the exit it leaves
    // through. Entries of tiles that are not recomputed stay valid.
    const uint32_t tbase = (uint32_t)tile * (uint32_t)LG::NFACE;
    auto exit_of = [&](uint32_t s) -> uint32_t {
      if (!MSZ_IN(st, s, LG::SHELL)) s = 0;
      const uint32_t sl = tbase + (uint32_t)s_slotd[s];
      return MSZ_IN(st, sl, F.nface) ? sl : 0u;
    };
    for (int f = threadIdx.x; f < LG::NFACE; f += kThreads) {
      int lx, ly, lz;
      face_cell<ND>(f, lx, ly, lz);
      if (x0 + lx >= G.nx || y0 + ly >= G.ny || z0 + lz >= G.nz) continue;
      const uint32_t p = PP[(lx + 1) + HS * ((ly + 1) + LG::SY * ((ND == 3) ? lz + 1 : 0))];
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        const uint32_t t = d ? (p >> 16) : (p & 0xffffu);
        const uint32_t e = (t & kTermExtr) ? ((uint32_t)extremum_vertex<ND>(G, t, x0, y0, z0) | kRes)
                                           : exit_of(t & kTermIdx);
        F.lf[d][tbase + f] = e;
        F.lw[d][tbase + f] = e;  // the working table starts from the first level
      }
    }
    // Exit marks (the entries the jumping resolves): the slot of each exit
    // of the tile's lines. Marks are cleared only when a fix starts.
    for (int k = threadIdx.x; k < 2 * kShW; k += kThreads) {
      const int d = k / kShW, wd = k % kShW;
      for (uint32_t b = shx[d][wd]; b; b &= b - 1) F.xm[d][exit_of((uint32_t)(wd * 32 + __ffs(b) - 1))] = 1;
    }
    if (!job) {
      // g's first direction bytes; from here on the classification after
      // every apply keeps them exact
      cp_async_wait_all();
      __syncthreads();
#pragma unroll
      for (int k = 0; k < LG::PER_THREAD; ++k)
        if (cw.inside(G, x0, y0, z0, k))
          F.gdir[v0 + k * vs] = (uint8_t)halo_dir<T, ND>(val, hc0 + k * CellWalk<ND>::HSTEP);
    }
    // recomputed, for the R-check to examine (f's pass leaves every tile
    // dirty for g's first)
    if (job && threadIdx.x == 0) F.tdirty[tile] = 2;
    // algorithmic bytes (kernel timing runs): per vertex, g's direction byte
    // read and the terminal word written (f's pass: f and g read, both
    // direction bytes and the terminal word written); per face cell, its
    // entries in both tables of both directions
    if (threadIdx.x == 0)
      log_units(A, st, KID_LABEL,
                (job ? 5ull : 14ull) * min(LG::TX, G.nx - x0) * min(LG::TY, G.ny - y0) * min(LG::TZ, G.nz - z0) +
                    16ull * LG::NFACE);
  }
  tl.flush(A, K_LABEL, none, done);
}

// Labels, second level (Sec. 5.2, across tiles). Each direction has two
// exit tables with one slot per face cell of every label tile (exit_slot):
// lf holds the first-level entries that k_label_tile writes for the face
// cells of each tile it recomputes (a label with kRes, or the slot of the
// exit where the cell's line leaves its tile), lw the entries being resolved.
// xm marks the slots that are exits of some tile's lines; only those are
// resolved (and looked up).
//
// k_jump: label propagation by pointer jumping over the marked slots of lw,
// which the label tiles restart from lf at every evaluation (recomputed
// tiles write both, the others copy theirs). A walk stores each pointer it
// reaches in its own entry, and all entries walk at once. A value read is the entry of an exit further along the same line, or
// the line's label, whether it was read before or after its owner advanced
// it, so every step makes progress and the other entries' stores shorten the
// walk (each read skips the steps its owner has taken). Loads of lw bypass
// L1 to see those stores. An entry takes at most A.chase steps per launch; a
// launch that leaves no pointer ends the labelling.
template <class T>
__global__ void __launch_bounds__(kThreads) k_jump(GroupArgs<T> A) {
  const int* pre = A.prefix + K_DENSE * (A.nf + 1);
  auto active = [](const Field<T>& F) { return F.st->action == ACT_LABELS && F.st->lstate == L_JUMP; };
  uint32_t open[1] = {0};
  auto pre_flush = [&](DevState* st) {
    block_add_striped<1>(open, st);
    open[0] = 0;
  };
  auto done = [&](DevState* st) {
    ctrl_after_jump(st);
    log_work(A);
  };
  UnitTally tl;
  MSZ_ACTIVE_UNITS(A, K_DENSE, pre, i, active) {
    tl.enter(A, K_DENSE, i, pre_flush, done);
    const Field<T>& F = A.fields[i];
    DevState* st = F.st;
    const uint64_t u = (uint64_t)(u_ - pre[i]), U = (uint64_t)F.units[K_DENSE];
    uint32_t acc = 0;
    constexpr int kJB = 4;  // entries per thread and iteration, their walks advanced together
    // The unit's share of both directions' slots taken as one range (all of
    // direction 0 before direction 1), so that the units in flight at a time
    // work mostly on one direction's tables.
    const uint32_t ne = F.nface, chunk = (2u * ne + (uint32_t)U - 1u) / (uint32_t)U;
    const uint32_t c0 = min(2u * ne, chunk * (uint32_t)u), c1 = min(2u * ne, c0 + chunk);
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      const uint32_t lo = max(c0, (uint32_t)d * ne), hi = min(c1, (uint32_t)(d + 1) * ne);
      const uint32_t r0 = lo - (uint32_t)d * ne, re = (hi > lo) ? hi - (uint32_t)d * ne : r0;
      uint32_t* lw = F.lw[d];
      const uint8_t* xm = F.xm[d];
      for (uint32_t rb = r0 + threadIdx.x; rb < re; rb += kJB * kThreads) {
        uint32_t x[kJB], mk = 0;  // mk bit k: entry k is an exit
#pragma unroll
        for (int k = 0; k < kJB; ++k) {
          const uint32_t r = rb + k * kThreads;
          if (r < re && xm[r]) mk |= 1u << k;
        }
#pragma unroll
        for (int k = 0; k < kJB; ++k) {
          const uint32_t r = rb + k * kThreads;
          x[k] = ((mk >> k) & 1u) ? __ldcg(lw + r) : kRes;
        }
        acc += (uint32_t)__popc(mk);
        for (int h = 0; h < A.chase; ++h) {
          uint32_t walk = 0;  // bit k: entry k still holds a pointer
#pragma unroll
          for (int k = 0; k < kJB; ++k) walk |= (x[k] & kRes) ? 0u : (1u << k);
          if (!walk) break;
#pragma unroll
          for (int k = 0; k < kJB; ++k)
            if ((walk >> k) & 1u) x[k] = MSZ_IN(st, x[k], ne) ? __ldcg(lw + x[k]) : kRes;
#pragma unroll
          for (int k = 0; k < kJB; ++k)
            if ((walk >> k) & 1u) lw[rb + k * kThreads] = x[k];
          acc += 2u * (uint32_t)__popc(walk);
        }
#pragma unroll
        for (int k = 0; k < kJB; ++k) open[0] += (x[k] & kRes) ? 0u : 1u;
      }
    }
    log_units_warp(A, st, KID_JUMP, acc);
  }
  tl.flush(A, K_DENSE, pre_flush, done);
}

// Labels from the tile terminals once the exit tables hold labels. Job 0:
// f's labels into Mf / mf. Job 1, the R-loop check (Sec. 4.2): count wrong
// labels; a wrongly labelled vertex whose steepest neighbour in g differs
// from f's is a troublemaker. Wrong max label: decrease its ascending
// neighbour in g (Eq. 6). Wrong min label: decrease the descending neighbour
// that f prescribes. Units are label tiles: a block first looks up the labels
// of the tile's shell cells that are exits (one (bitmap word, exits before
// it) load, and one table load per exit), then gives every vertex its labels
// from its terminals by a shared-memory lookup (or, for a line ending inside
// the tile, the extremum's index).
template <class T, int ND>
__global__ void __launch_bounds__(kThreads, 4) k_rcheck(GroupArgs<T> A) {
  using LG = LabelGeom<ND>;
  const int* pre = A.prefix + K_LABEL * (A.nf + 1);
  auto active = [](const Field<T>& F) { return F.st->action == ACT_LABELS && F.st->lstate == L_DONE; };
  uint32_t acc[4] = {0, 0, 0, 0};
  auto pre_flush = [&](DevState* st) {
    block_add_striped<4>(acc, st);
    acc[0] = acc[1] = acc[2] = acc[3] = 0;
  };
  auto done = [&](DevState* st) {
    if (st->ljob == 0) ctrl_after_flabels(st);
    else ctrl_after_rcheck(st);
    log_work(A);
  };
  // labels of the tile's shell cells (ascending, descending lines), and the
  // tile's exit record (which of them its lines leave through)
  __shared__ uint32_t s_lab[2][LG::SHELL];
  __shared__ uint32_t s_shx[2 * LabelGeom<ND>::SHW];
  __shared__ int s_slotd[LG::SHELL];  // shell cells' exit-table slots, relative (shell_slot_delta)
  int slot_field = -1;                // the field s_slotd was filled for
  // the tile's exits as bit positions of its record (direction * SHW * 32 +
  // shell index), and the scan sums that list them
  __shared__ uint16_t s_xl[2 * LG::SHELL];
  __shared__ uint32_t s_wsum[kThreads / 32];
  __shared__ uint32_t s_nxl;
  // Troublemakers whose request freezes a ring: their anchors, marked by
  // the block's warps at the end of the unit (a lane per ring vertex)
  // instead of vertex by vertex in one thread.
  constexpr uint32_t kRFreeze = 1024;
  __shared__ uint32_t s_fz[kRFreeze];
  __shared__ uint32_t s_nfz;
  // freezing requests of the unit by kind (wrong max, wrong min) and cause
  // (target frozen, target at its bound), added to the counters per unit
  __shared__ uint32_t s_fzc[2][2];
  // The unit's touched vertices, staged here and added to the field's list
  // with one atomic per unit (a single counter for the whole grid otherwise).
  constexpr uint32_t kRStage = 2048;
  __shared__ uint32_t s_tv[kRStage];
  __shared__ uint32_t s_ntv, s_base;
  TouchSink ts;
  ts.n = &s_ntv;
  ts.buf = s_tv;
  ts.cap = kRStage;
  if (threadIdx.x == 0) s_nfz = s_ntv = 0;
  if (threadIdx.x < 4) s_fzc[threadIdx.x >> 1][threadIdx.x & 1] = 0;
  UnitTally tl;
  MSZ_ACTIVE_UNITS(A, K_LABEL, pre, i, active) {
    tl.enter(A, K_LABEL, i, pre_flush, done);
    const Field<T>& F = A.fields[i];
    DevState* st = F.st;
    const Geom G = F.G;
    const int tiles_x = (G.nx + LG::TX - 1) / LG::TX;
    const int tiles_y = (G.ny + LG::TY - 1) / LG::TY;
    const int tile = u_ - pre[i];
    const int x0 = (tile % tiles_x) * LG::TX;
    const int y0 = ((tile / tiles_x) % tiles_y) * LG::TY;
    const int z0 = (tile / (tiles_x * tiles_y)) * LG::TZ;
    constexpr int kShW = LabelGeom<ND>::SHW;
    __syncthreads();  // the previous tile's tables have been read
    if (i != slot_field) {  // the same for every thread of the block
      fill_slot_table<ND>(s_slotd, G);
      slot_field = i;
    }
    for (int k = threadIdx.x; k < 2 * kShW; k += kThreads) s_shx[k] = F.texit[(size_t)tile * 2 * kShW + k];
    __syncthreads();
    // The tile's exits (the shell cells its lines leave through) listed in
    // shared memory, then their labels looked up a few per thread with the
    // loads in flight together, and compared with the tile's snapshot of
    // them from its last check (R-check only).
    const bool job = st->ljob != 0;
    int relabel = 0;
    {
      uint32_t bits = threadIdx.x < 2 * kShW ? s_shx[threadIdx.x] : 0u;
      const uint32_t cnt = (uint32_t)__popc(bits);
      uint32_t incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if ((threadIdx.x & 31) >= o) incl += y;
      }
      if ((threadIdx.x & 31) == 31) s_wsum[threadIdx.x >> 5] = incl;
      __syncthreads();
      uint32_t off = incl - cnt;
      for (int k = 0; k < (int)(threadIdx.x >> 5); ++k) off += s_wsum[k];
      for (; bits; bits &= bits - 1) s_xl[off++] = (uint16_t)(threadIdx.x * 32 + __ffs(bits) - 1);
      if (threadIdx.x == kThreads - 1) s_nxl = off;
      __syncthreads();
    }
    const uint32_t nxl = s_nxl;
    for (uint32_t j0 = threadIdx.x; j0 < nxl; j0 += 4 * kThreads) {
      int q[4];
      uint32_t lab[4], old[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t j = j0 + k * kThreads;
        q[k] = j < nxl ? (int)s_xl[j] : -1;
        const int d = q[k] >= kShW * 32 ? 1 : 0, s = q[k] - d * kShW * 32;
        uint32_t sl = q[k] >= 0 ? (uint32_t)tile * (uint32_t)LG::NFACE + (uint32_t)s_slotd[s] : 0u;
        if (!MSZ_IN(st, sl, F.nface)) sl = 0;
        lab[k] = q[k] >= 0 ? F.lw[d][sl] & ~kRes : 0u;
        // the snapshot is kept in the order of the tile's exit list, which
        // only changes when the tile is recomputed (and then examined)
        old[k] = (q[k] >= 0 && job) ? F.tsnap[(size_t)tile * 2 * LG::SHELL + j0 + k * kThreads] : 0u;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (q[k] < 0) continue;
        const int d = q[k] >= kShW * 32 ? 1 : 0, s = q[k] - d * kShW * 32;
        s_lab[d][s] = lab[k];
        if (job && old[k] != lab[k]) {
          F.tsnap[(size_t)tile * 2 * LG::SHELL + j0 + k * kThreads] = lab[k];
          relabel = 1;
        }
      }
    }
    // A tile whose terminals were not recomputed, whose exits kept their
    // labels and whose last check found no wrong label has none now: its
    // vertices' labels and direction bytes are those of that check (any edit
    // in the tile or its halo would have marked it for recomputation), so
    // it holds no troublemaker and adds nothing to the counts.
    const uint8_t tstate = job ? F.tdirty[tile] : 0;
    const bool examine = __syncthreads_or(relabel) || !job || (tstate & 2) || F.twrong[tile];
    // algorithmic bytes (kernel timing runs): each exit's table entry and
    // snapshot, and, for an examined tile, each vertex's terminal word and
    // f's two labels
    if (threadIdx.x == 0)
      log_units(A, st, KID_RCHECK,
                8ull * nxl + (examine ? 12ull * min(LG::TX, G.nx - x0) * min(LG::TY, G.ny - y0) *
                                             min(LG::TZ, G.nz - z0)
                                       : 0ull));
    if (!examine) continue;
    // label of one terminal half t (direction d) of a vertex of this tile
    auto label_of = [&](uint32_t t, int d) -> int32_t {
      return (t & kTermExtr) ? extremum_vertex<ND>(G, t, x0, y0, z0) : (int32_t)s_lab[d][t & kTermIdx];
    };
    // kRB vertices per thread and iteration, their loads issued together
    constexpr int kRB = 4;
    static_assert(LG::PER_THREAD % kRB == 0, "whole batches");
    const CellWalk<ND> cw;
    const int vs = cw.vstep(G);
    const int v0 = (x0 + cw.lx) + G.nx * ((y0 + cw.ly(0)) + G.ny * (z0 + cw.lz(0)));
    if (!job) {
#pragma unroll
      for (int kb = 0; kb < LG::PER_THREAD; kb += kRB) {
        int vv[kRB];
        uint32_t tt[kRB];
#pragma unroll
        for (int k = 0; k < kRB; ++k) {
          vv[k] = cw.inside(G, x0, y0, z0, kb + k) ? v0 + (kb + k) * vs : -1;
          tt[k] = vv[k] >= 0 ? F.term[vv[k]] : 0u;
        }
#pragma unroll
        for (int k = 0; k < kRB; ++k)
          if (vv[k] >= 0) {
            F.Mf[vv[k]] = label_of(tt[k] & 0xffffu, 0);
            F.mf[vv[k]] = label_of(tt[k] >> 16, 1);
          }
      }
      continue;
    }
    // the request of troublemaker a for target t (Eq. 6); k: 4 for a wrong
    // max label, 5 for a wrong min label
    auto trouble = [&](int a, int t, int k) {
      const int cause = request_cause(F, t);
      if (cause == RQ_DEC) {
        mark(F, t, FL_DEC, ts);
        return;
      }
      atomicAdd(&s_fzc[k - 4][cause - 1], 1u);
      const uint32_t q = atomicAdd(&s_nfz, 1u);
      if (q < kRFreeze) s_fz[q] = (uint32_t)a;
      else request<T, ND>(F, a, t, ts);  // list full: the same freeze, vertex by vertex
    };
    uint32_t any_wrong = 0;
#pragma unroll 1
    for (int kb = 0; kb < LG::PER_THREAD; kb += kRB) {
      int vv[kRB];
      uint32_t tt[kRB];
      int32_t M[kRB], m[kRB];
#pragma unroll
      for (int k = 0; k < kRB; ++k) {
        vv[k] = cw.inside(G, x0, y0, z0, kb + k) ? v0 + (kb + k) * vs : -1;
        const bool in = vv[k] >= 0;
        tt[k] = in ? F.term[vv[k]] : 0u;
        M[k] = in ? F.Mf[vv[k]] : 0;
        m[k] = in ? F.mf[vv[k]] : 0;
      }
      uint32_t wrong = 0;  // bit 2k: max label wrong, bit 2k+1: min label wrong
#pragma unroll
      for (int k = 0; k < kRB; ++k)
        if (vv[k] >= 0)
          wrong |= ((uint32_t)(label_of(tt[k] & 0xffffu, 0) != M[k]) << (2 * k)) |
                   ((uint32_t)(label_of(tt[k] >> 16, 1) != m[k]) << (2 * k + 1));
      any_wrong |= wrong;
      for (; wrong; wrong &= wrong - 1) {
        const int bit = __ffs(wrong) - 1;
        int v = vv[0];  // vv[bit >> 1], selected without indexing the array
#pragma unroll
        for (int k = 1; k < kRB; ++k)
          if ((bit >> 1) == k) v = vv[k];
        const uint8_t d = F.gdir[v], fd = F.fdir[v];
        if ((bit & 1) == 0) {
          ++acc[0];
          if ((d & 15) != (fd & 15)) {
            ++acc[2];
            trouble(v, v + slot_offset(d & 15, ND, G.nx, G.nxny), 4);
          }
        } else {
          ++acc[1];
          if ((d >> 4) != (fd >> 4)) {
            ++acc[3];
            trouble(v, v + slot_offset(fd >> 4, ND, G.nx, G.nxny), 5);
          }
        }
      }
    }
    const int tile_wrong = __syncthreads_or(any_wrong != 0u);
    if (threadIdx.x == 0) {
      F.twrong[tile] = (uint8_t)tile_wrong;
      if (tstate & 2) F.tdirty[tile] = 0;
    }
    if (threadIdx.x < 4) {
      // k: wrong max / min label; c: 0 target frozen, 1 target at its bound
      const int k = threadIdx.x >> 1, c = threadIdx.x & 1;
      const uint32_t n = s_fzc[k][c];
      if (n) {
        s_fzc[k][c] = 0;  // read by this thread alone
        atomicAdd((unsigned long long*)&st->cnt.freeze_req[4 + k], (unsigned long long)n);
        if (c == 0) atomicAdd((unsigned long long*)&st->cnt.freeze_req_frozen[4 + k], (unsigned long long)n);
      }
    }
    const uint32_t nfz = min(s_nfz, kRFreeze);
    if (nfz) {
      __syncthreads();  // every thread has read the count
      if (threadIdx.x == 0) s_nfz = 0;
      for (uint32_t q = threadIdx.x >> 5; q < nfz; q += kThreads / 32)
        freeze_ring_warp<T, ND>(F, (int)s_fz[q], (int)(threadIdx.x & 31), ts);
      __syncthreads();  // the list is free for the next unit
    }
    const uint32_t ntv = min(s_ntv, kRStage);
    if (ntv) {
      __syncthreads();  // every thread has read the count
      if (threadIdx.x == 0) {
        s_base = atomicAdd(&st->ntouch, ntv);
        s_ntv = 0;
      }
      __syncthreads();
      for (uint32_t j = threadIdx.x; j < ntv; j += kThreads)
        if (MSZ_IN(st, s_base + j, G.n)) F.touched[s_base + j] = s_tv[j];
      __syncthreads();  // the buffer is free for the next unit
    }
  }
  tl.flush(A, K_LABEL, pre_flush, done);
}

// Applies the flags of touched vertex u: a freeze sets g = f and freezes u
// (acc[1]), a decrease halves g towards the lower bound (acc[0]); the label
// tiles around u are marked dirty.
template <class T>
__device__ __forceinline__ void apply_vertex(const Field<T>& F, int u, uint32_t (&acc)[2]) {
  // u's flags, g and f loaded together (one round trip, not two); no other
  // thread writes them during the apply
  uint8_t bb = F.flags[u];
  const T gu = F.g[u], fu = F.f[u];
  if (bb & FL_FREEZE) {
    F.g[u] = fu;
    bb = (uint8_t)((bb & ~(FL_DEC | FL_FREEZE)) | FL_FROZEN | FL_EDITED);
    ++acc[1];
  } else if (bb & FL_DEC) {
    F.g[u] = decrease(gu, lower_bound_of(fu, F.xi));
    bb = (uint8_t)((bb & ~FL_DEC) | FL_EDITED);
    ++acc[0];
  }
  F.flags[u] = bb;
  if (F.G.nd == 3) mark_dirty_tiles<3>(F.tdirty, F.G, u);
  else mark_dirty_tiles<2>(F.tdirty, F.G, u);
}

// Applies a round's requests to the touched vertices only. Units are slices
// of the touched list.
template <class T>
__global__ void __launch_bounds__(kThreads) k_apply(GroupArgs<T> A) {
  const int* pre = A.prefix + K_SPARSE * (A.nf + 1);
  auto active = [](const Field<T>& F) { return F.st->action == ACT_MARK_C || F.st->action == ACT_APPLY_R; };
  uint32_t acc[2] = {0, 0};
  auto pre_flush = [&](DevState* st) {
    block_add_striped<2>(acc, st);
    acc[0] = acc[1] = 0;
  };
  auto done = [&](DevState* st) {
    ctrl_after_apply(st, st->action);  // the action this launch applied
    log_work(A);
  };
  UnitTally tl;
  MSZ_ACTIVE_UNITS(A, K_SPARSE, pre, i, active) {
    const Field<T>& F = A.fields[i];
    DevState* st = F.st;
    uint64_t b64, e64;
    const uint32_t act = sparse_slice(st->ntouch, F.units[K_SPARSE], u_ - pre[i], b64, e64);
    if ((uint32_t)(u_ - pre[i]) >= act) continue;  // left out: not counted
    tl.enter(A, K_SPARSE, i, pre_flush, done);
    tl.target = act;
    const uint32_t b = (uint32_t)b64, e = (uint32_t)e64;
    if (threadIdx.x == 0) log_units(A, st, KID_APPLY, e - b);
    for (uint32_t j = b + threadIdx.x; j < e; j += blockDim.x) {
      const uint32_t u = F.touched[j];
      if (MSZ_IN(st, u, F.G.n)) apply_vertex(F, (int)u, acc);
    }
  }
  tl.flush(A, K_SPARSE, pre_flush, done);
}

// ---------------------------------------------------------------------------
// Small C-loop rounds (Sec. 4.1) in one thread-block cluster per field. Most
// rounds of a fix hold a few thousand cases or fewer, where four grid-wide
// launches per round are mostly latency. This kernel takes a field whose
// listed round is small and runs whole rounds - requests, apply,
// reclassification, the next round's case list - with cluster barriers
// between the steps, through the same state transitions and counters as the
// grid kernels. The next list is the current one without the vertices that
// lost the type plus those the reclassification gave it: every vertex of the
// type, the set a gather lists. The field goes back to the grid kernels (with
// its cases listed, a type to gather, or the R-loop) when a round outgrows
// the cluster, the type changes, or after A.small_rounds rounds. The cluster's
// counters live in the shared memory of its block 0.
// ---------------------------------------------------------------------------
constexpr int kSmallThreads = 1024;
constexpr int kSmallCluster = 16;     // blocks per field (a non-portable cluster size)
constexpr int kSmallClusterLite = 4;  // blocks per small field of an engine with many fields
// In an engine with more fields than 16-block clusters fit on the device at
// once, fields of at most kSmallLiteVertices vertices take a 4-block cluster:
// their rounds rarely hold more cases than it does, and a quarter of the SMs
// per field lets four times as many fields run their rounds at once.
constexpr int kSmallLiteVertices = 1 << 22;
constexpr uint32_t kSmallSpan = (uint32_t)kSmallThreads * kSmallCluster;
constexpr int kSmallPer = 4;  // cases per thread
constexpr uint32_t kSmallCases = kSmallSpan * kSmallPer;  // the most a launch can hold (A.small_cases <= this)

// Barrier of the cluster, release / acquire at cluster scope: every memory
// access (global or shared) before it happens before those after it in all
// of the cluster's threads.
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// The address of shared variable p in the cluster's block 0.
__device__ __forceinline__ uint32_t* in_block0(uint32_t* p) {
  return cooperative_groups::this_cluster().map_shared_rank(p, 0);
}

// Adds each thread's n counters into s[0 .. n-1] (shared memory of this or
// another block of the cluster), one atomic per warp.
template <int N>
__device__ __forceinline__ void warp_add_shared(const uint32_t (&v)[N], uint32_t* s) {
#pragma unroll
  for (int k = 0; k < N; ++k) {
    uint32_t x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(&s[k], x);
  }
}

template <class T, int ND, int CS>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(kSmallThreads) k_csmall(GroupArgs<T> A) {
  constexpr uint32_t kSpan = (uint32_t)kSmallThreads * CS;  // the cluster's threads
  const int fi = (int)blockIdx.x / CS;  // a cluster per field
  if (fi >= A.nf) return;
  const Field<T>& F = A.fields[fi];
  if (F.small_cluster != CS) return;  // the field's rounds run in the other cluster size
  DevState* st = F.st;
  // the same for the whole cluster: nothing writes the state before the first barrier
  const uint32_t cap = min(A.small_cases, kSpan * kSmallPer);
  if (!(st->phase == PH_C && st->action == ACT_REQUEST && st->ncase <= cap)) return;
  // The sub-loop's type stays while the cluster runs (a round of another type
  // goes back to the grid), and each round adds one to st->rounds.
  const uint32_t type = st->T;
  uint64_t r1 = st->rounds;
  const uint64_t max_rounds = st->max_rounds;
  constexpr int NPOS = Slots<ND>::NPOS;
  constexpr int R = 2 * NPOS + 1;
  // block 0's: touched count, freezes, next list length, 1 + the round's case
  // count (0: stop), apply sums (2), count changes (4)
  __shared__ uint32_t s_ctl[10];
  uint32_t* const C = in_block0(s_ctl);
  TouchSink ts;
  ts.n = &C[0];  // the cluster counts the round's touched list itself
  const uint32_t gt = cluster_rank() * kSmallThreads + threadIdx.x;
  // the bookkeeping thread's copy of the type counts (it alone writes them
  // during the launch), and whether the field has timed out
  uint32_t cnt[4] = {0, 0, 0, 0};
  bool timeout = false;
  if (gt == 0) {
    for (int k = 0; k < 10; ++k) C[k] = 0;
    C[3] = st->ncase + 1;
    for (int c = 0; c < 4; ++c) cnt[c] = st->counts[c];
    timeout = (vload(&st->err_bits) & E_TIMEOUT) != 0;
  }
  uint32_t rounds = 0;
  for (int it = 0; it < A.small_rounds; ++it) {
    cluster_barrier();  // the round's case list, state and counters are in place
    const uint32_t go = C[3];
    if (!go) break;
    const uint32_t nc = go - 1;
    ++r1;  // the round's number once applied
    // requests (Eqs. 2-5) for this thread's cases, all from one snapshot of
    // g: decreases at once; freezes are listed (lw[0], idle in the C-loop)
    // for the warps below, since a freeze marks a whole ring
    int cv[kSmallPer];
#pragma unroll
    for (int k = 0; k < kSmallPer; ++k) {
      const uint32_t j = gt + (uint32_t)k * kSpan;
      cv[k] = j < nc ? (int)F.cases[j] : -1;
      if (cv[k] >= 0 && !MSZ_IN(st, cv[k], F.G.n)) cv[k] = -1;
    }
#pragma unroll
    for (int k = 0; k < kSmallPer; ++k) {
      if (cv[k] < 0) continue;
      const int v = cv[k];
      const int t = (type == FPMAX || type == FNMIN) ? v : v + slot_offset(F.gdir[v] & 15, ND, F.G.nx, F.G.nxny);
      const int cause = request_cause(F, t);
      if (cause == RQ_DEC) {
        mark(F, t, FL_DEC, ts);
      } else {
        count_freeze_req(st, (int)type, cause);
        const uint32_t q = atomicAdd(&C[1], 1u);
        if (MSZ_IN(st, q, F.fz_cap)) F.lw[0][q] = (uint32_t)v;
      }
    }
    cluster_barrier();
    if (const uint32_t nfz = C[1]) {
      // a warp per freeze, a lane per vertex of the anchor's closed ring
      for (uint32_t q = gt >> 5; q < nfz; q += kSpan >> 5)
        freeze_ring_warp<T, ND>(F, (int)F.lw[0][q], (int)(threadIdx.x & 31), ts);
      cluster_barrier();
    }
    const uint32_t nt = C[0];
    {
      uint32_t acc[2] = {0, 0};
      for (uint32_t j = gt; j < nt; j += kSpan) {
        const uint32_t u = F.touched[j];
        if (MSZ_IN(st, u, F.G.n)) apply_vertex(F, (int)u, acc);
      }
      warp_add_shared<2>(acc, C + 4);
    }
    cluster_barrier();
    if (gt == 0) ctrl_after_apply_small(st, type, C[4], C[5], cnt[type], nt, r1, max_rounds);
    if (r1 > max_rounds) break;  // the round cap: the bookkeeping above ends the fix
    {
      // Reclassification, and the next list in the same pass: every vertex
      // the round claims (the closed rings of the touched vertices, and this
      // round's cases, each claimed by the thread holding it) is listed by
      // its claimer when it has the type after the apply. A vertex no item
      // claims kept its bits and was no case, so the list ends up holding
      // every vertex of the type. The old cases are in registers, so the
      // list is written over them. Ring items run from the top of the
      // cluster's threads down, the cases sit at the bottom.
      const uint32_t stamp = (uint32_t)r1;
      uint32_t acc[4] = {0, 0, 0, 0};
      auto list = [&](uint32_t ch, int vc) {
        if ((ch >> type) & 1u) {
          const uint32_t q = atomicAdd(&C[2], 1u);
          if (MSZ_IN(st, q, F.G.n)) F.cases[q] = (uint32_t)vc;
        }
      };
      for (uint32_t j = kSpan - 1 - gt; j < nt * R; j += kSpan) {
        int vc = 0;
        const uint32_t u = F.touched[j / R];
        list(MSZ_IN(st, u, F.G.n) ? reclass_item<T, ND>(F, (int)u, (int)(j % R), stamp, acc, vc) : 0u, vc);
      }
#pragma unroll
      for (int k = 0; k < kSmallPer; ++k)
        if (cv[k] >= 0) {
          int vc = 0;
          list(reclass_item<T, ND>(F, cv[k], 2 * NPOS, stamp, acc, vc), vc);
        }
      warp_add_shared<4>(acc, C + 6);
    }
    cluster_barrier();
    ++rounds;
    if (gt == 0) {
      for (int c = 0; c < 4; ++c) cnt[c] += C[6 + c];
      // go on with the same type while its round stays small and the list
      // holds every vertex of the type; otherwise the grid's gather lists it
      const uint32_t len = C[2];
      const bool more = ctrl_after_classify_small(st, type, cnt, len, cap, timeout);
      for (int k = 0; k < 10; ++k) C[k] = 0;
      C[3] = more ? len + 1 : 0;
    }
  }
  // block 0's shared memory stays until every block is done with it
  cluster_barrier();
  if (gt == 0 && rounds) {
    log_units(A, st, KID_CSMALL, rounds);
    log_work(A);
  }
}

// ---------------------------------------------------------------------------
// Edit list (Sec. 5.3): every vertex whose final value differs bitwise from
// fhat, ascending. Count per tile, scan per field, write.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ bool bits_differ(T a, T b);
template <>
__device__ __forceinline__ bool bits_differ<float>(float a, float b) {
  return __float_as_uint(a) != __float_as_uint(b);
}
template <>
__device__ __forceinline__ bool bits_differ<double>(double a, double b) {
  return __double_as_longlong(a) != __double_as_longlong(b);
}

// Fields whose edit list is written: converged ones, and ones stopped by
// the round cap (their edits so far).
__device__ __forceinline__ bool emit_wanted(const DevState* st) {
  return !st->emitted && (st->phase == PH_DONE || (st->phase == PH_ERR && st->status == MSZ_ERR_NOCONVERGE));
}

template <class T>
__device__ __forceinline__ uint32_t emit_mask(const Field<T>& F, int base) {
  const uint4 wv = *reinterpret_cast<const uint4*>(F.flags + base);
  const uint32_t ws[4] = {wv.x, wv.y, wv.z, wv.w};
  uint32_t m = 0;
#pragma unroll
  for (int k = 0; k < kEmitItems; ++k) {
    const uint32_t byte = (ws[k >> 2] >> ((k & 3) * 8)) & 0xffu;
    if (byte & FL_EDITED) {
      const int v = base + k;
      if (v < F.G.n && bits_differ(F.g[v], F.fhat[v])) m |= 1u << k;
    }
  }
  return m;
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_emit_count(GroupArgs<T> A) {
  const int* pre = A.prefix + K_EMIT * (A.nf + 1);
  __shared__ uint32_t s;
  auto active = [](const Field<T>& F) { return emit_wanted(F.st); };
  MSZ_ACTIVE_UNITS(A, K_EMIT, pre, i, active) {
    const Field<T>& F = A.fields[i];
    const int tile = u_ - pre[i];
    const int base = tile * kEmitTile + threadIdx.x * kEmitItems;
    // (the final labels are already in place: f's, resolved into the
    // output arrays, which g's equal once the loop has converged)
    __syncthreads();
    if (threadIdx.x == 0) s = 0;
    __syncthreads();
    uint32_t x = __popc(emit_mask(F, base));
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s, x);
    __syncthreads();
    if (threadIdx.x == 0) F.tile_cnt[tile] = s;
  }
}

// Exclusive scan of one field's tile counts per block (grid = nf).
template <class T>
__global__ void __launch_bounds__(1024) k_emit_scan(GroupArgs<T> A) {
  const Field<T>& F = A.fields[blockIdx.x];
  DevState* st = F.st;
  if (!emit_wanted(st)) return;
  const int ntiles = F.units[K_EMIT];
  __shared__ uint32_t warp_sums[32];
  __shared__ uint32_t carry_s;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base < ntiles; base += 1024) {
    const int i = base + threadIdx.x;
    const uint32_t x = (i < ntiles) ? F.tile_cnt[i] : 0u;
    uint32_t incl = x;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      uint32_t wsum = warp_sums[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, wsum, o);
        if (lane >= o) wsum += y;
      }
      warp_sums[lane] = wsum;
    }
    __syncthreads();
    const uint32_t carry = carry_s;
    const uint32_t warp_off = wid ? warp_sums[wid - 1] : 0u;
    if (i < ntiles) F.tile_cnt[i] = carry + warp_off + incl - x;
    __syncthreads();
    if (threadIdx.x == 0) carry_s = carry + warp_sums[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    st->n_edits = carry_s;
    st->cnt.edits = carry_s;
  }
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_emit_write(GroupArgs<T> A) {
  const int* pre = A.prefix + K_EMIT * (A.nf + 1);
  __shared__ uint32_t ws[kThreads / 32];
  auto active = [](const Field<T>& F) { return emit_wanted(F.st); };
  MSZ_ACTIVE_UNITS(A, K_EMIT, pre, fi, active) {
    const Field<T>& F = A.fields[fi];
    DevState* st = F.st;
    const int tile = u_ - pre[fi];
    const int base = tile * kEmitTile + threadIdx.x * kEmitItems;
    const uint32_t m = emit_mask(F, base);
    const uint32_t c = __popc(m);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t incl = c;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    __syncthreads();
    if (lane == 31) ws[wid] = incl;
    __syncthreads();
    uint32_t off = F.tile_cnt[tile] + incl - c;
    for (int wv = 0; wv < wid; ++wv) off += ws[wv];
    uint32_t mm = m;
    while (mm) {
      const int k = __ffs(mm) - 1;
      mm &= mm - 1;
      const int v = base + k;
      if (MSZ_IN(st, off, F.G.n)) {
        F.edit_idx[off] = (uint32_t)v;
        F.edit_val[off] = F.g[v];
      }
      ++off;
    }
    if (unit_done(st, F.units[K_EMIT]) && threadIdx.x == 0) {
      st->emitted = 1;
      st->units_done = 0;
    }
  }
}

// Standalone direction kernel (msz_directions).
template <class T, int ND>
__global__ void __launch_bounds__(kThreads) k_directions(const T* __restrict__ g, Geom G, uint8_t* out) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < G.n; v += gridDim.x * blockDim.x) {
    int x, y, z;
    coords(G, v, x, y, z);
    out[v] = direction_of<T, ND>(g, G, v, x, y, z);
  }
}

// Decompression-side scatter (msz_apply).
template <class T>
__global__ void __launch_bounds__(kThreads) k_scatter(T* dst, int n, const uint32_t* idx, const T* val,
                                                      uint64_t ne, uint32_t* bad) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < ne; k += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t i = idx[k];
    if (i < (uint32_t)n) dst[i] = val[k];
    else atomicOr(bad, 1u);
  }
}

#undef MSZ_ACTIVE_UNITS

}  // namespace msz
