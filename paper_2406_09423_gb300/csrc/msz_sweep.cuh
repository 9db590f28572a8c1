// C-loop sweep: extremum classification of every vertex of g and detection
// of the four false critical point types (Sec. 4.1 Definitions 1-3; the
// "find false critical points" and "update directions" steps of Sec. 5.1).
//
// GB300 design. A vertex v is the greatest of its closed Freudenthal ring iff
//   g_v > max(U*(v))  and  g_v >= max(L*(v)),
// where U*(v) = v + ({0,1}^d \ 0) holds the neighbours of larger index and
// L*(v) = v - ({0,1}^d \ 0) those of smaller index (ties go to the larger
// index); symmetrically for the least. Both sets are unit cubes minus a corner,
// so their max/min are built separably from row pairs and 2x2 squares of each
// plane: about twenty FMNMX per vertex instead of a 14-way argmax with index
// tie-breaks. Out-of-grid vertices are NaN, which fmax/fmin ignore, and an
// empty set gives NaN, which the negated comparisons treat as "no neighbour".
//
// Data movement: a block owns an x-y tile and marches along z (3D; rows
// along y in 2D). Each plane of the tile plus a one-vertex halo (widened in x
// to a 16-byte multiple) is fetched by TMA (cp.async.bulk.tensor) into a
// ring of shared-memory stages guarded by mbarriers; the tensor map's
// out-of-bounds fill supplies the NaN halo. Grids whose row pitch is not a
// multiple of 16 bytes use the same kernel with plain coalesced loads.
// The original field's extremum flags come from its direction bytes, fetched
// through the same stages (a second tensor map), so the sweep reads 5 bytes
// per float32 vertex and writes only the (sparse) case list.
#pragma once

#include <cuda.h>

#include "msz_device.cuh"

namespace msz {

__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double vmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ double vmin(double a, double b) { return fmin(a, b); }

template <class T>
__device__ __forceinline__ T qnan();
template <>
__device__ __forceinline__ float qnan<float>() { return __int_as_float(0x7fc00000); }
template <>
__device__ __forceinline__ double qnan<double>() { return __longlong_as_double(0x7ff8000000000000ll); }

// Tile geometry. PADX keeps the TMA box start and width 16-byte aligned.
// 3D: a block of 256 threads covers 32 x 16 vertices of a plane, two rows per
// thread (rows 2w, 2w+1 for warp w). 2D: 128 threads cover 128 vertices of a
// row, one per thread.
template <class T, int ND>
struct SweepGeom {
  static constexpr int PADX = 16 / (int)sizeof(T);
  static constexpr int TX = (ND == 3) ? 32 : 128;
  static constexpr int RPT = (ND == 3) ? 2 : 1;   // rows per thread
  static constexpr int TY = (ND == 3) ? 16 : 1;
  static constexpr int NT = (ND == 3) ? 256 : 128;
  static constexpr int BX = TX + 2 * PADX;
  static constexpr int BY = (ND == 3) ? TY + 2 : 1;
  static constexpr int STAGE_ELEMS = BX * BY;
  static constexpr int G_BYTES = ((STAGE_ELEMS * (int)sizeof(T) + 127) / 128) * 128;
  static constexpr int D_BYTES = ((TX * TY + 127) / 128) * 128;  // f's direction bytes of the tile plane
  static constexpr int STAGE_BYTES = G_BYTES + D_BYTES;
  static constexpr int STAGES = (ND == 3) ? 8 : 4;
};

struct SweepTiling {
  int tiles_x, tiles_y, chunks, chunk, ntiles;  // chunk = planes (3D) or rows (2D) per tile
};

// ---------------------------------------------------------------------------
// mbarrier / TMA primitives (inline PTX, sm_90+)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false if the phase did not complete within the limit.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < (1u << 26); ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                            int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
      "%4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// Per-plane quantities of one thread's vertices (RPT rows, see the header
// comment): the values the plane contributes when it is the vertex's own
// plane (A), the next plane (B) or the previous plane (C).
template <class T, int RPT>
struct PlaneVals {
  T a0[RPT], am[RPT], ap[RPT];   // g at (x, y), (x-1, y), (x+1, y)
  T rupM[RPT], rupm[RPT];        // max/min of row y+1, columns x..x+1     (3D only)
  T rdnM[RPT], rdnm[RPT];        // max/min of row y-1, columns x-1..x     (3D only)
  T supM[RPT], supm[RPT];        // max/min of square x..x+1 by y..y+1 (3D); x..x+1 (2D)
  T sdnM[RPT], sdnm[RPT];        // max/min of square x-1..x by y-1..y (3D); x-1..x (2D)
};

// Reads the thread's neighbourhood from a staged plane and derives the
// row-pair and square extrema. 3D: rows 2w-1 .. 2w+2 (stage rows 2w .. 2w+3)
// at columns x-1, x, x+1; each row pair is computed once for both vertices.
template <class T, int ND>
__device__ __forceinline__ PlaneVals<T, SweepGeom<T, ND>::RPT> plane_vals(const T* s, int tx, int w) {
  using SG = SweepGeom<T, ND>;
  PlaneVals<T, SG::RPT> P;
  const int c = tx + SG::PADX;
  if constexpr (ND == 3) {
    const T* r0 = s + (2 * w) * SG::BX + c;  // row y-1
    T a[4][3];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      a[r][0] = r0[r * SG::BX - 1];
      a[r][1] = r0[r * SG::BX];
      a[r][2] = r0[r * SG::BX + 1];
    }
    // hi pair: columns x..x+1; lo pair: columns x-1..x
    T hiM[4], him[4], loM[4], lom[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      hiM[r] = vmax(a[r][1], a[r][2]);
      him[r] = vmin(a[r][1], a[r][2]);
      loM[r] = vmax(a[r][0], a[r][1]);
      lom[r] = vmin(a[r][0], a[r][1]);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {  // vertex row = r k+1
      P.a0[k] = a[k + 1][1];
      P.am[k] = a[k + 1][0];
      P.ap[k] = a[k + 1][2];
      P.rupM[k] = hiM[k + 2];
      P.rupm[k] = him[k + 2];
      P.rdnM[k] = loM[k];
      P.rdnm[k] = lom[k];
      P.supM[k] = vmax(hiM[k + 1], hiM[k + 2]);
      P.supm[k] = vmin(him[k + 1], him[k + 2]);
      P.sdnM[k] = vmax(loM[k], loM[k + 1]);
      P.sdnm[k] = vmin(lom[k], lom[k + 1]);
    }
  } else {
    const T* m0 = s + c;
    P.a0[0] = m0[0];
    P.am[0] = m0[-1];
    P.ap[0] = m0[1];
    P.rupM[0] = P.rupm[0] = P.rdnM[0] = P.rdnm[0] = P.a0[0];  // unused in 2D
    P.supM[0] = vmax(P.a0[0], P.ap[0]);
    P.supm[0] = vmin(P.a0[0], P.ap[0]);
    P.sdnM[0] = vmax(P.am[0], P.a0[0]);
    P.sdnm[0] = vmin(P.am[0], P.a0[0]);
  }
  return P;
}

// Extremum flags of the thread's k-th vertex of plane A, with B the next
// plane (larger indices) and C the previous one. Bit 0: maximum, bit 1:
// minimum (closed-ring order with ties to the larger index).
template <class T, int ND, int RPT>
__device__ __forceinline__ unsigned extremum_bits(const PlaneVals<T, RPT>& C, const PlaneVals<T, RPT>& A,
                                                  const PlaneVals<T, RPT>& B, int k) {
  T maxU, maxL, minU, minL;
  if constexpr (ND == 3) {
    maxU = vmax(A.ap[k], vmax(A.rupM[k], B.supM[k]));
    maxL = vmax(A.am[k], vmax(A.rdnM[k], C.sdnM[k]));
    minU = vmin(A.ap[k], vmin(A.rupm[k], B.supm[k]));
    minL = vmin(A.am[k], vmin(A.rdnm[k], C.sdnm[k]));
  } else {
    maxU = vmax(A.ap[k], B.supM[k]);
    maxL = vmax(A.am[k], C.sdnM[k]);
    minU = vmin(A.ap[k], B.supm[k]);
    minL = vmin(A.am[k], C.sdnm[k]);
  }
  const T g = A.a0[k];
  const bool is_max = !(maxU >= g) && !(maxL > g);
  const bool is_min = !(minU < g) && !(minL <= g);
  return (unsigned)is_max | ((unsigned)is_min << 1);
}

}  // namespace msz
