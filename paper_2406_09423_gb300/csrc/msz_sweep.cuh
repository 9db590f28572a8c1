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
template <class T, int ND>
struct SweepGeom {
  static constexpr int PADX = 16 / (int)sizeof(T);
  static constexpr int TX = (ND == 3) ? 32 : 128;
  static constexpr int TY = (ND == 3) ? 8 : 1;
  static constexpr int NT = TX * TY;
  static constexpr int BX = TX + 2 * PADX;
  static constexpr int BY = (ND == 3) ? TY + 2 : 1;
  static constexpr int STAGE_ELEMS = BX * BY;
  static constexpr int G_BYTES = ((STAGE_ELEMS * (int)sizeof(T) + 127) / 128) * 128;
  static constexpr int D_BYTES = ((NT + 127) / 128) * 128;  // f's direction bytes of the tile plane
  static constexpr int STAGE_BYTES = G_BYTES + D_BYTES;
  static constexpr int STAGES = 4;
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

// Per-plane quantities of one thread's column (see the header comment).
template <class T>
struct PlaneVals {
  T a0, am, ap;          // g at (x, y), (x-1, y), (x+1, y)
  T rup_max, rup_min;    // row y+1, columns x..x+1          (3D only)
  T rdn_max, rdn_min;    // row y-1, columns x-1..x          (3D only)
  T sup_max, sup_min;    // square x..x+1 by y..y+1 (3D); x..x+1 (2D)
  T sdn_max, sdn_min;    // square x-1..x by y-1..y (3D); x-1..x (2D)
};

template <class T, int ND>
__device__ __forceinline__ PlaneVals<T> plane_vals(const T* s, int tx, int ty) {
  using SG = SweepGeom<T, ND>;
  PlaneVals<T> P;
  const int c = tx + SG::PADX;
  if (ND == 3) {
    const int r = ty + 1;
    const T* m1 = s + (r - 1) * SG::BX + c;
    const T* m0 = s + r * SG::BX + c;
    const T* p1 = s + (r + 1) * SG::BX + c;
    P.a0 = m0[0];
    P.am = m0[-1];
    P.ap = m0[1];
    const T u0 = p1[0], u1 = p1[1], d0 = m1[-1], d1 = m1[0];
    P.rup_max = vmax(u0, u1);
    P.rup_min = vmin(u0, u1);
    P.rdn_max = vmax(d0, d1);
    P.rdn_min = vmin(d0, d1);
    P.sup_max = vmax(vmax(P.a0, P.ap), P.rup_max);
    P.sup_min = vmin(vmin(P.a0, P.ap), P.rup_min);
    P.sdn_max = vmax(vmax(P.am, P.a0), P.rdn_max);
    P.sdn_min = vmin(vmin(P.am, P.a0), P.rdn_min);
  } else {
    const T* m0 = s + c;
    P.a0 = m0[0];
    P.am = m0[-1];
    P.ap = m0[1];
    P.rup_max = P.rup_min = P.rdn_max = P.rdn_min = P.a0;  // unused in 2D
    P.sup_max = vmax(P.a0, P.ap);
    P.sup_min = vmin(P.a0, P.ap);
    P.sdn_max = vmax(P.am, P.a0);
    P.sdn_min = vmin(P.am, P.a0);
  }
  return P;
}

// Extremum flags of the vertex at the centre of plane A, with B the next
// plane (larger indices) and C the previous one. Bit 0: maximum, bit 1:
// minimum (closed-ring order with ties to the larger index).
template <class T, int ND>
__device__ __forceinline__ unsigned extremum_bits(const PlaneVals<T>& C, const PlaneVals<T>& A,
                                                  const PlaneVals<T>& B) {
  T maxU, maxL, minU, minL;
  if (ND == 3) {
    maxU = vmax(A.ap, vmax(A.rup_max, B.sup_max));
    maxL = vmax(A.am, vmax(A.rdn_max, C.sdn_max));
    minU = vmin(A.ap, vmin(A.rup_min, B.sup_min));
    minL = vmin(A.am, vmin(A.rdn_min, C.sdn_min));
  } else {
    maxU = vmax(A.ap, B.sup_max);
    maxL = vmax(A.am, C.sdn_max);
    minU = vmin(A.ap, B.sup_min);
    minL = vmin(A.am, C.sdn_min);
  }
  const T g = A.a0;
  const bool is_max = !(maxU >= g) && !(maxL > g);
  const bool is_min = !(minU < g) && !(minL <= g);
  return (unsigned)is_max | ((unsigned)is_min << 1);
}

}  // namespace msz
