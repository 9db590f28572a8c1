// C-loop sweep: extremum classification of every vertex of g and detection
// of the four false critical point types (Sec. 4.1 Definitions 1-3; the
// false-critical-point and direction-update steps of Sec. 5.1).
//
// GB300 design. A vertex v is the greatest of its closed Freudenthal ring iff
//   g_v > max(U*(v))  and  g_v >= max(L*(v)),
// where U*(v) = v + ({0,1}^d \ 0) holds the neighbours of larger index and
// L*(v) = v - ({0,1}^d \ 0) those of smaller index (ties go to the larger
// index); symmetrically for the least. With A the plane of v, B the next and
// C the previous plane, and the "L" corners
//   LUR_P(x,y) = {P(x+1,y), P(x,y+1), P(x+1,y+1)},
//   LLL_P(x,y) = {P(x-1,y), P(x,y-1), P(x-1,y-1)}
// (in 2D, where planes are rows: LUR_P(x) = {P(x+1)}, LLL_P(x) = {P(x-1)}),
//   U*(v) = LUR_A u {B(x,y)} u LUR_B,   L*(v) = LLL_A u {C(x,y)} u LLL_C,
// so each plane contributes one three-input max and min per vertex and the
// test costs about a dozen FMNMX/FSETP per vertex. Out-of-grid vertices are
// NaN, which max/min ignore; an empty set gives NaN, which the negated
// comparisons treat as "no neighbour".
//
// Data movement: a block owns an x-y tile and marches along z (3D; rows
// along y in 2D). Each plane of the tile plus a one-vertex halo (widened in x
// to a 16-byte multiple) is fetched by TMA (cp.async.bulk.tensor) into a
// ring of shared-memory stages guarded by full/empty mbarriers; a producer
// warp issues the copies and the tensor map's out-of-bounds fill supplies
// the NaN halo. Grids whose row pitch is not a multiple of 16 bytes use the
// same kernel with plain coalesced loads. The original field's extremum
// flags come from its direction bytes, fetched through the same stages (a
// second tensor map), so the sweep reads 5 bytes per float32 vertex and
// writes only the (sparse) case list.
#pragma once

#include <cuda.h>

#include "msz_device.cuh"

namespace msz {

__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double vmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ double vmin(double a, double b) { return fmin(a, b); }
// Three-input max / min (a single instruction for float32 on sm_100+; NaN
// operands are ignored like in the two-input form).
__device__ __forceinline__ float vmax3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float vmin3(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ double vmax3(double a, double b, double c) { return fmax(fmax(a, b), c); }
__device__ __forceinline__ double vmin3(double a, double b, double c) { return fmin(fmin(a, b), c); }

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
  static constexpr int NT = (ND == 3) ? 256 : 128;  // consumer threads
  static constexpr int NTP = NT + 32;               // + one producer warp (TMA path)
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
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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
  for (uint32_t i = 0; i < (1u << 24); ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// try_wait that may suspend the thread for up to ~1 us while the phase is
// incomplete (fewer polling instructions than a tight loop).
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(1000u)
      : "memory");
  return ok != 0;
}
// Bounded wait that also gives up as soon as *abort is set by another warp.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity, const int* abort) {
  for (uint32_t i = 0; i < (1u << 24); ++i) {
    if (mbar_try_wait_sleep(bar, parity)) return true;
    if ((i & 63u) == 63u && *(const volatile int*)abort) return false;
  }
  return false;
}
// Orders the tensor-map proxy after writes to the 128-byte map at `map` made
// by other means (host copies into device memory between launches): without
// it, a map rewritten at an address that an earlier launch used may be read
// from a stale descriptor cache.
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map))
               : "memory");
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

// Per-plane quantities of one thread's vertices (RPT rows): the centre value
// and the extrema of the two "L" corners (see the header comment).
template <class T, int RPT>
struct PlaneVals {
  T a0[RPT];                 // g at (x, y)
  T lurM[RPT], lurm[RPT];    // max / min of LUR
  T lllM[RPT], lllm[RPT];    // max / min of LLL
};

// Reads the thread's neighbourhood from a staged plane. 3D: rows y-1 .. y+RPT
// (stage rows RPT*w .. RPT*w+RPT+1) at columns x-1, x, x+1 for the RPT
// vertices of rows y = RPT*w .. RPT*w+RPT-1 (tile-local).
template <class T, int ND>
__device__ __forceinline__ PlaneVals<T, SweepGeom<T, ND>::RPT> plane_vals(const T* s, int tx, int w) {
  using SG = SweepGeom<T, ND>;
  PlaneVals<T, SG::RPT> P;
  const int c = tx + SG::PADX;
  if constexpr (ND == 3) {
    constexpr int R = SG::RPT;
    const T* r0 = s + (R * w) * SG::BX + c;  // row y-1
    T a[R + 2][3];
#pragma unroll
    for (int r = 0; r < R + 2; ++r) {
      a[r][0] = r0[r * SG::BX - 1];
      a[r][1] = r0[r * SG::BX];
      a[r][2] = r0[r * SG::BX + 1];
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {  // vertex row = r k+1
      P.a0[k] = a[k + 1][1];
      P.lurM[k] = vmax3(a[k + 1][2], a[k + 2][1], a[k + 2][2]);
      P.lurm[k] = vmin3(a[k + 1][2], a[k + 2][1], a[k + 2][2]);
      P.lllM[k] = vmax3(a[k + 1][0], a[k][0], a[k][1]);
      P.lllm[k] = vmin3(a[k + 1][0], a[k][0], a[k][1]);
    }
  } else {
    const T* m0 = s + c;
    P.a0[0] = m0[0];
    P.lurM[0] = P.lurm[0] = m0[1];
    P.lllM[0] = P.lllm[0] = m0[-1];
  }
  return P;
}

// Extremum flags of the thread's vertices of plane A (B next, C previous),
// packed two bits per vertex: bit 4k maximum, bit 4k+2 minimum... see
// kBitMax / kBitMin.
template <class T, int RPT>
__device__ __forceinline__ bool is_max_at(const PlaneVals<T, RPT>& C, const PlaneVals<T, RPT>& A,
                                          const PlaneVals<T, RPT>& B, int k) {
  const T maxU = vmax3(A.lurM[k], B.a0[k], B.lurM[k]);
  const T maxL = vmax3(A.lllM[k], C.a0[k], C.lllM[k]);
  const T g = A.a0[k];
  return !(maxU >= g) && !(maxL > g);
}
template <class T, int RPT>
__device__ __forceinline__ bool is_min_at(const PlaneVals<T, RPT>& C, const PlaneVals<T, RPT>& A,
                                          const PlaneVals<T, RPT>& B, int k) {
  const T minU = vmin3(A.lurm[k], B.a0[k], B.lurm[k]);
  const T minL = vmin3(A.lllm[k], C.a0[k], C.lllm[k]);
  const T g = A.a0[k];
  return !(minU < g) && !(minL <= g);
}

}  // namespace msz
