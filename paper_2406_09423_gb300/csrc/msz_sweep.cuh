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
// Data movement: a block owns an x-y tile (128 x 8 vertices of float32,
// 64 x 8 of float64; a warp per row, 16 bytes of a row per thread) and
// marches along z (3D; 128-vertex row segments along y in 2D). Each plane of the tile plus a one-vertex halo (widened in x
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

// Tile geometry. PADX keeps the TMA box start and width 16-byte aligned. In
// 3D a thread owns VX vertices consecutive in x (16 bytes of g: one vector
// load per staged row), a warp one row of a TX x TY tile; in 2D a thread owns
// one vertex and 128 threads cover 128 vertices of a row.
template <class T, int ND>
struct SweepGeom {
  static constexpr int PADX = 16 / (int)sizeof(T);
  static constexpr int VX = (ND == 3) ? 16 / (int)sizeof(T) : 1;  // vertices per thread
  static constexpr int TX = (ND == 3) ? 32 * VX : 128;
  static constexpr int TPR = TX / VX;  // threads per tile row
  static constexpr int TY = (ND == 3) ? 8 : 1;
  static constexpr int NT = TPR * TY;  // consumer threads (256 in 3D, 128 in 2D)
  static constexpr int NTP = NT + 32;  // + one producer warp (TMA path)
  static constexpr int BX = TX + 2 * PADX;
  static constexpr int BY = (ND == 3) ? TY + 2 : 1;
  static constexpr int STAGE_ELEMS = BX * BY;
  static constexpr int G_BYTES = ((STAGE_ELEMS * (int)sizeof(T) + 127) / 128) * 128;
  static constexpr int D_BYTES = ((TX * TY + 127) / 128) * 128;  // f's direction bytes of the tile plane
  static constexpr int STAGE_BYTES = G_BYTES + D_BYTES;
  static constexpr int STAGES = 4;
  static_assert(VX * (int)sizeof(T) == 16 || VX == 1, "one 16-byte row load per thread");
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

// The values a thread needs from one staged row: its VX vertices and one
// more on either side (columns c - 1 .. c + VX of the stage row r).
template <class T, int VX>
__device__ __forceinline__ void load_row(const T* row, T (&a)[VX + 2]) {
  if constexpr (VX == 1) {
    a[0] = row[-1];
    a[1] = row[0];
    a[2] = row[1];
  } else {
    static_assert(VX * sizeof(T) == 16, "16-byte row segment");
    const uint4 v = *reinterpret_cast<const uint4*>(row);  // 16-byte aligned: the stage column is
    const T* m = reinterpret_cast<const T*>(&v);             // PADX + VX * lane
    a[0] = row[-1];
#pragma unroll
    for (int k = 0; k < VX; ++k) a[k + 1] = m[k];
    a[VX + 1] = row[VX];
  }
}

// Per-plane quantities of a thread's VX vertices: the centre value and the
// max / min of the two "L" corners (see the header comment).
template <class T, int VX>
struct Partials {
  T a0[VX];
  T uM[VX], um[VX];  // LUR max / min
  T lM[VX], lm[VX];  // LLL max / min
};

// Partials of plane P from the stage: in 3D rows y-1, y, y+1 of the
// thread's row w (stage rows w .. w + 2) at its columns; in 2D the row.
template <class T, int ND>
__device__ __forceinline__ void plane_partials(const T* stage, int col, int w,
                                               Partials<T, SweepGeom<T, ND>::VX>& P) {
  using SG = SweepGeom<T, ND>;
  constexpr int VX = SG::VX;
  if constexpr (ND == 3) {
    T a[3][VX + 2];
#pragma unroll
    for (int r = 0; r < 3; ++r) load_row<T, VX>(stage + (w + r) * SG::BX + col, a[r]);
#pragma unroll
    for (int k = 0; k < VX; ++k) {  // vertex column k + 1 of row 1
      P.a0[k] = a[1][k + 1];
      P.uM[k] = vmax3(a[1][k + 2], a[2][k + 1], a[2][k + 2]);
      P.um[k] = vmin3(a[1][k + 2], a[2][k + 1], a[2][k + 2]);
      P.lM[k] = vmax3(a[1][k], a[0][k + 1], a[0][k]);
      P.lm[k] = vmin3(a[1][k], a[0][k + 1], a[0][k]);
    }
  } else {
    T a[3];
    load_row<T, 1>(stage + col, a);
    P.a0[0] = a[1];
    P.uM[0] = P.um[0] = a[2];
    P.lM[0] = P.lm[0] = a[0];
  }
}

}  // namespace msz
