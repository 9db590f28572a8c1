// Device-side building blocks of the MSz correction loop: grid geometry,
// the Freudenthal stencil, the error-bound arithmetic and per-vertex flags.
//
// Paper references (Li et al., MSz): Sec. 3 (PL field, critical points,
// integral lines, labels), Sec. 4.1 (false critical points, Eqs. 1-5),
// Sec. 4.2 (troublemaker, Eq. 6), Sec. 5 (parallel C-loop / R-loop).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "msz.h"

namespace msz {

constexpr int kThreads = 256;
constexpr uint32_t kFull = 0xffffffffu;
constexpr int kSelf = 15;

// Per-vertex flag byte.
enum : uint8_t {
  FL_DEC = 1,      // decreasing edit requested this round
  FL_FREEZE = 2,   // freeze requested this round
  FL_FROZEN = 4,   // reset to f by the termination guard; never edited again
  FL_EDITED = 8,   // edited at least once (candidate for the edit list)
};

// False critical point types, in sub-loop order (Sec. 4.1).
enum { FPMAX = 0, FPMIN = 1, FNMAX = 2, FNMIN = 3 };

// ---------------------------------------------------------------------------
// Stencil slots. Slot s < NPOS is the neighbour v + e_s, slot s >= NPOS is
// v - e_{s-NPOS}, slot 15 is v. 3D: e = (1,0,0) (0,1,0) (0,0,1) (1,1,0)
// (1,0,1) (0,1,1) (1,1,1); 2D: (1,0) (0,1) (1,1). Each e is stored as a
// 3-bit mask (x = bit 0, y = bit 1, z = bit 2), one nibble per slot.
// ---------------------------------------------------------------------------
template <int ND>
struct Slots {
  static constexpr int NPOS = (ND == 3) ? 7 : 3;
  static constexpr uint32_t MASKS = (ND == 3) ? 0x7653421u : 0x321u;
};

__host__ __device__ __forceinline__ int slot_mask(int nd, int b) {
  return (int)(((nd == 3 ? 0x7653421u : 0x321u) >> (4 * b)) & 7u);
}

// Linear offset of slot s (0 for the vertex itself).
__device__ __forceinline__ int slot_offset(int s, int nd, int nx, int nxny) {
  if (s == kSelf) return 0;
  const int npos = (nd == 3) ? 7 : 3;
  const bool neg = s >= npos;
  const int m = slot_mask(nd, neg ? s - npos : s);
  const int o = (m & 1) + ((m >> 1) & 1) * nx + ((m >> 2) & 1) * nxny;
  return neg ? -o : o;
}

// Division of 0 <= x < 2^31 by an invariant d >= 1 through one multiply-high
// (Granlund and Montgomery, "Division by invariant integers using
// multiplication", 1994): with s = ceil(log2 d) and
// m = floor(2^32 (2^s - d) / d) + 1, x / d = (mulhi(x, m) + x) >> s; the sum
// does not overflow since mulhi(x, m) <= x < 2^31.
struct FastDiv {
  uint32_t m, s;
};
inline FastDiv fast_div(uint32_t d) {
  FastDiv f{1u, 0u};
  while ((1ull << f.s) < d) ++f.s;
  f.m = (uint32_t)((((1ull << 32) * ((1ull << f.s) - d)) / d) + 1);
  return f;
}
__device__ __forceinline__ uint32_t fdiv(uint32_t x, FastDiv f) { return (__umulhi(x, f.m) + x) >> f.s; }

struct Geom {
  int nx, ny, nz, nxny, n, nd;
  FastDiv dx, dy;  // division by nx and by ny
};

__device__ __forceinline__ void coords(const Geom& G, int v, int& x, int& y, int& z) {
  const int t = (int)fdiv((uint32_t)v, G.dx);
  x = v - t * G.nx;
  z = (int)fdiv((uint32_t)t, G.dy);
  y = t - z * G.ny;
}

// ---------------------------------------------------------------------------
// IEEE round-to-nearest arithmetic without contraction (the build also
// passes -fmad=false). Each call is exactly one rounded operation.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }

__device__ __forceinline__ bool finite(float a) { return isfinite(a); }
__device__ __forceinline__ bool finite(double a) { return isfinite(a); }

// Next representable value towards +inf / -inf for finite a (bit stepping).
__device__ __forceinline__ float next_up(float a) {
  if (a == 0.0f) return __int_as_float(1);
  const int b = __float_as_int(a);
  return __int_as_float(a > 0.0f ? b + 1 : b - 1);
}
__device__ __forceinline__ double next_up(double a) {
  if (a == 0.0) return __longlong_as_double(1ll);
  const long long b = __double_as_longlong(a);
  return __longlong_as_double(a > 0.0 ? b + 1 : b - 1);
}
__device__ __forceinline__ float next_down(float a) { return -next_up(-a); }
__device__ __forceinline__ double next_down(double a) { return -next_up(-a); }

// Exact error of s = RN(a + b) (TwoSum): a + b == s + err.
template <class T>
__device__ __forceinline__ T two_sum_err(T a, T b, T s) {
  const T bp = rn_sub(s, a);
  const T ap = rn_sub(s, bp);
  return rn_add(rn_sub(a, ap), rn_sub(b, bp));
}

// Smallest representable value >= f - xi (the lower bound of Eq. 1).
template <class T>
__device__ __forceinline__ T lower_bound_of(T f, T xi) {
  T s = rn_sub(f, xi);
  if (!finite(s)) return s;
  if (two_sum_err(f, -xi, s) > T(0)) s = next_up(s);
  return s;
}

// Largest representable value <= f + xi (upper end of the bound).
template <class T>
__device__ __forceinline__ T upper_bound_of(T f, T xi) {
  T s = rn_add(f, xi);
  if (!finite(s)) return s;
  if (two_sum_err(f, xi, s) < T(0)) s = next_down(s);
  return s;
}

// One decreasing edit (Eqs. 2-6): g <- (g + f - xi)/2 with f - xi read as
// lb, as RN(RN(g/2) + RN(lb/2)); a step that rounds back to g snaps to lb.
template <class T>
__device__ __forceinline__ T decrease(T g, T lb) {
  T m = rn_add(rn_mul(T(0.5), g), rn_mul(T(0.5), lb));
  if (!(m < g) || m < lb) m = lb;
  return m;
}

// ---------------------------------------------------------------------------
// Steepest ascending / descending neighbour of vertex v (Sec. 3 "Integral
// lines", Sec. 5.1 "Updating directions"): the greatest / least vertex of the
// closed 1-ring under (value, index) order. Returns up | dn << 4.
// ---------------------------------------------------------------------------
template <class T, int ND>
__device__ __forceinline__ uint8_t direction_of(const T* __restrict__ g, const Geom& G, int v, int x,
                                                int y, int z) {
  constexpr int NPOS = Slots<ND>::NPOS;
  const T gv = g[v];
  T hv = gv, lv = gv;
  int hi = v, lo = v, hs = kSelf, ls = kSelf;
  // interior vertices (all neighbours in the grid) skip the bounds tests
  const bool interior = x > 0 && x < G.nx - 1 && y > 0 && y < G.ny - 1 && (ND == 2 || (z > 0 && z < G.nz - 1));
  if (interior) {
    T gu[2 * NPOS];
#pragma unroll
    for (int s = 0; s < 2 * NPOS; ++s) {
      const int sg = (s < NPOS) ? 1 : -1;
      const int m = (int)((Slots<ND>::MASKS >> (4 * (s < NPOS ? s : s - NPOS))) & 7u);
      gu[s] = g[v + sg * ((m & 1) + ((m >> 1) & 1) * G.nx + ((m >> 2) & 1) * G.nxny)];
    }
#pragma unroll
    for (int s = 0; s < 2 * NPOS; ++s) {
      const int sg = (s < NPOS) ? 1 : -1;
      const int m = (int)((Slots<ND>::MASKS >> (4 * (s < NPOS ? s : s - NPOS))) & 7u);
      const int u = v + sg * ((m & 1) + ((m >> 1) & 1) * G.nx + ((m >> 2) & 1) * G.nxny);
      if (gu[s] > hv || (gu[s] == hv && u > hi)) { hv = gu[s]; hi = u; hs = s; }
      if (gu[s] < lv || (gu[s] == lv && u < lo)) { lv = gu[s]; lo = u; ls = s; }
    }
    return (uint8_t)(hs | (ls << 4));
  }
#pragma unroll
  for (int s = 0; s < 2 * NPOS; ++s) {
    const int sg = (s < NPOS) ? 1 : -1;
    const int m = (int)((Slots<ND>::MASKS >> (4 * (s < NPOS ? s : s - NPOS))) & 7u);
    const int dx = sg * (m & 1), dy = sg * ((m >> 1) & 1), dz = sg * ((m >> 2) & 1);
    const int X = x + dx, Y = y + dy, Z = z + dz;
    bool in = X >= 0 && X < G.nx && Y >= 0 && Y < G.ny;
    if (ND == 3) in = in && Z >= 0 && Z < G.nz;
    if (in) {
      const int u = v + dx + dy * G.nx + dz * G.nxny;
      const T gu = g[u];
      if (gu > hv || (gu == hv && u > hi)) { hv = gu; hi = u; hs = s; }
      if (gu < lv || (gu == lv && u < lo)) { lv = gu; lo = u; ls = s; }
    }
  }
  return (uint8_t)(hs | (ls << 4));
}

// False critical point bits from the direction bytes of g and f
// (Definitions 1-3 as set differences of extremum sets).
__device__ __forceinline__ unsigned case_bits(uint8_t dg, uint8_t df) {
  const bool gmax = (dg & 15) == kSelf, gmin = (dg >> 4) == kSelf;
  const bool fmax = (df & 15) == kSelf, fmin = (df >> 4) == kSelf;
  return (unsigned)(gmax && !fmax) | (unsigned)(gmin && !fmin) << 1 |
         (unsigned)(fmax && !gmax) << 2 | (unsigned)(fmin && !gmin) << 3;
}

}  // namespace msz
