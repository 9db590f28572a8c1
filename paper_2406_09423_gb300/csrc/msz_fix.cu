// MSz correction loop on one GPU: plan, device-resident state machine and
// the C-ABI entry points declared in include/msz.h.
//
// The loop (Sec. 4 of the paper; control flow of Fig. 3) runs as a fixed
// sequence of kernels per "step":
//   sweep      - directions of g + false critical point detection (Sec. 5.1)
//   mark_c     - C-loop edit requests of the current type (Eqs. 2-5)
//   label_init - pointer initialisation for the labels (Sec. 5.2)
//   jump x J   - pointer jumping rounds
//   rcheck     - label mismatches + troublemaker requests (Sec. 4.2, Eq. 6)
//   apply      - applies the round's requests (iteration-synchronous)
// Every kernel reads the per-field state word and returns at once when it
// has nothing to do; the last block of a kernel advances the state machine.
// The host launches steps in growing chunks and reads one word per chunk, so
// it never synchronises per iteration.
//
// Edit requests of a round are flags (idempotent atomicOr) collected before
// any value changes, so the result does not depend on thread order (the
// deterministic mode of Sec. 5.1); a freeze overrides a decrease.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "msz.h"
#include "msz_device.cuh"
#include "msz_sweep.cuh"

namespace msz {

enum : uint32_t { PH_INIT = 0, PH_FLABELS = 1, PH_C = 2, PH_R = 3, PH_DONE = 4, PH_ERR = 5 };
enum : uint32_t { ACT_NONE = 0, ACT_MARK_C = 1, ACT_LABELS = 2, ACT_APPLY_R = 3 };
enum : uint32_t { L_INIT = 0, L_JUMP = 1, L_DONE = 2 };
enum : uint32_t { E_NONFINITE = 1, E_ARG = 2, E_BOUND = 4, E_TIMEOUT = 8 };

struct DevState {
  uint32_t phase, action, T, lstate, ljob, blocks_done, err_bits;
  int32_t status;
  uint32_t counts[4];
  uint32_t ncase, ntouch;
  uint32_t acc_changed;
  uint32_t acc_ap[2];  // apply: decreases, freezes
  uint32_t acc_r[4];   // rcheck: wrong max, wrong min, asc troublemakers, desc troublemakers
  uint32_t jump_rounds, pad0;
  uint64_t rounds, max_rounds, n_edits;
  uint64_t ticks;      // advanced by every state transition (stall detection)
  msz_counts cnt;
};

template <class T>
struct Field {
  const T* f;
  const T* fhat;
  T* g;
  uint8_t* fdir;
  uint8_t* gdir;
  uint8_t* flags;
  uint32_t* fbits;  // packed extremum bits of f: [0, nw) maxima, [nw, 2nw) minima
  int nwords;
  int32_t* Mf;
  int32_t* mf;
  int32_t* Pup;
  int32_t* Pdn;
  uint32_t* cases;
  uint32_t* touched;
  uint32_t* tile_cnt;
  uint32_t* edit_idx;
  T* edit_val;
  DevState* st;
  T xi;
  Geom G;
};

// ---------------------------------------------------------------------------
// Last-block detection (threadfence reduction): returns true in the block
// that finishes last; all other blocks' global writes are visible to it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool last_block(DevState* st) {
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t t = atomicAdd(&st->blocks_done, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last;
}

__device__ __forceinline__ uint32_t vload(const uint32_t* p) { return *(volatile const uint32_t*)p; }

template <int NW>
__device__ __forceinline__ void block_add(uint32_t (&v)[NW], uint32_t* dst) {
  __shared__ uint32_t s[NW];
  if (threadIdx.x < NW) s[threadIdx.x] = 0;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NW; ++k) {
    uint32_t x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(&s[k], x);
  }
  __syncthreads();
  if (threadIdx.x < NW && s[threadIdx.x]) atomicAdd(&dst[threadIdx.x], s[threadIdx.x]);
}

// ---------------------------------------------------------------------------
// Edit requests
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void mark(const Field<T>& F, int u, uint8_t bit) {
  uint32_t* w = reinterpret_cast<uint32_t*>(F.flags) + (u >> 2);
  const int sh = (u & 3) * 8;
  const uint32_t old = atomicOr(w, (uint32_t)bit << sh);
  if (((old >> sh) & (FL_DEC | FL_FREEZE)) == 0) {
    const uint32_t k = atomicAdd(&F.st->ntouch, 1u);
    F.touched[k] = (uint32_t)u;
  }
}

// A false case anchored at a asks for a decreasing edit of t. If t is frozen
// or already at its lower bound, the non-frozen part of a's closed 1-ring is
// frozen instead (termination guard; the paper argues convergence in the
// reals, Sec. 4.3).
template <class T, int ND>
__device__ void request(const Field<T>& F, int a, int t) {
  const uint8_t ft = F.flags[t];
  if (!(ft & FL_FROZEN) && F.g[t] > lower_bound_of(F.f[t], F.xi)) {
    mark(F, t, FL_DEC);
    return;
  }
  int x, y, z;
  coords(F.G, a, x, y, z);
  if (!(F.flags[a] & FL_FROZEN)) mark(F, a, FL_FREEZE);
  constexpr int NPOS = Slots<ND>::NPOS;
#pragma unroll
  for (int s = 0; s < 2 * NPOS; ++s) {
    const int sg = (s < NPOS) ? 1 : -1;
    const int m = (int)((Slots<ND>::MASKS >> (4 * (s < NPOS ? s : s - NPOS))) & 7u);
    const int dx = sg * (m & 1), dy = sg * ((m >> 1) & 1), dz = sg * ((m >> 2) & 1);
    const int X = x + dx, Y = y + dy, Z = z + dz;
    bool in = X >= 0 && X < F.G.nx && Y >= 0 && Y < F.G.ny;
    if (ND == 3) in = in && Z >= 0 && Z < F.G.nz;
    if (in) {
      const int u = a + dx + dy * F.G.nx + dz * F.G.nxny;
      if (!(F.flags[u] & FL_FROZEN)) mark(F, u, FL_FREEZE);
    }
  }
}

// ---------------------------------------------------------------------------
// Init: validate inputs (Sec. 3 constraint), g = fhat, directions of f,
// clear flags. Last block: error status or start the labels of f.
// ---------------------------------------------------------------------------
template <class T, int ND>
__global__ void __launch_bounds__(kThreads) k_init(Field<T> F) {
  DevState* st = F.st;
  if (st->phase != PH_INIT) return;
  uint32_t err = 0;
  const int n = F.G.n;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
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
  }
  if (err) atomicOr(&st->err_bits, err);
  if (last_block(st) && threadIdx.x == 0) {
    const uint32_t e = vload(&st->err_bits);
    if (e) {
      st->phase = PH_ERR;
      st->status = (e & E_NONFINITE) ? MSZ_ERR_NONFINITE : (e & E_ARG) ? MSZ_ERR_ARG : MSZ_ERR_BOUND;
    } else {
      st->phase = PH_FLABELS;
      st->action = ACT_LABELS;
      st->lstate = L_INIT;
      st->ljob = 0;
    }
    st->ticks++;
    st->blocks_done = 0;
  }
}

// C-loop control after a sweep (runs in the last block): picks the next
// sub-loop with cases, ends a pass after FNmin, or hands over to the R-loop
// when a whole pass finds no false critical point.
__device__ void ctrl_after_sweep(DevState* st) {
  uint32_t c[4];
  for (int t = 0; t < 4; ++t) c[t] = vload(&st->counts[t]);
  if (vload(&st->err_bits) & E_TIMEOUT) {
    st->phase = PH_ERR;
    st->status = MSZ_ERR_TIMEOUT;
    return;
  }
  st->cnt.sweeps++;
  uint32_t T_ = st->T;
  for (;;) {
    if (c[T_]) { st->action = ACT_MARK_C; break; }
    if (T_ < 3) { ++T_; continue; }
    st->cnt.c_passes++;
    if ((c[0] | c[1] | c[2] | c[3]) == 0) {
      st->phase = PH_R;
      st->action = ACT_LABELS;
      st->lstate = L_INIT;
      st->ljob = 1;
      break;
    }
    T_ = 0;
  }
  st->T = T_;
  st->ticks++;
}

// ---------------------------------------------------------------------------
// C-loop sweep (see msz_sweep.cuh): extremum bits of g per vertex, false
// critical points of every type counted with warp ballots and appended to
// the case list. A block marches over planes of its tiles; with kTMA the
// planes stream through a ring of TMA stages, otherwise through one stage
// filled by plain loads.
// ---------------------------------------------------------------------------
// Cursor over the (tile, plane) sequence of one block: tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...; planes 0 .. chunk+1 of each. Divisions only
// happen when a new tile starts.
struct PlaneCursor {
  int tile, p, x0, y0, c0;
  __device__ __forceinline__ void origin(const SweepTiling& TL, int tx_, int ty_) {
    const int bx = tile % TL.tiles_x;
    const int r = tile / TL.tiles_x;
    x0 = bx * tx_;
    y0 = (r % TL.tiles_y) * ty_;
    c0 = (r / TL.tiles_y) * TL.chunk;
  }
  __device__ __forceinline__ void start(const SweepTiling& TL, int tx_, int ty_) {
    tile = (int)blockIdx.x;
    p = 0;
    origin(TL, tx_, ty_);
  }
  __device__ __forceinline__ void next(const SweepTiling& TL, int tx_, int ty_) {
    if (++p == TL.chunk + 2) {
      p = 0;
      tile += (int)gridDim.x;
      origin(TL, tx_, ty_);
    }
  }
};

template <class T, int ND, bool kTMA>
__global__ void __launch_bounds__(kTMA ? SweepGeom<T, ND>::NTP : SweepGeom<T, ND>::NT)
    k_csweep(Field<T> F, const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap dmap,
             SweepTiling TL) {
  using SG = SweepGeom<T, ND>;
  constexpr int RPT = SG::RPT;
  constexpr int NCW = SG::NT / 32;  // consumer warps
  using PV = PlaneVals<T, RPT>;
  static_assert((SG::STAGES & (SG::STAGES - 1)) == 0, "power-of-two stages");
  DevState* st = F.st;
  if (st->phase != PH_C) return;
  __shared__ alignas(128) unsigned char smem[(kTMA ? SG::STAGES : 1) * SG::STAGE_BYTES];
  __shared__ alignas(8) uint64_t full[SG::STAGES];
  __shared__ alignas(8) uint64_t empty[SG::STAGES];
  __shared__ int s_abort;
  const int tid = threadIdx.x;
  const bool producer = kTMA && tid >= SG::NT;
  const int tx = tid % SG::TX, w = (tid / SG::TX) % (SG::NT / SG::TX);  // 3D: consumer warp w owns rows 2w, 2w+1
  const int lane = tid & 31;
  const int ppt = TL.chunk + 2;  // planes per tile, a multiple of 3
  const int my_tiles =
      (blockIdx.x < (unsigned)TL.ntiles) ? (TL.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int total = my_tiles * ppt;
  const Geom G = F.G;
  constexpr int SM1 = SG::STAGES - 1;
  uint32_t cnt[4] = {0, 0, 0, 0};

  if (kTMA) {
    if (tid == 0) {
      for (int s = 0; s < SG::STAGES; ++s) {
        mbar_init(&full[s], 1);
        mbar_init(&empty[s], NCW);
      }
      s_abort = 0;
      mbar_fence_init();
    }
    __syncthreads();
  }

  if (producer) {
    // Producer warp (lane 0): streams planes into the stage ring. Before it
    // refills a stage it waits until every consumer warp has released it.
    if (lane == 0) {
      PlaneCursor pc{};
      pc.start(TL, SG::TX, SG::TY);
      int issued = 0;
      for (int q = 0; q < total; ++q) {
        const int s = q & SM1;
        if (q >= SG::STAGES) {
          if (!mbar_wait_or_abort(&empty[s], (uint32_t)(((q - SG::STAGES) / SG::STAGES) & 1), &s_abort)) {
            atomicExch(&s_abort, 1);
            break;
          }
        }
        const int pcoord = pc.c0 - 1 + pc.p;
        unsigned char* sp = smem + s * SG::STAGE_BYTES;
        mbar_expect_tx(&full[s], (uint32_t)(SG::STAGE_ELEMS * sizeof(T) + SG::TX * SG::TY));
        if (ND == 3) {
          tma_load_3d(sp, &tmap, &full[s], pc.x0 - SG::PADX, pc.y0 - 1, pcoord);
          tma_load_3d(sp + SG::G_BYTES, &dmap, &full[s], pc.x0, pc.y0, pcoord);
        } else {
          tma_load_2d(sp, &tmap, &full[s], pc.x0 - SG::PADX, pcoord);
          tma_load_2d(sp + SG::G_BYTES, &dmap, &full[s], pc.x0, pcoord);
        }
        pc.next(TL, SG::TX, SG::TY);
        issued = q + 1;
      }
      if (*(volatile int*)&s_abort) {
        // wait (bounded) for the loads still in flight before leaving
        const int first = (issued > SG::STAGES) ? issued - SG::STAGES : 0;
        for (int q = first; q < issued; ++q) mbar_wait(&full[q & SM1], (uint32_t)((q / SG::STAGES) & 1));
        atomicOr(&st->err_bits, E_TIMEOUT);
      }
    }
  } else {
    PlaneCursor cur;
    cur.start(TL, SG::TX, SG::TY);
    // vertices of this thread inside the grid in x and y (bits 8k, 8k+4)
    auto xy_mask = [&]() -> uint32_t {
      uint32_t m = 0;
      const int x = cur.x0 + tx;
#pragma unroll
      for (int k = 0; k < RPT; ++k) {
        const int y = (ND == 3) ? cur.y0 + RPT * w + k : 0;
        if (x < G.nx && y < G.ny) m |= 0x11u << (8 * k);
      }
      return m;
    };
    uint32_t vmask = xy_mask();
    // One plane: stage it, derive its quantities into dst (role B), then
    // classify the vertices of plane A using C (previous) and dst (next).
    auto step = [&](int q, PV& dst, uint16_t& fd_dst, const PV& Cv, const PV& Av, uint16_t fdA) -> bool {
      const int p = cur.p;
      const int pcoord = cur.c0 - 1 + p;  // plane coordinate (z in 3D, y in 2D)
      unsigned char* sp = smem + (kTMA ? (q & SM1) * SG::STAGE_BYTES : 0);
      const T* stage = reinterpret_cast<const T*>(sp);
      if (kTMA) {
        const bool got = mbar_wait_or_abort(&full[q & SM1], (uint32_t)((q / SG::STAGES) & 1), &s_abort);
        if (!__all_sync(kFull, got)) {
          if (lane == 0) atomicExch(&s_abort, 1);
          return false;
        }
        dst = plane_vals<T, ND>(stage, tx, w);
        if (ND == 3) fd_dst = (uint16_t)(sp[SG::G_BYTES + (2 * w) * SG::TX + tx] |
                                         (sp[SG::G_BYTES + (2 * w + 1) * SG::TX + tx] << 8));
        else fd_dst = sp[SG::G_BYTES + tx];
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[q & SM1]);
      } else {
        __syncthreads();
        T* wst = reinterpret_cast<T*>(sp);
        for (int i = tid; i < SG::STAGE_ELEMS; i += SG::NT) {
          const int col = i % SG::BX, row = i / SG::BX;
          const int gx = cur.x0 - SG::PADX + col;
          const int gy = (ND == 3) ? cur.y0 - 1 + row : pcoord;
          const int gz = (ND == 3) ? pcoord : 0;
          const bool in = gx >= 0 && gx < G.nx && gy >= 0 && gy < G.ny && gz >= 0 && gz < G.nz;
          wst[i] = in ? F.g[gx + G.nx * (gy + G.ny * gz)] : qnan<T>();
        }
        __syncthreads();
        dst = plane_vals<T, ND>(stage, tx, w);
        uint16_t fd = 0;
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
          const int vx = cur.x0 + tx, vy = (ND == 3) ? cur.y0 + RPT * w + k : pcoord, vz = (ND == 3) ? pcoord : 0;
          if (vx < G.nx && vy >= 0 && vy < G.ny && vz >= 0 && vz < G.nz)
            fd |= (uint16_t)(F.fdir[vx + G.nx * (vy + G.ny * vz)] << (8 * k));
        }
        fd_dst = fd;
      }
      if (p >= 2) {
        // g's extremum flags and f's, both packed at bits 8k (max) and 8k+4
        // (min) for vertex k; a vertex is a case when they differ.
        uint32_t gb = 0;
#pragma unroll
        for (int k = 0; k < RPT; ++k)
          gb |= ((uint32_t)is_max_at<T, RPT>(Cv, Av, dst, k) << (8 * k)) |
                ((uint32_t)is_min_at<T, RPT>(Cv, Av, dst, k) << (8 * k + 4));
        const uint32_t fa = fdA;
        const uint32_t fb = fa & (fa >> 1) & (fa >> 2) & (fa >> 3) & 0x1111u;  // nibble == 15
        uint32_t diff = (gb ^ fb) & vmask;
        if (!(p - 2 < TL.chunk && pcoord - 1 < ((ND == 3) ? G.nz : G.ny))) diff = 0;
        if (__any_sync(kFull, diff != 0)) {
          const int x = cur.x0 + tx;
          const int z = (ND == 3) ? pcoord - 1 : 0;
#pragma unroll
          for (int k = 0; k < RPT; ++k) {
            const int y = (ND == 3) ? cur.y0 + RPT * w + k : pcoord - 1;
            const uint32_t gk = gb >> (8 * k), fk = fb >> (8 * k), dk = diff >> (8 * k);
            unsigned bits = 0;
            if (dk & 0x11u) {
              const unsigned gmx = gk & 1u, gmn = (gk >> 4) & 1u, fmx = fk & 1u, fmn = (fk >> 4) & 1u;
              bits = (gmx & ~fmx) | ((gmn & ~fmn) << 1) | ((fmx & ~gmx) << 2) | ((fmn & ~gmn) << 3);
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const uint32_t b = __ballot_sync(kFull, (bits >> t) & 1u);
              if (lane == 0) cnt[t] += __popc(b);
            }
            const uint32_t mask = __ballot_sync(kFull, bits != 0);
            if (mask) {
              const int leader = __ffs(mask) - 1;
              uint32_t b0 = 0;
              if (lane == leader) b0 = atomicAdd(&st->ncase, (uint32_t)__popc(mask));
              b0 = __shfl_sync(kFull, b0, leader);
              if (bits) F.cases[b0 + __popc(mask & ((1u << lane) - 1u))] = (uint32_t)(x + G.nx * (y + G.ny * z));
            }
          }
        }
      }
      const int tile_before = cur.tile;
      cur.next(TL, SG::TX, SG::TY);
      if (cur.tile != tile_before) vmask = xy_mask();
      return true;
    };

    PV P0{}, P1{}, P2{};
    uint16_t f0 = 0, f1 = 0, f2 = 0;
    for (int q = 0; q < total; q += 3) {  // planes rotate through P0, P1, P2
      if (!step(q, P0, f0, P1, P2, f2)) break;
      if (!step(q + 1, P1, f1, P2, P0, f0)) break;
      if (!step(q + 2, P2, f2, P0, P1, f1)) break;
    }
  }
  block_add<4>(cnt, st->counts);
  if (last_block(st) && threadIdx.x == 0) {
    ctrl_after_sweep(st);
    st->blocks_done = 0;
  }
}

// C-loop requests for the current type (Eqs. 2-5): FPmax and FNmin edit the
// false vertex itself; FPmin and FNmax edit its neighbour that is maximal in
// g, which is its steepest ascent since it is not a maximum of g's ring.
template <class T, int ND>
__global__ void __launch_bounds__(kThreads) k_mark_c(Field<T> F) {
  DevState* st = F.st;
  if (st->action != ACT_MARK_C) return;
  const uint32_t type = st->T, nc = st->ncase;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    const int v = (int)F.cases[i];
    int x, y, z;
    coords(F.G, v, x, y, z);
    const uint8_t d = direction_of<T, ND>(F.g, F.G, v, x, y, z);
    if (!((case_bits(d, F.fdir[v]) >> type) & 1u)) continue;
    const int t = (type == FPMAX || type == FNMIN) ? v : v + slot_offset(d & 15, ND, F.G.nx, F.G.nxny);
    request<T, ND>(F, v, t);
  }
}

// ---------------------------------------------------------------------------
// Labels, first level (Sec. 5.2 path compression, Maack et al.): a block
// loads a tile of the field plus a one-vertex halo into shared memory,
// computes every tile vertex's steepest ascending / descending neighbour
// (candidates in ascending index order, so ties go to the larger index for
// the maximum and the smaller one for the minimum; NaN halo cells never
// win), and follows the pointers inside the tile by pointer doubling in
// shared memory. Each vertex leaves with a pointer to the first vertex
// outside the tile on its integral line, or to the extremum it reaches
// inside the tile. Global jumping then only crosses tiles.
// Job 0: f, writing fdir and (Mf, mf). Job 1: g, writing gdir and (Pup, Pdn).
// ---------------------------------------------------------------------------
template <int ND>
struct LabelGeom {
  static constexpr int TX = (ND == 3) ? 32 : 64;
  static constexpr int TY = (ND == 3) ? 8 : 32;
  static constexpr int TZ = (ND == 3) ? 8 : 1;
  static constexpr int TV = TX * TY * TZ;  // 2048 vertices
  static constexpr int SX = TX + 2, SY = TY + 2, SZ = (ND == 3) ? TZ + 2 : 1;
  static constexpr int HALO = SX * SY * SZ;  // < 65536: pointers fit in 16 bits
  static constexpr int PER_THREAD = TV / kThreads;
  static constexpr int ROWS = SY * SZ;
};

template <class T, int ND>
__global__ void __launch_bounds__(kThreads) k_label_tile(Field<T> F) {
  using LG = LabelGeom<ND>;
  DevState* st = F.st;
  if (st->action != ACT_LABELS || st->lstate != L_INIT) return;
  extern __shared__ __align__(16) unsigned char lsm[];
  T* val = reinterpret_cast<T*>(lsm);
  // Pointers live in halo coordinates: a halo cell or an extremum points to
  // itself (terminal); an interior cell points to its steepest neighbour.
  uint16_t* Pu = reinterpret_cast<uint16_t*>(lsm + ((LG::HALO * sizeof(T) + 15) / 16) * 16);
  uint16_t* Pd = Pu + ((LG::HALO + 7) / 8) * 8;
  const bool job = st->ljob != 0;
  const T* src = job ? F.g : F.f;
  uint8_t* dir = job ? F.gdir : F.fdir;
  int32_t* A = job ? F.Pup : F.Mf;
  int32_t* B = job ? F.Pdn : F.mf;
  const Geom G = F.G;
  const int tiles_x = (G.nx + LG::TX - 1) / LG::TX;
  const int tiles_y = (G.ny + LG::TY - 1) / LG::TY;
  const int tiles_z = (G.nz + LG::TZ - 1) / LG::TZ;
  const int ntiles = tiles_x * tiles_y * tiles_z;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // halo-space offset of every stencil slot (slots 0..13, 15 = self)
  constexpr int HS = LG::SX, HSS = LG::SX * LG::SY;
  constexpr int NC = (ND == 3) ? 15 : 7;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int x0 = (tile % tiles_x) * LG::TX;
    const int y0 = ((tile / tiles_x) % tiles_y) * LG::TY;
    const int z0 = (tile / (tiles_x * tiles_y)) * LG::TZ;
    __syncthreads();
    // halo load, one row (fixed hy, hz) per warp iteration; NaN outside the grid
    for (int row = warp; row < LG::ROWS; row += kThreads / 32) {
      const int hy = row % LG::SY, hz = row / LG::SY;
      const int gy = y0 - 1 + hy, gz = (ND == 3) ? z0 - 1 + hz : 0;
      const bool rin = gy >= 0 && gy < G.ny && gz >= 0 && gz < G.nz;
      const T* srow = src + (size_t)G.nx * ((size_t)gy + (size_t)G.ny * gz);
      for (int hx = lane; hx < LG::SX; hx += 32) {
        const int gx = x0 - 1 + hx;
        const int h = hx + HS * row;
        val[h] = (rin && gx >= 0 && gx < G.nx) ? srow[gx] : qnan<T>();
        Pu[h] = (uint16_t)h;
        Pd[h] = (uint16_t)h;
      }
    }
    __syncthreads();
    uint8_t dbyte[LG::PER_THREAD];
#pragma unroll
    for (int k = 0; k < LG::PER_THREAD; ++k) {
      const int i = threadIdx.x + k * kThreads;
      const int lx = i % LG::TX, ly = (i / LG::TX) % LG::TY, lz = i / (LG::TX * LG::TY);
      const int c = (lx + 1) + HS * (ly + 1) + ((ND == 3) ? HSS * (lz + 1) : 0);
      // candidates in ascending linear index = ascending (dz, dy, dx); ties go
      // to the larger index for the maximum and to the smaller for the minimum
      T hv = -INFINITY, lv = INFINITY;
      int hs = kSelf, ls = kSelf, ho = 0, lo = 0;
#pragma unroll
      for (int j = 0; j < NC; ++j) {
        int o, slot;
        if (ND == 3) {
          constexpr int tab[15][2] = {{-1 - HS - HSS, 13}, {-HS - HSS, 12}, {-1 - HSS, 11}, {-HSS, 9},
                                      {-1 - HS, 10},       {-HS, 8},        {-1, 7},        {0, kSelf},
                                      {1, 0},              {HS, 1},         {1 + HS, 3},    {HSS, 2},
                                      {1 + HSS, 4},        {HS + HSS, 5},   {1 + HS + HSS, 6}};
          o = tab[j][0]; slot = tab[j][1];
        } else {
          constexpr int tab[7][2] = {{-1 - HS, 5}, {-HS, 4}, {-1, 3}, {0, kSelf}, {1, 0}, {HS, 1}, {1 + HS, 2}};
          o = tab[j][0]; slot = tab[j][1];
        }
        const T u = val[c + o];
        if (u >= hv) { hv = u; hs = slot; ho = o; }
        if (u < lv) { lv = u; ls = slot; lo = o; }
      }
      dbyte[k] = (uint8_t)(hs | (ls << 4));
      // cells outside the grid are NaN: they keep self pointers and are never
      // chosen by a valid cell
      if (val[c] == val[c]) {
        Pu[c] = (uint16_t)(c + ho);
        Pd[c] = (uint16_t)(c + lo);
      }
    }
    __syncthreads();
    // pointer doubling inside the tile: P[c] <- P[P[c]] until all are terminal
    for (int round = 0; round < 2 * LG::TV; ++round) {
      int changed = 0;
#pragma unroll
      for (int k = 0; k < LG::PER_THREAD; ++k) {
        const int i = threadIdx.x + k * kThreads;
        const int lx = i % LG::TX, ly = (i / LG::TX) % LG::TY, lz = i / (LG::TX * LG::TY);
        const int c = (lx + 1) + HS * (ly + 1) + ((ND == 3) ? HSS * (lz + 1) : 0);
        const int a = Pu[c], a2 = Pu[a];
        if (a2 != a) { Pu[c] = (uint16_t)a2; changed = 1; }
        const int b = Pd[c], b2 = Pd[b];
        if (b2 != b) { Pd[c] = (uint16_t)b2; changed = 1; }
      }
      if (!__syncthreads_or(changed)) break;
    }
#pragma unroll
    for (int k = 0; k < LG::PER_THREAD; ++k) {
      const int i = threadIdx.x + k * kThreads;
      const int lx = i % LG::TX, ly = (i / LG::TX) % LG::TY, lz = i / (LG::TX * LG::TY);
      const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
      if (x < G.nx && y < G.ny && z < G.nz) {
        const int v = x + G.nx * (y + G.ny * z);
        const int c = (lx + 1) + HS * (ly + 1) + ((ND == 3) ? HSS * (lz + 1) : 0);
        // terminal halo cell -> global index (same offset from v as from c)
        auto global_of = [&](int h) -> int {
          const int hx = h % LG::SX, hy = (h / LG::SX) % LG::SY, hz = h / HSS;
          return (x0 - 1 + hx) + G.nx * ((y0 - 1 + hy) + G.ny * ((ND == 3) ? (z0 - 1 + hz) : 0));
        };
        dir[v] = dbyte[k];
        A[v] = global_of(Pu[c]);
        B[v] = global_of(Pd[c]);
      }
    }
  }
  if (last_block(st) && threadIdx.x == 0) {
    st->lstate = L_JUMP;
    st->jump_rounds = 0;
    st->ticks++;
    st->blocks_done = 0;
  }
}

// One pointer-jumping round, in place: P[v] <- P[P[v]]. A round that changes
// nothing means every pointer is a root.
template <class T>
__global__ void __launch_bounds__(kThreads) k_jump(Field<T> F) {
  DevState* st = F.st;
  if (st->action != ACT_LABELS || st->lstate != L_JUMP) return;
  const bool job = st->ljob != 0;
  int32_t* A = job ? F.Pup : F.Mf;
  int32_t* B = job ? F.Pdn : F.mf;
  const int n = F.G.n;
  uint32_t changed[1] = {0};
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int p = A[v], q = A[p];
    if (q != p) { A[v] = q; ++changed[0]; }
    const int r = B[v], s = B[r];
    if (s != r) { B[v] = s; ++changed[0]; }
  }
  block_add<1>(changed, &st->acc_changed);
  if (last_block(st) && threadIdx.x == 0) {
    const uint32_t c = vload(&st->acc_changed);
    st->acc_changed = 0;
    st->jump_rounds++;
    st->ticks++;
    if (c == 0) {
      if (st->ljob == 0) {
        st->phase = PH_C;
        st->action = ACT_NONE;
        st->T = 0;
      } else {
        st->lstate = L_DONE;
      }
    } else if (st->jump_rounds > 64) {
      st->phase = PH_ERR;
      st->status = MSZ_ERR_TIMEOUT;
    }
    st->blocks_done = 0;
  }
}

// R-loop check (Sec. 4.2): count wrong labels; a wrongly labelled vertex whose
// steepest neighbour in g differs from f's is a troublemaker. Wrong max label:
// decrease its ascending neighbour in g (Eq. 6). Wrong min label: decrease the
// descending neighbour that f prescribes.
template <class T, int ND>
__global__ void __launch_bounds__(kThreads) k_rcheck(Field<T> F) {
  DevState* st = F.st;
  if (st->action != ACT_LABELS || st->lstate != L_DONE || st->ljob != 1) return;
  const int n = F.G.n;
  uint32_t acc[4] = {0, 0, 0, 0};  // wrong max, wrong min, asc trouble, desc trouble
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const bool wM = F.Pup[v] != F.Mf[v];
    const bool wm = F.Pdn[v] != F.mf[v];
    acc[0] += wM;
    acc[1] += wm;
    if (wM || wm) {
      const uint8_t d = F.gdir[v], fd = F.fdir[v];
      if (wM && (d & 15) != (fd & 15)) {
        ++acc[2];
        request<T, ND>(F, v, v + slot_offset(d & 15, ND, F.G.nx, F.G.nxny));
      }
      if (wm && (d >> 4) != (fd >> 4)) {
        ++acc[3];
        request<T, ND>(F, v, v + slot_offset(fd >> 4, ND, F.G.nx, F.G.nxny));
      }
    }
  }
  block_add<4>(acc, st->acc_r);
  if (last_block(st) && threadIdx.x == 0) {
    const uint32_t wM = vload(&st->acc_r[0]), wm = vload(&st->acc_r[1]);
    const uint32_t ta = vload(&st->acc_r[2]), td = vload(&st->acc_r[3]);
    st->cnt.label_evals++;
    st->cnt.mismatch[0] += wM;
    st->cnt.mismatch[1] += wm;
    st->acc_r[0] = st->acc_r[1] = 0;
    st->ticks++;
    st->lstate = L_INIT;
    if (wM + wm == 0) {
      st->phase = PH_DONE;
      st->action = ACT_NONE;
    } else if (ta + td == 0) {
      st->phase = PH_ERR;
      st->status = MSZ_ERR_NOCONVERGE;
    } else {
      st->action = ACT_APPLY_R;
    }
    st->blocks_done = 0;
  }
}

// Applies the round's requests to the touched vertices only.
template <class T>
__global__ void __launch_bounds__(kThreads) k_apply(Field<T> F) {
  DevState* st = F.st;
  const uint32_t act = st->action;
  if (act != ACT_MARK_C && act != ACT_APPLY_R) return;
  const uint32_t nt = st->ntouch;
  uint32_t acc[2] = {0, 0};  // decreases, freezes
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nt; i += gridDim.x * blockDim.x) {
    const int u = (int)F.touched[i];
    uint8_t b = F.flags[u];
    if (b & FL_FREEZE) {
      F.g[u] = F.f[u];
      b = (uint8_t)((b & ~(FL_DEC | FL_FREEZE)) | FL_FROZEN | FL_EDITED);
      ++acc[1];
    } else if (b & FL_DEC) {
      F.g[u] = decrease(F.g[u], lower_bound_of(F.f[u], F.xi));
      b = (uint8_t)((b & ~FL_DEC) | FL_EDITED);
      ++acc[0];
    }
    F.flags[u] = b;
  }
  block_add<2>(acc, st->acc_ap);
  if (last_block(st) && threadIdx.x == 0) {
    st->cnt.dec_edits += vload(&st->acc_ap[0]);
    st->cnt.freezes += vload(&st->acc_ap[1]);
    st->ticks++;
    if (act == ACT_MARK_C) {
      const uint32_t t = st->T;
      st->cnt.c_rounds[t]++;
      st->cnt.c_cases[t] += st->counts[t];
    } else {
      st->cnt.r_rounds++;
      st->cnt.r_cases[0] += st->acc_r[2];
      st->cnt.r_cases[1] += st->acc_r[3];
      st->phase = PH_C;
      st->T = 0;
    }
    st->rounds++;
    if (st->rounds > st->max_rounds) {
      st->phase = PH_ERR;
      st->status = MSZ_ERR_NOCONVERGE;
    }
    st->action = ACT_NONE;
    st->ncase = st->ntouch = 0;
    st->counts[0] = st->counts[1] = st->counts[2] = st->counts[3] = 0;
    st->acc_ap[0] = st->acc_ap[1] = 0;
    st->acc_r[2] = st->acc_r[3] = 0;
    st->blocks_done = 0;
  }
}

// ---------------------------------------------------------------------------
// Edit list emission (Sec. 5.3): every vertex whose final value differs
// bitwise from fhat, ascending. Tiles of kEmitTile vertices; count, scan,
// write.
// ---------------------------------------------------------------------------
constexpr int kEmitItems = 16;
constexpr int kEmitTile = kThreads * kEmitItems;

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

template <class T>
__device__ __forceinline__ uint32_t emit_mask(const Field<T>& F, int base) {
  // bit k set iff vertex base + k is an edit (k < kEmitItems)
  const uint4 w = *reinterpret_cast<const uint4*>(F.flags + base);
  const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
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
__global__ void __launch_bounds__(kThreads) k_emit_count(Field<T> F) {
  if (F.st->phase != PH_DONE) return;
  const int base = blockIdx.x * kEmitTile + threadIdx.x * kEmitItems;
  uint32_t c[1] = {(uint32_t)__popc(emit_mask(F, base))};
  __shared__ uint32_t s;
  if (threadIdx.x == 0) s = 0;
  __syncthreads();
  uint32_t x = c[0];
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(&s, x);
  __syncthreads();
  if (threadIdx.x == 0) F.tile_cnt[blockIdx.x] = s;
}

// Exclusive scan of the tile counts by one block of 1024 threads.
template <class T>
__global__ void __launch_bounds__(1024) k_emit_scan(Field<T> F, int ntiles) {
  DevState* st = F.st;
  if (st->phase != PH_DONE) return;
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
      uint32_t w = warp_sums[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, w, o);
        if (lane >= o) w += y;
      }
      warp_sums[lane] = w;  // inclusive over warps
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
__global__ void __launch_bounds__(kThreads) k_emit_write(Field<T> F) {
  if (F.st->phase != PH_DONE) return;
  const int base = blockIdx.x * kEmitTile + threadIdx.x * kEmitItems;
  const uint32_t m = emit_mask(F, base);
  const uint32_t c = __popc(m);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t incl = c;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  __shared__ uint32_t ws[kThreads / 32];
  if (lane == 31) ws[wid] = incl;
  __syncthreads();
  uint32_t off = F.tile_cnt[blockIdx.x] + incl - c;
  for (int w = 0; w < wid; ++w) off += ws[w];
  uint32_t mm = m;
  while (mm) {
    const int k = __ffs(mm) - 1;
    mm &= mm - 1;
    const int v = base + k;
    F.edit_idx[off] = (uint32_t)v;
    F.edit_val[off] = F.g[v];
    ++off;
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
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < ne;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t i = idx[k];
    if (i < (uint32_t)n) dst[i] = val[k];
    else atomicOr(bad, 1u);
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static int g_num_sms = 0;
static std::mutex g_mu;

int num_sms() {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_num_sms == 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      sms = 152;
    g_num_sms = sms;
  }
  return g_num_sms;
}

bool geom_from(int ndim, const int64_t* dims, Geom& G) {
  if (ndim != 2 && ndim != 3) return false;
  if (!dims) return false;
  const int64_t nx = dims[0], ny = dims[1], nz = (ndim == 3) ? dims[2] : 1;
  if (nx < 1 || ny < 1 || nz < 1) return false;
  const int64_t n = nx * ny * nz;
  if (nx > 0x7fffffff || ny > 0x7fffffff || nz > 0x7fffffff || n > 0x7fffffffLL) return false;
  G.nx = (int)nx;
  G.ny = (int)ny;
  G.nz = (int)nz;
  G.nxny = (int)(nx * ny);
  G.n = (int)n;
  G.nd = ndim;
  return true;
}

size_t esize(int dtype) { return dtype == MSZ_F32 ? 4 : 8; }

constexpr int kMaxChunk = 32;  // steps launched between two state reads
constexpr int kKinds = 4;      // timed kernel kinds: sweep, labels, rcheck, mark+apply
size_t round_up(size_t a, size_t b) { return (a + b - 1) / b * b; }

}  // namespace msz

using namespace msz;

struct msz_plan_s {
  Geom G;
  int dtype;
  int device;
  msz_options opt;
  void* g = nullptr;
  uint8_t* fdir = nullptr;
  uint8_t* gdir = nullptr;
  uint8_t* flags = nullptr;
  uint32_t* fbits = nullptr;
  int nwords = 0;
  int32_t* Mf = nullptr;
  int32_t* mf = nullptr;
  int32_t* Pup = nullptr;
  int32_t* Pdn = nullptr;
  uint32_t* cases = nullptr;
  uint32_t* touched = nullptr;
  uint32_t* tile_cnt = nullptr;
  uint32_t* edit_idx = nullptr;
  void* edit_val = nullptr;
  void* in_f = nullptr;  // staging for msz_fix_host
  void* in_fhat = nullptr;
  DevState* st = nullptr;
  DevState* host_st = nullptr;  // pinned
  uint32_t* host_phase = nullptr;  // pinned
  uint64_t* host_ticks = nullptr;  // pinned
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int ntiles = 0;
  int dense_blocks = 0;
  int sparse_blocks = 0;
  bool use_tma = false;
  CUtensorMap tmap;  // g, float box with a one-vertex halo (NaN fill)
  CUtensorMap dmap;  // f's direction bytes, tile box
  SweepTiling tiling;
  int csweep_blocks = 0;
  int label_blocks = 0;
  int label_smem = 0;
  uint64_t launches = 0;  // kernel launches of the last fix
  // Optional per-kind kernel timing (MSZ_OPT_TIME_KERNELS): event pairs per
  // step of a chunk, read back after the chunk's synchronisation.
  cudaEvent_t tev[kMaxChunk][2 * kKinds] = {};
  bool tev_ready = false;
  double kernel_ms[kKinds] = {0, 0, 0, 0};
};

namespace {

struct Layout {
  size_t g, fdir, flags, lab, cases, tiles, edit_val, total;
};

Layout layout_of(const Geom& G, int dtype) {
  Layout L;
  const size_t n = (size_t)G.n;
  const size_t es = esize(dtype);
  const size_t ntiles = (n + kEmitTile - 1) / kEmitTile;
  L.g = round_up(n * es, 256);
  L.fdir = round_up(n, 256);
  L.flags = round_up(ntiles * kEmitTile, 256);
  L.lab = round_up(n * 4, 256);
  L.cases = round_up(n * 4, 256);
  L.tiles = round_up(ntiles * 4, 256);
  L.edit_val = round_up(n * es, 256);
  // g, fdir, gdir, flags, Mf, mf, Pup, Pdn, cases, touched, tiles, edit_idx,
  // edit_val, two staging buffers, state
  L.total = L.g + 2 * L.fdir + L.flags + 4 * L.lab + 2 * L.cases + L.tiles + L.cases + L.edit_val +
            2 * L.g + round_up(sizeof(DevState), 256);
  return L;
}

void free_plan(msz_plan_s* p) {
  void* ptrs[] = {p->g, p->fdir, p->gdir, p->flags, p->fbits, p->Mf, p->mf, p->Pup, p->Pdn, p->cases,
                  p->touched, p->tile_cnt, p->edit_idx, p->edit_val, p->in_f, p->in_fhat, p->st};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (p->host_st) cudaFreeHost(p->host_st);
  if (p->host_phase) cudaFreeHost(p->host_phase);
  if (p->host_ticks) cudaFreeHost(p->host_ticks);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->tev_ready)
    for (int i = 0; i < kMaxChunk; ++i)
      for (int j = 0; j < 2 * kKinds; ++j) cudaEventDestroy(p->tev[i][j]);
  if (p->ev1) cudaEventDestroy(p->ev1);
  delete p;
}

template <class T>
Field<T> field_of(msz_plan_s* p, const void* f, const void* fhat, double xi) {
  Field<T> F;
  F.f = static_cast<const T*>(f);
  F.fhat = static_cast<const T*>(fhat);
  F.g = static_cast<T*>(p->g);
  F.fdir = p->fdir;
  F.gdir = p->gdir;
  F.flags = p->flags;
  F.fbits = p->fbits;
  F.nwords = p->nwords;
  F.Mf = p->Mf;
  F.mf = p->mf;
  F.Pup = p->Pup;
  F.Pdn = p->Pdn;
  F.cases = p->cases;
  F.touched = p->touched;
  F.tile_cnt = p->tile_cnt;
  F.edit_idx = p->edit_idx;
  F.edit_val = static_cast<T*>(p->edit_val);
  F.st = p->st;
  F.xi = static_cast<T>(xi);
  F.G = p->G;
  return F;
}

constexpr int kJumpsPerStep = 4;

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

template <class T, int ND>
void sweep_tiling(msz_plan_s* p) {
  using SG = SweepGeom<T, ND>;
  const Geom& G = p->G;
  SweepTiling& TL = p->tiling;
  const int axis = (ND == 3) ? G.nz : G.ny;  // marching axis
  const int nchunks = (axis + 63) / 64;
  TL.chunk = (axis + nchunks - 1) / nchunks;
  TL.chunk += (4 - TL.chunk % 3) % 3;  // chunk + 2 planes per tile must be a multiple of 3
  TL.chunks = (axis + TL.chunk - 1) / TL.chunk;
  TL.tiles_x = (G.nx + SG::TX - 1) / SG::TX;
  TL.tiles_y = (ND == 3) ? (G.ny + SG::TY - 1) / SG::TY : 1;
  TL.ntiles = TL.tiles_x * TL.tiles_y * TL.chunks;
  int occ = 0;
  if (p->use_tma)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_csweep<T, ND, true>, SG::NTP, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_csweep<T, ND, false>, SG::NT, 0);
  if (occ < 1) occ = 1;
  p->csweep_blocks = std::max(1, std::min(TL.ntiles, occ * num_sms()));
}

template <class T, int ND>
bool encode_tmap(msz_plan_s* p) {
  using SG = SweepGeom<T, ND>;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const Geom& G = p->G;
  const cuuint64_t es = sizeof(T);
  if (((cuuint64_t)G.nx * es) % 16 != 0) return false;
  const CUtensorMapDataType dt = (sizeof(T) == 4) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  cuuint64_t gdim[3] = {(cuuint64_t)G.nx, (cuuint64_t)G.ny, (cuuint64_t)G.nz};
  cuuint64_t gstride[2] = {(cuuint64_t)G.nx * es, (cuuint64_t)G.nx * (cuuint64_t)G.ny * es};
  cuuint32_t box[3] = {(cuuint32_t)SG::BX, (cuuint32_t)SG::BY, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  const cuuint32_t rank = (ND == 3) ? 3 : 2;
  if ((cuuint64_t)G.nx % 16 != 0) return false;  // direction-byte rows must be 16-byte multiples too
  CUresult r = enc(&p->tmap, dt, rank, p->g, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NAN_REQUEST_ZERO_FMA);
  if (r != CUDA_SUCCESS) return false;
  cuuint64_t dstride[2] = {(cuuint64_t)G.nx, (cuuint64_t)G.nx * (cuuint64_t)G.ny};
  cuuint32_t dbox[3] = {(cuuint32_t)SG::TX, (cuuint32_t)((ND == 3) ? SG::TY : 1), 1};
  r = enc(&p->dmap, CU_TENSOR_MAP_DATA_TYPE_UINT8, rank, p->fdir, gdim, dstride, dbox, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <class T, int ND>
int setup_labels_t(msz_plan_s* p) {
  using LG = LabelGeom<ND>;
  const Geom& G = p->G;
  p->label_smem = (int)(((LG::HALO * sizeof(T) + 15) / 16) * 16 + 2 * ((LG::HALO + 7) / 8) * 8 * sizeof(uint16_t));
  if (cudaFuncSetAttribute(k_label_tile<T, ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, p->label_smem) !=
      cudaSuccess)
    return MSZ_ERR_CUDA;
  const int ntiles = ((G.nx + LG::TX - 1) / LG::TX) * ((G.ny + LG::TY - 1) / LG::TY) * ((G.nz + LG::TZ - 1) / LG::TZ);
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_label_tile<T, ND>, kThreads, p->label_smem);
  if (occ < 1) occ = 1;
  p->label_blocks = std::max(1, std::min(ntiles, occ * num_sms()));
  return MSZ_OK;
}

template <class T, int ND>
int setup_sweep_t(msz_plan_s* p) {
  if (setup_labels_t<T, ND>(p) != MSZ_OK) return MSZ_ERR_CUDA;
  std::memset(&p->tmap, 0, sizeof(p->tmap));
  std::memset(&p->dmap, 0, sizeof(p->dmap));
  p->use_tma = !(p->opt.flags & MSZ_OPT_NO_TMA) && encode_tmap<T, ND>(p);
  sweep_tiling<T, ND>(p);
  return cudaGetLastError() == cudaSuccess ? MSZ_OK : MSZ_ERR_CUDA;
}

int setup_sweep(msz_plan_s* p) {
  if (p->dtype == MSZ_F32) return p->G.nd == 3 ? setup_sweep_t<float, 3>(p) : setup_sweep_t<float, 2>(p);
  return p->G.nd == 3 ? setup_sweep_t<double, 3>(p) : setup_sweep_t<double, 2>(p);
}

template <class T, int ND>
void launch_step(msz_plan_s* p, const Field<T>& F, cudaStream_t s, int slot) {
  const int db = p->dense_blocks, sb = p->sparse_blocks;
  constexpr int NT = SweepGeom<T, ND>::NT;
  constexpr int NTP = SweepGeom<T, ND>::NTP;
  cudaEvent_t* e = (slot >= 0) ? p->tev[slot] : nullptr;
  if (e) cudaEventRecord(e[0], s);
  if (p->use_tma) k_csweep<T, ND, true><<<p->csweep_blocks, NTP, 0, s>>>(F, p->tmap, p->dmap, p->tiling);
  else k_csweep<T, ND, false><<<p->csweep_blocks, NT, 0, s>>>(F, p->tmap, p->dmap, p->tiling);
  if (e) cudaEventRecord(e[1], s);
  if (e) cudaEventRecord(e[6], s);
  k_mark_c<T, ND><<<sb, kThreads, 0, s>>>(F);
  if (e) cudaEventRecord(e[2], s);
  k_label_tile<T, ND><<<p->label_blocks, kThreads, p->label_smem, s>>>(F);
  for (int j = 0; j < kJumpsPerStep; ++j) k_jump<T><<<db, kThreads, 0, s>>>(F);
  if (e) cudaEventRecord(e[3], s);
  if (e) cudaEventRecord(e[4], s);
  k_rcheck<T, ND><<<db, kThreads, 0, s>>>(F);
  if (e) cudaEventRecord(e[5], s);
  k_apply<T><<<sb, kThreads, 0, s>>>(F);
  if (e) cudaEventRecord(e[7], s);
  p->launches += 6 + kJumpsPerStep;
}

// Adds the event times of the last chunk's steps to the per-kind totals
// (mark+apply = e6..e2 plus e5..e7 minus nothing: the mark span e6..e2 and
// the apply span e5..e7).
void collect_times(msz_plan_s* p, int steps) {
  for (int i = 0; i < steps; ++i) {
    float a = 0, b = 0, c = 0, d1 = 0, d2 = 0;
    cudaEvent_t* e = p->tev[i];
    cudaEventElapsedTime(&a, e[0], e[1]);
    cudaEventElapsedTime(&b, e[2], e[3]);
    cudaEventElapsedTime(&c, e[4], e[5]);
    cudaEventElapsedTime(&d1, e[6], e[2]);
    cudaEventElapsedTime(&d2, e[5], e[7]);
    p->kernel_ms[0] += a;
    p->kernel_ms[1] += b;
    p->kernel_ms[2] += c;
    p->kernel_ms[3] += d1 + d2;
  }
}

template <class T, int ND>
int run_fix(msz_plan_s* p, const void* f, const void* fhat, double xi, cudaStream_t s, msz_result* out) {
  const Field<T> F = field_of<T>(p, f, fhat, xi);
  DevState init;
  std::memset(&init, 0, sizeof(init));
  init.phase = PH_INIT;
  init.max_rounds = p->opt.max_rounds ? p->opt.max_rounds : 10000000ull;
  std::memcpy(p->host_st, &init, sizeof(init));
  if (cudaMemcpyAsync(p->st, p->host_st, sizeof(DevState), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return MSZ_ERR_CUDA;
  if (p->ev0) cudaEventRecord(p->ev0, s);
  p->launches = 0;
  k_init<T, ND><<<p->dense_blocks, kThreads, 0, s>>>(F);
  p->launches += 1;
  // Steps in growing chunks; one small state read per chunk. Every step
  // advances the state machine at least once unless the field is finished,
  // so a chunk without a state transition is reported as a stall.
  int chunk = 2;
  uint64_t last_ticks = ~0ull;
  const bool timed = (p->opt.flags & MSZ_OPT_TIME_KERNELS) != 0;
  if (timed && !p->tev_ready) {
    for (int i = 0; i < kMaxChunk; ++i)
      for (int j = 0; j < 2 * kKinds; ++j) cudaEventCreate(&p->tev[i][j]);
    p->tev_ready = true;
  }
  for (int k = 0; k < kKinds; ++k) p->kernel_ms[k] = 0.0;
  for (;;) {
    for (int i = 0; i < chunk; ++i) launch_step<T, ND>(p, F, s, timed ? i : -1);
    cudaMemcpyAsync(p->host_phase, &p->st->phase, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(p->host_ticks, &p->st->ticks, sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return MSZ_ERR_CUDA;
    if (timed) collect_times(p, chunk);
    const uint32_t ph = *p->host_phase;
    if (ph == PH_DONE || ph == PH_ERR) break;
    if (*p->host_ticks == last_ticks) return MSZ_ERR_TIMEOUT;
    last_ticks = *p->host_ticks;
    chunk = std::min(chunk * 2, kMaxChunk);
  }
  k_emit_count<T><<<p->ntiles, kThreads, 0, s>>>(F);
  k_emit_scan<T><<<1, 1024, 0, s>>>(F, p->ntiles);
  k_emit_write<T><<<p->ntiles, kThreads, 0, s>>>(F);
  p->launches += 3;
  if (p->ev1) cudaEventRecord(p->ev1, s);
  cudaMemcpyAsync(p->host_st, p->st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return MSZ_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess) return MSZ_ERR_CUDA;
  const DevState& H = *p->host_st;
  int status = (H.phase == PH_DONE) ? MSZ_OK : (H.status ? H.status : MSZ_ERR_CUDA);
  if (out) {
    std::memset(out, 0, sizeof(*out));
    out->status = status;
    out->counts = H.cnt;
    if (status == MSZ_OK) {
      out->edit_idx = p->edit_idx;
      out->edit_val = p->edit_val;
      out->n_edits = H.n_edits;
      out->label_max = p->Pup;
      out->label_min = p->Pdn;
    }
    float ms = 0.f;
    if (p->ev0 && p->ev1 && cudaEventElapsedTime(&ms, p->ev0, p->ev1) == cudaSuccess) out->device_ms = ms;
    out->launches = p->launches;
    for (int k = 0; k < kKinds; ++k) out->kernel_ms[k] = (float)p->kernel_ms[k];
  }
  return status;
}

int dispatch_fix(msz_plan_s* p, const void* f, const void* fhat, double xi, cudaStream_t s,
                 msz_result* out) {
  if (p->dtype == MSZ_F32) {
    return p->G.nd == 3 ? run_fix<float, 3>(p, f, fhat, xi, s, out)
                        : run_fix<float, 2>(p, f, fhat, xi, s, out);
  }
  return p->G.nd == 3 ? run_fix<double, 3>(p, f, fhat, xi, s, out)
                      : run_fix<double, 2>(p, f, fhat, xi, s, out);
}

bool xi_ok(double xi, int dtype) {
  if (!(xi >= 0.0) || !std::isfinite(xi)) return false;
  if (dtype == MSZ_F32 && !std::isfinite((float)xi)) return false;
  return true;
}

}  // namespace

extern "C" {

int64_t msz_plan_bytes(int ndim, const int64_t dims[3], int dtype) {
  Geom G;
  if (!geom_from(ndim, dims, G)) return MSZ_ERR_ARG;
  if (dtype != MSZ_F32 && dtype != MSZ_F64) return MSZ_ERR_DTYPE;
  return (int64_t)layout_of(G, dtype).total;
}

int msz_plan_create(msz_plan* out, int ndim, const int64_t dims[3], int dtype, const msz_options* opt) {
  if (!out) return MSZ_ERR_ARG;
  *out = nullptr;
  Geom G;
  if (!geom_from(ndim, dims, G)) return MSZ_ERR_ARG;
  if (dtype != MSZ_F32 && dtype != MSZ_F64) return MSZ_ERR_DTYPE;
  msz_plan_s* p = new (std::nothrow) msz_plan_s();
  if (!p) return MSZ_ERR_OOM;
  p->G = G;
  p->dtype = dtype;
  cudaGetDevice(&p->device);
  std::memset(&p->opt, 0, sizeof(p->opt));
  if (opt) p->opt = *opt;
  const Layout L = layout_of(G, dtype);
  const size_t n = (size_t)G.n;
  const size_t es = esize(dtype);
  p->ntiles = (int)((n + kEmitTile - 1) / kEmitTile);
  bool ok = true;
  auto alloc = [&](void** q, size_t bytes) {
    if (ok && cudaMalloc(q, bytes) != cudaSuccess) ok = false;
  };
  alloc(&p->g, L.g);
  alloc((void**)&p->fdir, L.fdir);
  alloc((void**)&p->gdir, L.fdir);
  alloc((void**)&p->flags, L.flags);
  alloc((void**)&p->Mf, L.lab);
  alloc((void**)&p->mf, L.lab);
  alloc((void**)&p->Pup, L.lab);
  alloc((void**)&p->Pdn, L.lab);
  alloc((void**)&p->cases, L.cases);
  alloc((void**)&p->touched, L.cases);
  alloc((void**)&p->tile_cnt, L.tiles);
  alloc((void**)&p->edit_idx, L.cases);
  alloc(&p->edit_val, L.edit_val);
  alloc((void**)&p->st, round_up(sizeof(DevState), 256));
  if (ok && cudaMallocHost((void**)&p->host_st, sizeof(DevState)) != cudaSuccess) ok = false;
  if (ok && cudaMallocHost((void**)&p->host_phase, 4 * sizeof(uint64_t)) != cudaSuccess) ok = false;
  if (ok && cudaMallocHost((void**)&p->host_ticks, sizeof(uint64_t)) != cudaSuccess) ok = false;
  if (ok && (cudaEventCreate(&p->ev0) != cudaSuccess || cudaEventCreate(&p->ev1) != cudaSuccess)) ok = false;
  if (ok && cudaMemset(p->flags, 0, L.flags) != cudaSuccess) ok = false;
  if (!ok) {
    cudaGetLastError();
    free_plan(p);
    return MSZ_ERR_OOM;
  }
  (void)es;
  p->nwords = (int)((n + 31) / 32);
  if (cudaMalloc((void**)&p->fbits, (size_t)p->nwords * 8) != cudaSuccess) {
    cudaGetLastError();
    free_plan(p);
    return MSZ_ERR_OOM;
  }
  if (setup_sweep(p) != MSZ_OK) {
    free_plan(p);
    return MSZ_ERR_CUDA;
  }
  const int sms = num_sms();
  p->dense_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((G.n + kThreads - 1) / kThreads, (int64_t)sms * 8));
  p->sparse_blocks = sms * 4;
  *out = p;
  return MSZ_OK;
}

int msz_plan_destroy(msz_plan p) {
  if (!p) return MSZ_ERR_ARG;
  cudaDeviceSynchronize();
  free_plan(p);
  return MSZ_OK;
}

int msz_fix(msz_plan p, const void* orig_dev, const void* decomp_dev, double xi, void* stream,
            msz_result* out) {
  if (out) std::memset(out, 0, sizeof(*out));
  if (!p || !orig_dev || !decomp_dev) return out ? (out->status = MSZ_ERR_ARG) : MSZ_ERR_ARG;
  if (!xi_ok(xi, p->dtype)) return out ? (out->status = MSZ_ERR_ARG) : MSZ_ERR_ARG;
  const int st = dispatch_fix(p, orig_dev, decomp_dev, xi, static_cast<cudaStream_t>(stream), out);
  if (out) out->status = st;
  return st;
}

int msz_fix_host(msz_plan p, const void* orig_host, const void* decomp_host, double xi,
                 uint32_t* edit_idx_host, void* edit_val_host, int32_t* label_max_host,
                 int32_t* label_min_host, void* stream, msz_result* out) {
  if (out) std::memset(out, 0, sizeof(*out));
  if (!p || !orig_host || !decomp_host || !edit_idx_host || !edit_val_host) return MSZ_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)p->G.n * esize(p->dtype);
  if (!p->in_f || !p->in_fhat) {
    if ((!p->in_f && cudaMalloc(&p->in_f, bytes) != cudaSuccess) ||
        (!p->in_fhat && cudaMalloc(&p->in_fhat, bytes) != cudaSuccess)) {
      cudaGetLastError();
      return MSZ_ERR_OOM;
    }
  }
  if (cudaMemcpyAsync(p->in_f, orig_host, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(p->in_fhat, decomp_host, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return MSZ_ERR_CUDA;
  msz_result r;
  const int st = msz_fix(p, p->in_f, p->in_fhat, xi, stream, &r);
  if (st != MSZ_OK) {
    if (out) *out = r;
    return st;
  }
  const size_t ne = (size_t)r.n_edits;
  if (ne) {
    if (cudaMemcpyAsync(edit_idx_host, r.edit_idx, ne * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(edit_val_host, r.edit_val, ne * esize(p->dtype), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess)
      return MSZ_ERR_CUDA;
  }
  if (label_max_host)
    cudaMemcpyAsync(label_max_host, r.label_max, (size_t)p->G.n * 4, cudaMemcpyDeviceToHost, s);
  if (label_min_host)
    cudaMemcpyAsync(label_min_host, r.label_min, (size_t)p->G.n * 4, cudaMemcpyDeviceToHost, s);
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
  const int blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>((n_edits + kThreads - 1) / kThreads,
                                                                    (uint64_t)num_sms() * 8));
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
    default: return "unknown status";
  }
}

const char* msz_version(void) { return "msz-gb300 0.1"; }

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

// Device address of the scratch array on the current device (set up once).
int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MSZ_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return MSZ_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  return MSZ_OK;
}

// Carves the loop's scratch out of [base, base + cap); false if it does not fit.
bool carve_noalloc(msz_plan_s* p, unsigned char* base, size_t cap) {
  const Geom& G = p->G;
  const size_t n = (size_t)G.n;
  const size_t es = esize(p->dtype);
  const size_t ntiles = (n + kEmitTile - 1) / kEmitTile;
  size_t off = 0;
  auto take = [&](size_t bytes) -> unsigned char* {
    unsigned char* q = base + off;
    off += round_up(bytes, 256);
    return q;
  };
  p->g = take(n * es);
  p->fdir = take(n);
  p->gdir = take(n);
  p->flags = take(ntiles * kEmitTile);
  p->Mf = reinterpret_cast<int32_t*>(take(n * 4));
  p->mf = reinterpret_cast<int32_t*>(take(n * 4));
  p->cases = reinterpret_cast<uint32_t*>(take(n * 4));
  p->touched = reinterpret_cast<uint32_t*>(take(n * 4));
  p->tile_cnt = reinterpret_cast<uint32_t*>(take(ntiles * 4));
  p->st = reinterpret_cast<DevState*>(take(sizeof(DevState)));
  p->ntiles = (int)ntiles;
  return off <= cap;
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
  // A plan whose arrays point into the static scratch and the caller's
  // outputs; host-side state lives on this stack frame (pageable memory).
  msz_plan_s P;
  P.G = G;
  P.dtype = dtype;
  cudaGetDevice(&P.device);
  std::memset(&P.opt, 0, sizeof(P.opt));
  if (!carve_noalloc(&P, static_cast<unsigned char*>(base), kNoAllocScratchBytes)) return fail(MSZ_ERR_TOO_LARGE);
  P.Pup = label_max_dev;
  P.Pdn = label_min_dev;
  P.edit_idx = edit_idx_dev;
  P.edit_val = edit_val_dev;
  DevState host_state;
  uint32_t host_phase[2] = {0, 0};
  uint64_t host_ticks = 0;
  P.host_st = &host_state;
  P.host_phase = host_phase;
  P.host_ticks = &host_ticks;
  const int sms = num_sms();
  P.dense_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((G.n + kThreads - 1) / kThreads, (int64_t)sms * 8));
  P.sparse_blocks = sms * 4;
  if (setup_sweep(&P) != MSZ_OK) return fail(MSZ_ERR_CUDA);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(P.flags, 0, (size_t)P.ntiles * kEmitTile, s) != cudaSuccess) return fail(MSZ_ERR_CUDA);
  msz_result r;
  const int st = dispatch_fix(&P, orig_dev, decomp_dev, xi, s, &r);
  // P owns nothing: clear the pointers so that no destructor-like path frees them
  P.host_st = nullptr;
  P.host_phase = nullptr;
  P.host_ticks = nullptr;
  if (out) {
    *out = r;
    out->status = st;
  }
  return st;
}
