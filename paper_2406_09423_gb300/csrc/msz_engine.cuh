// Multi-field engine of the MSz correction loop: per-field state machine,
// work-unit kernels and the host-side group/engine machinery. One engine runs
// one field (msz_fix, msz_fix_noalloc) or many of uneven sizes and mixed
// float32 / float64 (msz_batch_*, msz_server_*) through the same kernels.
//
// Every kernel walks "units" (vertex chunks, sweep tiles, label tiles, list
// slices) of all fields of a (dtype, dimension) group; a unit finds its field
// through prefix sums, checks that field's state and skips it when the field
// has nothing to do in this kernel (per-field convergence mask). The unit that
// completes a field's work in a kernel advances that field's state machine.
// The host launches a fixed sequence of kernels per step (captured once in a
// CUDA graph) and reads the fields' states once per chunk of steps.
//
// Paper references (Li et al., MSz): Sec. 3 (PL field, critical points,
// integral lines, labels), Sec. 4.1 (false critical points, Eqs. 1-5),
// Sec. 4.2 (troublemaker, Eq. 6), Sec. 5 (parallel C-loop / R-loop, lock-free
// lists, deterministic conflict resolution), Sec. 5.3 (edit list).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <stdint.h>

#include "msz.h"
#include "msz_device.cuh"
#include "msz_sweep.cuh"

namespace msz {

enum : uint32_t { PH_INIT = 0, PH_FLABELS = 1, PH_C = 2, PH_R = 3, PH_DONE = 4, PH_ERR = 5, PH_PARKED = 6 };
// PH_PARKED: no kernel serves this phase (MSZ_OPT_TEST_STALL, a test of the
// host's stall detection): the field's state never moves.
// Actions within a phase. In PH_C, ACT_NONE means the field's first (full)
// classification sweep is pending; afterwards a C round runs ACT_GATHER
// (list the cases of the current type), ACT_REQUEST (their requests),
// ACT_MARK_C (apply) and ACT_RECLASS (reclassify the closed 1-rings of the
// edited vertices).
enum : uint32_t {
  ACT_NONE = 0, ACT_MARK_C = 1, ACT_LABELS = 2, ACT_APPLY_R = 3, ACT_GATHER = 4, ACT_RECLASS = 5, ACT_REQUEST = 6
};
// Stages of one label evaluation (job 0: f, job 1: g): tile terminals with
// the first-level exit-table entries of the recomputed tiles, pointer
// jumping on the exit tables, then f's labels in place (job 0) or the
// R-loop check.
enum : uint32_t { L_INIT = 0, L_JUMP = 1, L_DONE = 2 };
// Tile terminal flag: the terminal is an extremum (else a tile exit).
constexpr uint32_t kExt = 0x80000000u;
// Exit-table entry flag: the entry holds the exit's label (an extremum),
// else the slot of the next exit on its line.
constexpr uint32_t kRes = 0x80000000u;
enum : uint32_t { E_NONFINITE = 1, E_ARG = 2, E_BOUND = 4, E_TIMEOUT = 8, E_CHECK = 16 };

// Work-unit kinds.
enum { K_DENSE = 0, K_SWEEP = 1, K_LABEL = 2, K_SPARSE = 3, K_EMIT = 4, K_CASE = 5, NKIND = 6 };
constexpr int kDenseChunk = 8192;  // vertices per dense unit
constexpr int kEmitItems = 16;
constexpr int kEmitTile = kThreads * kEmitItems;  // vertices per emission unit and per case-count tile
constexpr int kTilesPerWarp = 4;                   // case-count tiles a gather warp checks at once
constexpr int kCaseTiles = kTilesPerWarp * kThreads / 32;  // case-count tiles per gather unit

// Kernels of a loop step, in launch order of their kinds (per-kernel timing).
enum {
  KID_SWEEP = 0, KID_GATHER, KID_MARK, KID_LABEL, KID_JUMP, KID_RCHECK, KID_APPLY, KID_RECLASS, KID_CSMALL, NKID
};

constexpr int kStripes = 16;

// Per-field device state (one contiguous array per engine).
struct DevState {
  uint32_t phase, action, T, lstate, ljob, units_done, err_bits;
  int32_t status;
  uint32_t counts[4];  // false critical points of g per type (kept current by every classification)
  uint32_t ntouch;  // entries of the touched list (apply, then reclassification)
  uint32_t ncase;   // entries of the case list (the round's cases of the current type)
  uint32_t acc_changed;
  uint32_t acc_ap[2];  // apply: decreases, freezes
  uint32_t acc_r[4];   // rcheck: wrong max, wrong min, asc troublemakers, desc troublemakers
  // Blocks add their partial counters to stripe blockIdx % kStripes (not one
  // address: same-address atomics serialise in L2); the completing thread
  // folds the stripes into the counters above (see fold_stripes).
  uint32_t stripe[kStripes][4];
  uint32_t jump_rounds, emitted;
  uint64_t rounds, max_rounds, n_edits;
  uint64_t ticks;  // advanced by every state transition (stall detection)
  uint64_t kunits[NKID];  // work units per kernel (kernel timing runs only)
  msz_counts cnt;
};

// Per-field descriptor (device array per group).
template <class T>
struct Field {
  const T* f;
  const T* fhat;
  T* g;
  uint8_t* fdir;
  uint8_t* gdir;
  uint8_t* flags;
  int32_t* Mf;    // f's labels once f's evaluation is done: the output arrays Pup / Pdn,
  int32_t* mf;    // which hold the final labels once the field has converged (g's equal f's)
  int32_t* Pup;   // outputs: max / min labels
  int32_t* Pdn;
  uint32_t* term; // tile terminals (kTermFlag form) of the current evaluation
  // per direction (0: ascending lines / max labels, 1: descending / min)
  // exit tables, one slot per face cell of every label tile (exit_slot)
  uint32_t* lf[2];  // first-level entries: a label (kRes) or the slot of the next exit on the line
  uint32_t* lw[2];  // entries being resolved by the jumping; lw[0] is the C-loop's freeze list
  uint8_t* xm[2];   // 1: the slot is an exit of some tile's lines (cleared when a fix starts)
  uint32_t nface;   // slots per direction (label tiles times face cells, a multiple of 16)
  uint32_t fz_cap;  // entries of lw[0] (at least nface; room for a launch's freezes in k_csmall)
  uint8_t* tdirty;  // per label tile: bit 0 terminals to recompute, bit 1 recomputed and not yet checked
  uint32_t* texit;  // per label tile and direction: bitmap over the shell cells its lines leave through
  uint32_t* tsnap;  // per label tile, in the order of its exit list: each exit's label at the tile's last check
  uint8_t* twrong;  // per label tile: its last check found a wrong label
  uint8_t* cls;     // false-type bits of g per vertex (FPmax, FPmin, FNmax, FNmin), padded to kEmitTile
  uint32_t* cases;  // the round's cases of the current type
  uint32_t* epoch;  // round in which a vertex was last reclassified (claims a vertex once per round)
  uint32_t* ccnt;   // false critical points per kEmitTile-vertex tile and type: [tile][4]
  uint32_t* touched;
  uint32_t* tile_cnt;
  uint32_t* edit_idx;
  T* edit_val;
  DevState* st;
  T xi;
  Geom G;
  SweepTiling TL;
  int units[NKIND];
  int small_cluster;  // blocks of the cluster that runs the field's small C-loop rounds
};

// Kernel argument: one (dtype, dimension) group of fields.
template <class T>
struct GroupArgs {
  const Field<T>* fields;
  const int* prefix;        // [NKIND][nf + 1]
  const CUtensorMap* maps;  // [2 * nf]: g (halo box, NaN fill), f's direction bytes
  int nf;
  int total[NKIND];
  // Kernel timing runs only (null otherwise): the launch's step and slot; the
  // block completing a field's work sets bit `slot` of steplog[step].
  uint32_t* steplog;
  int step, slot;
  // launch parameters (msz_tuning): exit-table steps an entry follows per
  // k_jump launch; C-loop rounds a k_csmall launch may run and the largest
  // round (cases) it takes
  int chase, small_rounds;
  uint32_t small_cases;
};

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t vload(const uint32_t* p) { return *(volatile const uint32_t*)p; }

// Bounds checks of the checked build (compiled with -DMSZ_CHECKED): an index
// read from data (a list entry, a list slot, a pointer, a table rank) that
// lies outside [0, n) sets E_CHECK in the field's error bits and the access
// it guards is skipped; the fix then ends with MSZ_ERR_CHECK. The normal
// build compiles the checks away.
#ifdef MSZ_CHECKED
__device__ __forceinline__ bool msz_in_range(DevState* st, long long i, long long n) {
  if (i >= 0 && i < n) return true;
  atomicOr(&st->err_bits, E_CHECK);
  return false;
}
#define MSZ_IN(st, i, n) msz_in_range((st), (long long)(i), (long long)(n))
#else
#define MSZ_IN(st, i, n) true
#endif

// Field owning global unit u of a kind: pre[i] <= u < pre[i + 1].
__device__ __forceinline__ int field_of_unit(const int* pre, int nf, int u) {
  int lo = 0, hi = nf;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(pre + mid) <= u) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Kernel timing runs: this launch did work (moved a field's state machine),
// and the work units it processed.
template <class T>
__device__ __forceinline__ void log_work(const GroupArgs<T>& A) {
  if (A.steplog) atomicOr(&A.steplog[A.step], 1u << A.slot);
}
template <class T>
__device__ __forceinline__ void log_units(const GroupArgs<T>& A, DevState* st, int kid, uint64_t n) {
  if (A.steplog && n) atomicAdd((unsigned long long*)&st->kunits[kid], (unsigned long long)n);
}

// The same summed over a warp (every lane calls it).
template <class T>
__device__ __forceinline__ void log_units_warp(const GroupArgs<T>& A, DevState* st, int kid, uint32_t n) {
  if (!A.steplog) return;
  n = __reduce_add_sync(kFull, n);
  if ((threadIdx.x & 31) == 0 && n) atomicAdd((unsigned long long*)&st->kunits[kid], (unsigned long long)n);
}

// Sparse kernels: the units of a field (S fixed at setup) share a list of
// `items` entries known only at run time; only as many units as give each
// thread about one entry take part (returned; they alone count towards the
// field's completion), so short lists still spread over many blocks and idle
// blocks report nothing. [b, e) is unit k's slice (empty for the others).
__device__ __forceinline__ uint32_t sparse_slice(uint64_t items, int S, int k, uint64_t& b, uint64_t& e,
                                                 uint32_t per_unit = kThreads) {
  const uint64_t want = (items + per_unit - 1) / per_unit;
  const uint64_t act = want < (uint64_t)S ? (want ? want : 1) : (uint64_t)S;
  // slices of ceil(items / act) entries (the last one shorter); 32-bit
  // division when the list allows (always in practice)
  const uint64_t chunk = (items < (1ull << 32)) ? (uint64_t)(((uint32_t)items + (uint32_t)act - 1u) / (uint32_t)act)
                                                : (items + act - 1) / act;
  b = (uint64_t)k < act ? min(items, chunk * (uint64_t)k) : 0;
  e = (uint64_t)k < act ? min(items, b + chunk) : 0;
  return (uint32_t)act;
}

// Completion of one unit of a field by the whole block: true in the block
// that completes the field's last unit (all other units' writes visible).
__device__ __forceinline__ bool unit_done(DevState* st, int units) {
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&st->units_done, 1u) == (uint32_t)(units - 1);
  __syncthreads();
  if (s_last) __threadfence();
  return s_last;
}

// The same for n units of one field completed by the block at once.
__device__ __forceinline__ bool units_done_n(DevState* st, uint32_t n, int units) {
  __shared__ bool s_last_n;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last_n = atomicAdd(&st->units_done, n) + n == (uint32_t)units;
  __syncthreads();
  if (s_last_n) __threadfence();
  return s_last_n;
}

// Per-block completion of a kernel's units, reported per field: the block
// counts the units it completes of its current field and reports them with
// one atomic when it moves to another field or runs out of units (instead of
// one per unit: same-address atomics serialise in L2). flush() first runs
// pre(st) in every thread (the kernel's own counters), then, in the block
// that completes the field, done(st) in thread 0.
struct UnitTally {
  int cur = -1;
  uint32_t n = 0;
  uint32_t target = 0;  // units that complete the field (0: all of the kind's units)
  template <class T, class Pre, class Done>
  __device__ __forceinline__ void flush(const GroupArgs<T>& A, int kind, Pre&& pre, Done&& done) {
    if (cur < 0) return;
    DevState* st = A.fields[cur].st;
    pre(st);
    if (units_done_n(st, n, target ? (int)target : A.fields[cur].units[kind]) && threadIdx.x == 0) {
      done(st);
      st->units_done = 0;
    }
    n = 0;
  }
  // at the start of a unit of field i
  template <class T, class Pre, class Done>
  __device__ __forceinline__ void enter(const GroupArgs<T>& A, int kind, int i, Pre&& pre, Done&& done) {
    if (i != cur) {
      flush(A, kind, pre, done);
      cur = i;
    }
    ++n;
  }
};

template <int NW>
__device__ __forceinline__ void block_add(uint32_t (&v)[NW], uint32_t* dst) {
  __shared__ uint32_t s[NW];
  __syncthreads();
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

// block_add into the block's stripe of st->stripe (counters 0 .. NW-1).
template <int NW>
__device__ __forceinline__ void block_add_striped(uint32_t (&v)[NW], DevState* st) {
  block_add<NW>(v, &st->stripe[blockIdx.x % kStripes][0]);
}

// Sums the stripes of counters 0 .. nw-1 into dst (mod 2^32) and clears them.
__device__ __forceinline__ void fold_stripes(DevState* st, uint32_t* dst, int nw) {
  for (int k = 0; k < nw; ++k) {
    uint32_t sum = 0;
    for (int s = 0; s < kStripes; ++s) {
      sum += vload(&st->stripe[s][k]);
      st->stripe[s][k] = 0;
    }
    dst[k] += sum;
  }
}

// ---------------------------------------------------------------------------
// State transitions (run by one thread of the block completing the field)
// ---------------------------------------------------------------------------
__device__ void ctrl_after_init(DevState* st) {
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
}

// C-loop control after a classification of g (the full sweep or the
// incremental one after an apply; Sec. 4.1): the next sub-loop type with
// cases, the end of a pass after FNmin, or the R-loop when a whole pass is
// clean. The type counts are those of the current g, so advancing the type
// needs no new sweep. _counted: the classification's count changes are
// already in st->counts (a single writer); the other form first folds them
// in from the stripes.
__device__ void ctrl_after_classify_counted(DevState* st) {
  uint32_t c[4];
  for (int t = 0; t < 4; ++t) c[t] = vload(&st->counts[t]);
  st->ntouch = st->ncase = 0;
  if (vload(&st->err_bits) & E_TIMEOUT) {
    st->phase = PH_ERR;
    st->status = MSZ_ERR_TIMEOUT;
    st->ticks++;
    return;
  }
  st->cnt.sweeps++;
  uint32_t T_ = st->T;
  for (;;) {
    if (c[T_]) { st->action = ACT_GATHER; break; }
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

__device__ void ctrl_after_classify(DevState* st) {
  fold_stripes(st, st->counts, 4);  // the reclassification's count changes
  ctrl_after_classify_counted(st);
}

__device__ void ctrl_after_jump(DevState* st) {
  fold_stripes(st, &st->acc_changed, 1);
  const uint32_t c = vload(&st->acc_changed);
  st->acc_changed = 0;
  st->jump_rounds++;
  st->ticks++;
  if (c == 0) {
    st->lstate = L_DONE;
  } else if (st->jump_rounds > 64) {
    st->phase = PH_ERR;
    st->status = MSZ_ERR_TIMEOUT;
  }
}

// End of f's evaluation (its labels are in Mf / mf): the C-loop starts with
// the full classification sweep.
__device__ void ctrl_after_flabels(DevState* st) {
  st->phase = PH_C;
  st->action = ACT_NONE;
  st->T = 0;
  st->ticks++;
}

__device__ void ctrl_after_rcheck(DevState* st) {
  fold_stripes(st, st->acc_r, 4);
  const uint32_t wM = vload(&st->acc_r[0]), wm = vload(&st->acc_r[1]);
  const uint32_t ta = vload(&st->acc_r[2]), td = vload(&st->acc_r[3]);
  st->cnt.label_evals++;
  st->cnt.mismatch[0] += wM;
  st->cnt.mismatch[1] += wm;
  st->acc_r[0] = st->acc_r[1] = 0;
  st->lstate = L_INIT;
  st->ticks++;
  if (wM + wm == 0) {
    st->phase = PH_DONE;
    st->action = ACT_NONE;
  } else if (ta + td == 0) {
    st->phase = PH_ERR;  // cannot happen once the extremum sets agree
    st->status = MSZ_ERR_NOCONVERGE;
  } else {
    st->action = ACT_APPLY_R;
  }
}

// Round bookkeeping after an apply (act: the C-loop's requests or the
// R-loop's). _counted: the apply's sums are already in st->acc_ap (a single
// writer); the other form first folds them in from the stripes.
__device__ void ctrl_after_apply_counted(DevState* st, uint32_t act) {
  st->cnt.dec_edits += vload(&st->acc_ap[0]);
  st->cnt.freezes += vload(&st->acc_ap[1]);
  st->ticks++;
  if (act == ACT_MARK_C) {
    const uint32_t t = st->T;
    st->cnt.c_rounds[t]++;
    st->cnt.c_cases[t] += st->counts[t];  // the cases of this round (counts are pre-apply)
  } else {
    st->cnt.r_rounds++;
    st->cnt.r_cases[0] += st->acc_r[2];
    st->cnt.r_cases[1] += st->acc_r[3];
    st->phase = PH_C;
    st->T = 0;
  }
  st->rounds++;
  // the touched list stays for the reclassification that follows
  st->action = ACT_RECLASS;
  if (st->rounds > st->max_rounds) {
    st->phase = PH_ERR;
    st->status = MSZ_ERR_NOCONVERGE;
    st->action = ACT_NONE;
  }
  st->acc_ap[0] = st->acc_ap[1] = 0;
  st->acc_r[2] = st->acc_r[3] = 0;
}

__device__ void ctrl_after_apply(DevState* st, uint32_t act) {
  fold_stripes(st, st->acc_ap, 2);
  ctrl_after_apply_counted(st, act);
}

// The same two transitions for the C-loop rounds of a thread-block cluster
// (k_csmall), made by its one bookkeeping thread, which is the only writer of
// the field's state during the launch and keeps the type counts and the round
// number in registers: nothing is read from the state on the round's path.
// In the C-loop the apply and R-check accumulators (acc_ap, acc_r) are zero,
// so the apply's sums go straight into the counters; the increments are
// atomics whose result is not used.
//
// After the apply of C-loop round r (its type's case count `cases`, before
// the apply; max_rounds: st->max_rounds): what
// ctrl_after_apply_counted(st, ACT_MARK_C) does.
__device__ void ctrl_after_apply_small(DevState* st, uint32_t type, uint32_t dec, uint32_t frz, uint64_t cases,
                                       uint32_t ntouch, uint64_t r, uint64_t max_rounds) {
  atomicAdd((unsigned long long*)&st->cnt.dec_edits, (unsigned long long)dec);
  atomicAdd((unsigned long long*)&st->cnt.freezes, (unsigned long long)frz);
  atomicAdd((unsigned long long*)&st->cnt.c_rounds[type], 1ull);
  atomicAdd((unsigned long long*)&st->cnt.c_cases[type], (unsigned long long)cases);
  atomicAdd((unsigned long long*)&st->ticks, 1ull);
  st->ntouch = ntouch;
  st->rounds = r;
  st->action = ACT_RECLASS;
  if (r > max_rounds) {
    st->phase = PH_ERR;
    st->status = MSZ_ERR_NOCONVERGE;
    st->action = ACT_NONE;
  }
}

// After the reclassification that follows: the type counts c are stored;
// when the type still has cases, at most cap of them, all len of them in the
// case list, the state lists the next round (what ctrl_after_classify_counted
// and the listing of the cases leave) and it returns true; otherwise the
// general transition runs and it returns false.
__device__ bool ctrl_after_classify_small(DevState* st, uint32_t type, const uint32_t (&c)[4], uint32_t len,
                                          uint32_t cap, bool timeout) {
  for (int t = 0; t < 4; ++t) st->counts[t] = c[t];
  if (!timeout && c[type] != 0 && c[type] <= cap && len == c[type]) {
    st->ntouch = 0;
    st->ncase = len;
    st->action = ACT_REQUEST;
    atomicAdd((unsigned long long*)&st->cnt.sweeps, 1ull);
    atomicAdd((unsigned long long*)&st->ticks, 1ull);
    return true;
  }
  ctrl_after_classify_counted(st);
  return false;
}

// ---------------------------------------------------------------------------
// Edit requests (Sec. 5.1 deterministic mode): idempotent flags collected
// from one snapshot of g, applied afterwards; a freeze overrides a decrease.
// ---------------------------------------------------------------------------
// Slot in a list whose length counter is *ctr: one atomic per group of
// lanes that arrive together with the same counter (lanes that arrive
// together with different counters form one group per counter).
__device__ __forceinline__ uint32_t list_slot(uint32_t* ctr) {
  const uint32_t active = __activemask();
  const uint32_t peers = __match_any_sync(active, (unsigned long long)(uintptr_t)ctr);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(ctr, (uint32_t)__popc(peers));
  base = __shfl_sync(active, base, leader);
  return base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
}

// Where a vertex's first flag of the round adds it to the touched list:
// by default a slot from st->ntouch; with n alone, slot *n (a block or
// cluster that owns the whole list counts it itself); with buf, the block's
// staging buffer (buf[*n], flushed to the list later; a full buffer sends the
// vertex straight to the list).
struct TouchSink {
  uint32_t* n = nullptr;
  uint32_t* buf = nullptr;
  uint32_t cap = 0;
};

// Flags vertex u; its first flag of the round puts it on the touched list.
template <class T>
__device__ __forceinline__ void mark(const Field<T>& F, int u, uint8_t bit, const TouchSink& ts = TouchSink()) {
  uint32_t* w = reinterpret_cast<uint32_t*>(F.flags) + (u >> 2);
  const int sh = (u & 3) * 8;
  const uint32_t old = atomicOr(w, (uint32_t)bit << sh);
  if (((old >> sh) & (FL_DEC | FL_FREEZE)) != 0) return;
  if (ts.buf) {
    const uint32_t q = atomicAdd(ts.n, 1u);
    if (q < ts.cap) {
      ts.buf[q] = (uint32_t)u;
      return;
    }
  } else if (ts.n) {
    const uint32_t q = atomicAdd(ts.n, 1u);
    if (MSZ_IN(F.st, q, F.G.n)) F.touched[q] = (uint32_t)u;
    return;
  }
  const uint32_t q = list_slot(&F.st->ntouch);
  if (MSZ_IN(F.st, q, F.G.n)) F.touched[q] = (uint32_t)u;
}

// What a request for target t does: RQ_DEC decreases t; otherwise its
// anchor's ring freezes because t is frozen (RQ_FROZEN) or at its lower
// bound (RQ_BOUND).
enum : int { RQ_DEC = 0, RQ_FROZEN = 1, RQ_BOUND = 2 };
template <class T>
__device__ __forceinline__ int request_cause(const Field<T>& F, int t) {
  // the three loads issued together (one round trip, not two)
  const uint8_t fl = F.flags[t];
  const T gt = F.g[t], ft = F.f[t];
  if (fl & FL_FROZEN) return RQ_FROZEN;
  return gt > lower_bound_of(ft, F.xi) ? RQ_DEC : RQ_BOUND;
}
template <class T>
__device__ __forceinline__ bool request_decreases(const Field<T>& F, int t) {
  return request_cause(F, t) == RQ_DEC;
}

// Counts a freezing request of case kind k (0-3 the C-loop types, 4 / 5 a
// troublemaker of a wrong max / min label) with its cause.
__device__ __forceinline__ void count_freeze_req(DevState* st, int k, int cause) {
  atomicAdd((unsigned long long*)&st->cnt.freeze_req[k], 1ull);
  if (cause == RQ_FROZEN) atomicAdd((unsigned long long*)&st->cnt.freeze_req_frozen[k], 1ull);
}

// A false case anchored at a asks for a decreasing edit of t. If t is frozen
// or already at its lower bound, the non-frozen part of a's closed 1-ring is
// frozen instead (termination guard; the paper argues convergence in the
// reals, Sec. 4.3).
template <class T, int ND>
__device__ void request(const Field<T>& F, int a, int t, const TouchSink& ts = TouchSink()) {
  if (request_decreases(F, t)) {
    mark(F, t, FL_DEC, ts);
    return;
  }
  int x, y, z;
  coords(F.G, a, x, y, z);
  if (!(F.flags[a] & FL_FROZEN)) mark(F, a, FL_FREEZE, ts);
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
      if (!(F.flags[u] & FL_FROZEN)) mark(F, u, FL_FREEZE, ts);
    }
  }
}

// The freeze of anchor a's closed 1-ring by a whole warp, one lane per
// vertex (lane = the thread's lane); touched list as in mark().
template <class T, int ND>
__device__ __forceinline__ void freeze_ring_warp(const Field<T>& F, int a, int lane,
                                                 const TouchSink& ts = TouchSink()) {
  constexpr int NPOS = Slots<ND>::NPOS;
  if (lane > 2 * NPOS) return;
  int u = a;
  if (lane < 2 * NPOS) {
    int x, y, z;
    coords(F.G, a, x, y, z);
    const int sg = (lane < NPOS) ? 1 : -1;
    const int m = (int)((Slots<ND>::MASKS >> (4 * (lane < NPOS ? lane : lane - NPOS))) & 7u);
    const int dx = sg * (m & 1), dy = sg * ((m >> 1) & 1), dz = sg * ((m >> 2) & 1);
    const int X = x + dx, Y = y + dy, Z = z + dz;
    bool in = X >= 0 && X < F.G.nx && Y >= 0 && Y < F.G.ny;
    if (ND == 3) in = in && Z >= 0 && Z < F.G.nz;
    if (!in) return;
    u = a + dx + dy * F.G.nx + dz * F.G.nxny;
  }
  if (!(F.flags[u] & FL_FROZEN)) mark(F, u, FL_FREEZE, ts);
}

}  // namespace msz
