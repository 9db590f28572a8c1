// MSz correction loop: CPU oracle.
//
// TEST INFRASTRUCTURE ONLY. This file is the plain, slow, single-threaded
// restatement of the MSz method (Li et al., "MSz: An Efficient Parallel
// Algorithm for Correcting Morse-Smale Segmentations in Error-Bounded Lossy
// Compressors", Sec. 3-4) against which the CUDA path is checked. Only the
// test suite, the smoke check and the CPU-baseline leg of the benchmark may
// load it. It shares no code, header or table with the CUDA library.
//
// Every step follows the paper's definitions directly:
//   * PL scalar field on a triangulated grid, SoS tie-break (Sec. 3)
//   * steepest ascending / descending neighbour, extrema, labels (Sec. 3)
//   * false critical points, Definitions 1-3 (Sec. 4.1)
//   * decreasing edits, Eqs. (2)-(5) (Sec. 4.1) and Eq. (6) (Sec. 4.2)
//   * C-loop / R-loop alternation (Sec. 4.1-4.3)
// Where the paper is silent the reading used is stated next to the code:
// Freudenthal (Kuhn) triangulation, ties broken by linear vertex index,
// the floating-point lower bound, the freeze guard and the loop order.
//
// Build: g++ -std=c++17 -O2 -ffp-contract=off -fPIC -shared (no fast-math:
// every floating-point operation is one IEEE round-to-nearest operation).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Grid and triangulation (Sec. 3: a mesh of triangles or tetrahedra).
// Reading: the Freudenthal/Kuhn triangulation of the regular grid. Vertex v
// at (x, y, z) has linear index x + nx*(y + ny*z). Its neighbours are v + e
// for every nonzero e in {0,1}^d and every -e, when inside the grid
// (6 neighbours in 2D, 14 in 3D; no padding, no periodicity).
// ---------------------------------------------------------------------------
struct Grid {
  int ndim;
  int64_t nx, ny, nz, n;
};

// Writes the in-grid neighbours of v to out[]; returns how many there are.
int neighbours(const Grid& G, int64_t v, int64_t out[14]) {
  const int64_t x = v % G.nx;
  const int64_t y = (v / G.nx) % G.ny;
  const int64_t z = v / (G.nx * G.ny);
  int k = 0;
  const int dmax = (G.ndim == 3) ? 1 : 0;
  for (int ez = 0; ez <= dmax; ++ez)
    for (int ey = 0; ey <= 1; ++ey)
      for (int ex = 0; ex <= 1; ++ex) {
        if (ex == 0 && ey == 0 && ez == 0) continue;
        for (int sgn = -1; sgn <= 1; sgn += 2) {
          const int64_t X = x + sgn * ex, Y = y + sgn * ey, Z = z + sgn * ez;
          if (X < 0 || X >= G.nx || Y < 0 || Y >= G.ny || Z < 0 || Z >= G.nz) continue;
          out[k++] = X + G.nx * (Y + G.ny * Z);
        }
      }
  return k;
}

// ---------------------------------------------------------------------------
// Order on vertices (Sec. 3, Problem Statement: distinct values assumed,
// otherwise simulation of simplicity). Reading: u precedes v iff
// g_u < g_v, or g_u == g_v and u < v (IEEE comparison, so -0 == +0).
// ---------------------------------------------------------------------------
template <class T>
bool precedes(const T* g, int64_t u, int64_t v) {
  return g[u] < g[v] || (g[u] == g[v] && u < v);
}

// Steepest ascending / descending neighbour (Sec. 3, "Integral lines": the
// line extends to the highest / lowest adjacent vertex). up[v] is the
// greatest vertex of v's closed 1-ring under the order, dn[v] the least; v is
// a maximum iff up[v] == v and a minimum iff dn[v] == v (Sec. 3, "Critical
// points").
template <class T>
void directions(const Grid& G, const T* g, int64_t* up, int64_t* dn) {
  int64_t nb[14];
  for (int64_t v = 0; v < G.n; ++v) {
    const int k = neighbours(G, v, nb);
    int64_t hi = v, lo = v;
    for (int j = 0; j < k; ++j) {
      if (precedes(g, hi, nb[j])) hi = nb[j];
      if (precedes(g, nb[j], lo)) lo = nb[j];
    }
    up[v] = hi;
    dn[v] = lo;
  }
}

// Maximum / minimum labels (Sec. 3, "Ascending/descending segmentations"):
// the extremum reached by following dir[] from v. Plain walk with
// memoisation of vertices already resolved.
void labels(const Grid& G, const int64_t* dir, int32_t* lab) {
  for (int64_t v = 0; v < G.n; ++v) lab[v] = -1;
  std::vector<int64_t> path;
  for (int64_t v = 0; v < G.n; ++v) {
    if (lab[v] >= 0) continue;
    path.clear();
    int64_t w = v;
    while (lab[w] < 0 && dir[w] != w) {
      path.push_back(w);
      w = dir[w];
    }
    const int32_t root = (lab[w] >= 0) ? lab[w] : (int32_t)w;
    lab[w] = root;
    for (int64_t u : path) lab[u] = root;
  }
}

// ---------------------------------------------------------------------------
// Error-bound arithmetic (Sec. 3 constraint |f_i - g_i| <= xi; Eq. (1)).
// The paper works in the reals. Reading for floating point:
//   lb_i = the smallest representable value >= f_i - xi,
//   ub_i = the largest representable value  <= f_i + xi,
// found from the rounded difference and its exact TwoSum error.
// ---------------------------------------------------------------------------
template <class T>
T two_sum_err(T a, T b, T s) {  // exact a + b - s, for s = RN(a + b)
  const T bp = s - a;
  const T ap = s - bp;
  return (a - ap) + (b - bp);
}

template <class T>
T lower_bound_of(T f, T xi) {
  T s = f - xi;
  if (!std::isfinite(s)) return s;
  const T e = two_sum_err<T>(f, -xi, s);
  if (e > 0) s = std::nextafter(s, (T)INFINITY);
  return s;
}

template <class T>
T upper_bound_of(T f, T xi) {
  T s = f + xi;
  if (!std::isfinite(s)) return s;
  const T e = two_sum_err<T>(f, xi, s);
  if (e < 0) s = std::nextafter(s, -(T)INFINITY);
  return s;
}

// One decreasing edit, Eqs. (2)-(6): g <- (g + f - xi) / 2 with f - xi read
// as lb. Evaluated as RN(RN(0.5*g) + RN(0.5*lb)) (the halvings are exact
// outside the subnormal range). If rounding gives no strict decrease the
// value snaps to lb, so every edit strictly decreases g and keeps g >= lb.
template <class T>
T decrease(T g, T lb) {
  const T h = (T)0.5;
  T m = h * g + h * lb;
  if (!(m < g) || m < lb) m = lb;
  return m;
}

// ---------------------------------------------------------------------------
// False critical points (Definitions 1-3), as set differences of the
// extremum sets of g and f under the order above.
// ---------------------------------------------------------------------------
enum { FPMAX = 0, FPMIN = 1, FNMAX = 2, FNMIN = 3 };

inline unsigned false_bits(int64_t v, const int64_t* up_g, const int64_t* dn_g,
                           const int64_t* up_f, const int64_t* dn_f) {
  const bool gmax = up_g[v] == v, gmin = dn_g[v] == v;
  const bool fmax = up_f[v] == v, fmin = dn_f[v] == v;
  unsigned b = 0;
  if (gmax && !fmax) b |= 1u << FPMAX;  // Def. 1
  if (gmin && !fmin) b |= 1u << FPMIN;  // Def. 2
  if (fmax && !gmax) b |= 1u << FNMAX;  // Def. 3 (maximum)
  if (fmin && !gmin) b |= 1u << FNMIN;  // Def. 3 (minimum)
  return b;
}

// Troublemaker test for vertex t (Sec. 4.2). Bit 0: wrong maximum label and
// a steepest ascent in g that differs from f's; bit 1: wrong minimum label
// and a steepest descent in g that differs from f's.
inline unsigned trouble_bits(int64_t t, const int32_t* Mg, const int32_t* mg, const int32_t* M,
                             const int32_t* m, const int64_t* up_g, const int64_t* dn_g,
                             const int64_t* up_f, const int64_t* dn_f) {
  unsigned b = 0;
  if (Mg[t] != M[t] && up_g[t] != up_f[t]) b |= 1u;
  if (mg[t] != m[t] && dn_g[t] != dn_f[t]) b |= 2u;
  return b;
}

// Counters reported with every fix (identical layout on the CUDA side).
struct Counts {
  uint64_t sweeps;         // direction evaluations of a changed field
  uint64_t c_rounds[4];    // C-loop edit rounds per false type
  uint64_t c_cases[4];     // false cases edited, summed over those rounds
  uint64_t c_passes;       // completed passes over the four sub-loops
  uint64_t r_rounds;       // R-loop edit rounds
  uint64_t r_cases[2];     // troublemakers edited (ascending, descending)
  uint64_t label_evals;    // label computations of g
  uint64_t mismatch[2];    // wrong max / min labels, summed over label evals
  uint64_t dec_edits;      // decreasing edits applied
  uint64_t freezes;        // vertices frozen by the termination guard
  uint64_t edits;          // length of the final edit list
  // Requests that froze their anchor's ring instead of decreasing their
  // target, by the case that made them: C-loop FPmax, FPmin, FNmax, FNmin,
  // R-loop wrong max label, wrong min label. freeze_req counts them all,
  // freeze_req_frozen those whose target was already frozen (the others
  // found the target at its lower bound).
  uint64_t freeze_req[6];
  uint64_t freeze_req_frozen[6];
};

enum { ST_OK = 0, ST_ARG = -1, ST_DTYPE = -2, ST_NONFINITE = -3, ST_BOUND = -4,
       ST_NOCONVERGE = -6 };

// Trace of edit rounds: (phase 0=C / 1=R, type or 0, cases, dec, freeze).
struct Trace {
  int64_t* buf;
  int64_t cap;
  int64_t len;
  void push(int64_t a, int64_t b, int64_t c, int64_t d, int64_t e) {
    if (buf && len < cap) {
      int64_t* r = buf + 5 * len;
      r[0] = a; r[1] = b; r[2] = c; r[3] = d; r[4] = e;
    }
    ++len;
  }
};

// ---------------------------------------------------------------------------
// The correction loop (Sec. 4, Fig. 3 workflow).
// ---------------------------------------------------------------------------
template <class T>
struct Fixer {
  Grid G;
  const T* f;
  T* g;
  T xi;
  std::vector<T> lb;
  std::vector<int64_t> up_f, dn_f, up_g, dn_g;
  std::vector<int32_t> M, m, Mg, mg;
  std::vector<uint8_t> frozen, mark;
  Counts cnt;
  Trace tr;
  uint64_t version = 0, swept = ~0ull;
  uint64_t max_rounds;

  enum { DEC = 1, FREEZE = 2 };

  void ensure_directions() {
    if (swept == version) return;
    directions(G, g, up_g.data(), dn_g.data());
    swept = version;
    ++cnt.sweeps;
  }

  // A false case at anchor a asks for a decreasing edit of target t.
  // Termination guard (reading; the paper argues convergence in the reals,
  // Sec. 4.3): if t is frozen or already at its lower bound, every non-frozen
  // vertex of a's closed 1-ring is frozen instead, i.e. reset to f and never
  // edited again. kind: the case that asks (0-3 the C-loop types, 4 / 5 a
  // troublemaker of a wrong max / min label), for the freeze counters.
  void request(int64_t a, int64_t t, int kind) {
    if (!frozen[t] && g[t] > lb[t]) {
      mark[t] |= DEC;
      return;
    }
    ++cnt.freeze_req[kind];
    if (frozen[t]) ++cnt.freeze_req_frozen[kind];
    int64_t nb[14];
    const int k = neighbours(G, a, nb);
    if (!frozen[a]) mark[a] |= FREEZE;
    for (int j = 0; j < k; ++j)
      if (!frozen[nb[j]]) mark[nb[j]] |= FREEZE;
  }

  // All requests of a round see the same snapshot of g; they are applied
  // together afterwards (iteration-synchronous; a freeze overrides a
  // decrease of the same vertex).
  void apply(int64_t* ndec, int64_t* nfrz) {
    *ndec = *nfrz = 0;
    for (int64_t u = 0; u < G.n; ++u) {
      if (mark[u] & FREEZE) {
        g[u] = f[u];
        frozen[u] = 1;
        ++*nfrz;
      } else if (mark[u] & DEC) {
        g[u] = decrease(g[u], lb[u]);
        ++*ndec;
      }
      mark[u] = 0;
    }
    cnt.dec_edits += *ndec;
    cnt.freezes += *nfrz;
    ++version;
  }

  // One C-loop sub-iteration of type T over the current snapshot.
  // Targets: FPmax -> i itself (Eq. 2); FPmin -> the neighbour of i that is
  // maximal in g (Eq. 3); FNmax -> the neighbour of i that is maximal in g
  // (Eq. 4); FNmin -> i itself (Eq. 5). For FPmin and FNmax that neighbour
  // is up_g[i], since i is not the greatest vertex of its ring in g.
  int64_t c_round(int type, int64_t* ncase) {
    int64_t k = 0;
    for (int64_t i = 0; i < G.n; ++i) {
      if (!(false_bits(i, up_g.data(), dn_g.data(), up_f.data(), dn_f.data()) >> type & 1u))
        continue;
      ++k;
      const int64_t t = (type == FPMAX || type == FNMIN) ? i : up_g[i];
      request(i, t, type);
    }
    *ncase = k;
    return k;
  }

  int run() {
    const int64_t n = G.n;
    // Directions and labels of the original field (fixed for the whole run).
    directions(G, f, up_f.data(), dn_f.data());
    labels(G, up_f.data(), M.data());
    labels(G, dn_f.data(), m.data());

    uint64_t rounds = 0;
    for (;;) {
      // ---- C-loop (Sec. 4.1): FPmax, FPmin, FNmax, FNmin sub-loops, each
      // repeated until its type is absent; passes repeat until no false
      // critical point of any type is left.
      int type = FPMAX;
      for (;;) {
        ensure_directions();
        int64_t nc = 0;
        if (c_round(type, &nc) > 0) {
          int64_t nd, nf;
          apply(&nd, &nf);
          ++cnt.c_rounds[type];
          cnt.c_cases[type] += (uint64_t)nc;
          tr.push(0, type, nc, nd, nf);
          if (++rounds > max_rounds) return ST_NOCONVERGE;
          continue;
        }
        if (type < FNMIN) { ++type; continue; }
        ++cnt.c_passes;
        bool any = false;
        for (int64_t i = 0; i < n && !any; ++i)
          any = false_bits(i, up_g.data(), dn_g.data(), up_f.data(), dn_f.data()) != 0;
        if (!any) break;
        type = FPMAX;
      }

      // ---- R-loop (Sec. 4.2): labels of g, compare with the original's.
      ensure_directions();
      labels(G, up_g.data(), Mg.data());
      labels(G, dn_g.data(), mg.data());
      ++cnt.label_evals;
      int64_t wrong_max = 0, wrong_min = 0;
      for (int64_t v = 0; v < n; ++v) {
        wrong_max += Mg[v] != M[v];
        wrong_min += mg[v] != m[v];
      }
      cnt.mismatch[0] += (uint64_t)wrong_max;
      cnt.mismatch[1] += (uint64_t)wrong_min;
      if (wrong_max == 0 && wrong_min == 0) return ST_OK;

      // Troublemaker (reading of the first place along an integral line
      // where g and f disagree): a wrongly labelled vertex t whose steepest
      // neighbour in g differs from the one in f. Wrong maximum label: the
      // ascending neighbour in g, up_g[t], is decreased (Eq. 6). Wrong
      // minimum label: the descending neighbour of f, dn_f[t], is decreased
      // so that it becomes t's steepest descent in g.
      int64_t ta = 0, td = 0;
      for (int64_t t = 0; t < n; ++t) {
        const unsigned tb = trouble_bits(t, Mg.data(), mg.data(), M.data(), m.data(),
                                         up_g.data(), dn_g.data(), up_f.data(), dn_f.data());
        if (tb & 1u) { ++ta; request(t, up_g[t], 4); }
        if (tb & 2u) { ++td; request(t, dn_f[t], 5); }
      }
      if (ta + td == 0) return ST_NOCONVERGE;  // cannot happen once extrema agree
      int64_t nd, nf;
      apply(&nd, &nf);
      ++cnt.r_rounds;
      cnt.r_cases[0] += (uint64_t)ta;
      cnt.r_cases[1] += (uint64_t)td;
      tr.push(1, 0, ta + td, nd, nf);
      if (++rounds > max_rounds) return ST_NOCONVERGE;
    }
  }
};

Grid make_grid(int ndim, const int64_t* dims) {
  Grid G;
  G.ndim = ndim;
  G.nx = dims[0];
  G.ny = dims[1];
  G.nz = (ndim == 3) ? dims[2] : 1;
  G.n = G.nx * G.ny * G.nz;
  return G;
}

bool grid_ok(int ndim, const int64_t* dims) {
  if (ndim != 2 && ndim != 3) return false;
  for (int d = 0; d < ndim; ++d)
    if (dims[d] < 1) return false;
  const Grid G = make_grid(ndim, dims);
  return G.n <= 0x7fffffffLL;
}

template <class T>
int fix_impl(int ndim, const int64_t* dims, const T* f, const T* fhat, double xi_in,
             uint64_t max_rounds, T* g_out, int32_t* M_out, int32_t* m_out,
             uint64_t* counts_out, int64_t* trace, int64_t trace_cap, int64_t* trace_len) {
  if (!grid_ok(ndim, dims)) return ST_ARG;
  const T xi = (T)xi_in;  // xi_eff: the bound rounded once to the field's type
  if (!(xi >= 0) || !std::isfinite(xi)) return ST_ARG;
  Fixer<T> F;
  F.G = make_grid(ndim, dims);
  const int64_t n = F.G.n;
  F.f = f;
  F.g = g_out;
  F.xi = xi;
  F.max_rounds = max_rounds;
  std::memset(&F.cnt, 0, sizeof(F.cnt));
  F.tr.buf = trace;
  F.tr.cap = trace_cap;
  F.tr.len = 0;
  // Validation of the inputs against the constraint |f - fhat| <= xi.
  for (int64_t v = 0; v < n; ++v)
    if (!std::isfinite(f[v]) || !std::isfinite(fhat[v])) return ST_NONFINITE;
  F.lb.resize(n);
  for (int64_t v = 0; v < n; ++v) {
    F.lb[v] = lower_bound_of(f[v], xi);
    if (!std::isfinite(F.lb[v])) return ST_ARG;  // f - xi overflows
  }
  for (int64_t v = 0; v < n; ++v)
    if (fhat[v] < F.lb[v] || fhat[v] > upper_bound_of(f[v], xi)) return ST_BOUND;
  for (int64_t v = 0; v < n; ++v) g_out[v] = fhat[v];  // g^(0) = fhat, Eq. (1)
  F.up_f.resize(n); F.dn_f.resize(n); F.up_g.resize(n); F.dn_g.resize(n);
  F.M.resize(n); F.m.resize(n); F.Mg.resize(n); F.mg.resize(n);
  F.frozen.assign(n, 0);
  F.mark.assign(n, 0);
  const int st = F.run();
  // Edits are the vertices whose final value differs bitwise from fhat.
  uint64_t e = 0;
  for (int64_t v = 0; v < n; ++v) e += std::memcmp(&g_out[v], &fhat[v], sizeof(T)) != 0;
  F.cnt.edits = e;
  if (M_out) std::memcpy(M_out, F.Mg.data(), n * sizeof(int32_t));
  if (m_out) std::memcpy(m_out, F.mg.data(), n * sizeof(int32_t));
  if (counts_out) std::memcpy(counts_out, &F.cnt, sizeof(Counts));
  if (trace_len) *trace_len = F.tr.len;
  return st;
}

}  // namespace

// ---------------------------------------------------------------------------
// C entry points (loaded by the tests with ctypes). dtype: 0 = float32,
// 1 = float64. All arrays are host memory, x fastest.
// ---------------------------------------------------------------------------
extern "C" {

int oracle_counts_words() { return (int)(sizeof(Counts) / sizeof(uint64_t)); }

int oracle_neighbours(int ndim, const int64_t* dims, int64_t v, int64_t* out) {
  if (!grid_ok(ndim, dims)) return -1;
  return neighbours(make_grid(ndim, dims), v, out);
}

int oracle_directions(int ndim, const int64_t* dims, int dtype, const void* g,
                      int64_t* up, int64_t* dn) {
  if (!grid_ok(ndim, dims)) return ST_ARG;
  const Grid G = make_grid(ndim, dims);
  if (dtype == 0) directions(G, (const float*)g, up, dn);
  else if (dtype == 1) directions(G, (const double*)g, up, dn);
  else return ST_DTYPE;
  return ST_OK;
}

int oracle_labels(int ndim, const int64_t* dims, const int64_t* dir, int32_t* lab) {
  if (!grid_ok(ndim, dims)) return ST_ARG;
  labels(make_grid(ndim, dims), dir, lab);
  return ST_OK;
}

int oracle_false_bits(int ndim, const int64_t* dims, int dtype, const void* f,
                      const void* g, uint8_t* bits) {
  if (!grid_ok(ndim, dims)) return ST_ARG;
  const Grid G = make_grid(ndim, dims);
  std::vector<int64_t> uf(G.n), df(G.n), ug(G.n), dg(G.n);
  int r = oracle_directions(ndim, dims, dtype, f, uf.data(), df.data());
  if (r) return r;
  oracle_directions(ndim, dims, dtype, g, ug.data(), dg.data());
  for (int64_t v = 0; v < G.n; ++v)
    bits[v] = (uint8_t)false_bits(v, ug.data(), dg.data(), uf.data(), df.data());
  return ST_OK;
}

int oracle_troublemakers(int ndim, const int64_t* dims, int dtype, const void* f,
                         const void* g, uint8_t* bits) {
  if (!grid_ok(ndim, dims)) return ST_ARG;
  const Grid G = make_grid(ndim, dims);
  std::vector<int64_t> uf(G.n), df(G.n), ug(G.n), dg(G.n);
  int r = oracle_directions(ndim, dims, dtype, f, uf.data(), df.data());
  if (r) return r;
  oracle_directions(ndim, dims, dtype, g, ug.data(), dg.data());
  std::vector<int32_t> M(G.n), m(G.n), Mg(G.n), mg(G.n);
  labels(G, uf.data(), M.data());
  labels(G, df.data(), m.data());
  labels(G, ug.data(), Mg.data());
  labels(G, dg.data(), mg.data());
  for (int64_t t = 0; t < G.n; ++t)
    bits[t] = (uint8_t)trouble_bits(t, Mg.data(), mg.data(), M.data(), m.data(), ug.data(),
                                    dg.data(), uf.data(), df.data());
  return ST_OK;
}

int oracle_bounds(int dtype, int64_t n, const void* f, double xi, void* lb, void* ub) {
  if (dtype == 0) {
    const float x = (float)xi;
    for (int64_t i = 0; i < n; ++i) {
      ((float*)lb)[i] = lower_bound_of(((const float*)f)[i], x);
      ((float*)ub)[i] = upper_bound_of(((const float*)f)[i], x);
    }
  } else if (dtype == 1) {
    for (int64_t i = 0; i < n; ++i) {
      ((double*)lb)[i] = lower_bound_of(((const double*)f)[i], xi);
      ((double*)ub)[i] = upper_bound_of(((const double*)f)[i], xi);
    }
  } else {
    return ST_DTYPE;
  }
  return ST_OK;
}

int oracle_decrease(int dtype, int64_t n, const void* g, const void* lb, void* out) {
  if (dtype == 0) {
    for (int64_t i = 0; i < n; ++i)
      ((float*)out)[i] = decrease(((const float*)g)[i], ((const float*)lb)[i]);
  } else if (dtype == 1) {
    for (int64_t i = 0; i < n; ++i)
      ((double*)out)[i] = decrease(((const double*)g)[i], ((const double*)lb)[i]);
  } else {
    return ST_DTYPE;
  }
  return ST_OK;
}

int oracle_fix(int ndim, const int64_t* dims, int dtype, const void* f, const void* fhat,
               double xi, uint64_t max_rounds, void* g_out, int32_t* M_out, int32_t* m_out,
               uint64_t* counts_out, int64_t* trace, int64_t trace_cap, int64_t* trace_len) {
  if (dtype == 0)
    return fix_impl(ndim, dims, (const float*)f, (const float*)fhat, xi, max_rounds,
                    (float*)g_out, M_out, m_out, counts_out, trace, trace_cap, trace_len);
  if (dtype == 1)
    return fix_impl(ndim, dims, (const double*)f, (const double*)fhat, xi, max_rounds,
                    (double*)g_out, M_out, m_out, counts_out, trace, trace_cap, trace_len);
  return ST_DTYPE;
}

}  // extern "C"
