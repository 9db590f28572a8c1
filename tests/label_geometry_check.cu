// Host-side check of the label-tile index maps (compiled for the host only
// by tests/test_label_geometry.py): the halo shell's and the face cells'
// index maps are bijections onto exactly the cells they name, and the
// exit-table slots are distinct per face vertex, below the slot count, and
// defined for every cell an integral line can leave a tile through (a shell
// cell inside the grid lies on a face of its own tile), where the per-field
// relative slot table gives the same slot.
#include <cstdio>
#include <set>
#include <vector>

#include "msz_kernels.cuh"

using namespace msz;

template <int ND>
int check_shell() {
  using LG = LabelGeom<ND>;
  std::set<int> seen;
  int bad = 0;
  for (int s = 0; s < LG::SHELL; ++s) {
    int hx, hy, hz;
    shell_cell<ND>(s, hx, hy, hz);
    const bool on = hx == 0 || hx == LG::SX - 1 || hy == 0 || hy == LG::SY - 1 || (ND == 3 && (hz == 0 || hz == LG::SZ - 1));
    if (!on || hx < 0 || hx >= LG::SX || hy < 0 || hy >= LG::SY || hz < 0 || hz >= LG::SZ) ++bad;
    if (shell_index<ND>(hx, hy, hz) != s) ++bad;
    seen.insert(hx + LG::SX * (hy + LG::SY * hz));
  }
  if ((int)seen.size() != LG::SHELL) ++bad;
  return bad;
}

template <int ND>
int check_faces() {
  using LG = LabelGeom<ND>;
  std::set<int> seen;
  int bad = 0;
  for (int f = 0; f < LG::NFACE; ++f) {
    int lx, ly, lz;
    face_cell<ND>(f, lx, ly, lz);
    const bool on = lx == 0 || lx == LG::TX - 1 || ly == 0 || ly == LG::TY - 1 || (ND == 3 && (lz == 0 || lz == LG::TZ - 1));
    if (!on || lx < 0 || lx >= LG::TX || ly < 0 || ly >= LG::TY || lz < 0 || lz >= LG::TZ) ++bad;
    if (face_index<ND>(lx, ly, lz) != f) ++bad;
    seen.insert(lx + LG::TX * (ly + LG::TY * lz));
  }
  int faces = 0;
  for (int lz = 0; lz < LG::TZ; ++lz)
    for (int ly = 0; ly < LG::TY; ++ly)
      for (int lx = 0; lx < LG::TX; ++lx) {
        const bool on = lx == 0 || lx == LG::TX - 1 || ly == 0 || ly == LG::TY - 1 || (ND == 3 && (lz == 0 || lz == LG::TZ - 1));
        faces += on;
      }
  if ((int)seen.size() != LG::NFACE || faces != LG::NFACE) ++bad;
  return bad;
}

// Every in-grid face vertex gets its own slot below the slot count, and
// every in-grid shell cell of every tile is such a vertex.
template <int ND>
int check_slots(int nx, int ny, int nz) {
  using LG = LabelGeom<ND>;
  Geom G{};
  G.nx = nx;
  G.ny = ny;
  G.nz = nz;
  G.nxny = nx * ny;
  G.n = nx * ny * nz;
  G.nd = ND;
  const int tx = (nx + LG::TX - 1) / LG::TX, ty = (ny + LG::TY - 1) / LG::TY, tz = (nz + LG::TZ - 1) / LG::TZ;
  const uint32_t nslots = (uint32_t)(tx * ty * tz) * LG::NFACE;
  std::vector<int> owner(nslots, -1);
  int bad = 0;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int lx = x % LG::TX, ly = y % LG::TY, lz = z % LG::TZ;
        const bool on = lx == 0 || lx == LG::TX - 1 || ly == 0 || ly == LG::TY - 1 || (ND == 3 && (lz == 0 || lz == LG::TZ - 1));
        if (!on) continue;
        const uint32_t s = exit_slot<ND>(G, x, y, z);
        if (s >= nslots || owner[s] != -1) {
          ++bad;
          continue;
        }
        owner[s] = x + nx * (y + ny * z);
      }
  for (int t = 0; t < tx * ty * tz; ++t) {
    const int x0 = (t % tx) * LG::TX, y0 = ((t / tx) % ty) * LG::TY, z0 = (t / (tx * ty)) * LG::TZ;
    for (int s = 0; s < LG::SHELL; ++s) {
      int hx, hy, hz;
      shell_cell<ND>(s, hx, hy, hz);
      const int x = x0 - 1 + hx, y = y0 - 1 + hy, z = (ND == 3) ? z0 - 1 + hz : 0;
      if (x < 0 || y < 0 || z < 0 || x >= nx || y >= ny || z >= nz) continue;
      const uint32_t sl = exit_slot<ND>(G, x, y, z);
      if (sl >= nslots || owner[sl] != x + nx * (y + ny * z)) ++bad;
      if ((long long)t * LG::NFACE + shell_slot_delta<ND>(s, tx, ty) != (long long)sl) ++bad;
    }
  }
  return bad;
}

int main() {
  int bad = 0;
  bad += check_shell<2>() + check_shell<3>();
  bad += check_faces<2>() + check_faces<3>();
  bad += check_slots<3>(16, 16, 16) + check_slots<3>(37, 20, 33) + check_slots<3>(48, 17, 5);
  bad += check_slots<2>(64, 32, 1) + check_slots<2>(150, 45, 1) + check_slots<2>(7, 300, 1);
  std::printf("label geometry: %d problems (shell %d/%d cells, faces %d/%d cells)\n", bad, LabelGeom<2>::SHELL,
              LabelGeom<3>::SHELL, LabelGeom<2>::NFACE, LabelGeom<3>::NFACE);
  return bad == 0 ? 0 : 1;
}
