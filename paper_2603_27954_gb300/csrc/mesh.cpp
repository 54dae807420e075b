// Block-structured refinement mesh (Sec. 2.2: octree leaves holding cubic
// blocks of cells) and the slot tables of the in-place (AA) update.
//
// Storage: every level keeps its blocks in one array f[block][27][B^3]
// (floats, x fastest inside a block).  Active blocks (those with cells this
// level updates) come first in Morton order, then ghost blocks, which only
// give storage to the populations that cross the level's edge: the domain
// faces, the cut links into solid cells, and the interface with the next
// finer or coarser level.
//
// AA pattern: an even step reads f_i(x) from slot (x, i) and writes the
// post-collision f*_i(x) to (x, ibar); an odd step reads f_i(x) from
// (x - c_i, ibar) and writes f*_i(x) to (x + c_i, i).  Consequently, after
// an even step f*_i(x) sits in (x, ibar) and the next step expects the
// incoming f_i(x) in (x - c_i, ibar); after an odd step f*_i(x) sits in
// (x + c_i, i) and the next step expects f_i(x) in (x, i).  Every table
// below is a list of (destination slot, source slots) pairs per parity.
#include <algorithm>
#include <atomic>
#include <functional>
#include <cmath>
#include <cstring>
#include <limits>
#include <unordered_map>

#include "internal.h"
#include "parallel.h"

namespace lbm {
namespace {

int floordiv(int a, int b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }
int wrapmod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1fffff;
  x = (x | x << 32) & 0x1f00000000ffffULL;
  x = (x | x << 16) & 0x1f0000ff0000ffULL;
  x = (x | x << 8) & 0x100f00f00f00f00fULL;
  x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
  x = (x | x << 2) & 0x1249249249249249ULL;
  return x;
}
uint64_t morton(int x, int y, int z) { return spread3(x) | spread3(y) << 1 | spread3(z) << 2; }

bool in_box(const int lo[3], const int hi[3], int x, int y, int z) {
  return x >= lo[0] && x < hi[0] && y >= lo[1] && y < hi[1] && z >= lo[2] && z < hi[2];
}

}  // namespace

int Level::locate(int x, int y, int z, int* local) const {
  int c[3] = {x, y, z};
  int b[3], r[3];
  for (int a = 0; a < 3; ++a) {
    if (wrap[a]) c[a] = wrapmod(c[a], dom[a]);
    int rel = c[a] - org[a];
    if (rel < 0) return -1;
    b[a] = rel / B;
    if (b[a] >= nb[a]) return -1;
    r[a] = rel - b[a] * B;
  }
  int s = slot[((size_t)b[2] * nb[1] + b[1]) * nb[0] + b[0]];
  if (s < 0) return -1;
  *local = (r[2] * B + r[1]) * B + r[0];
  return s;
}

CellType Level::cell_type(int x, int y, int z) const {
  int loc;
  int s = locate(x, y, z, &loc);
  if (s < 0) return OUTSIDE;
  return (CellType)type[(size_t)s * cells_per_block() + loc];
}

long long Level::addr(int x, int y, int z, int dir) const {
  int loc;
  int s = locate(x, y, z, &loc);
  if (s < 0) return -1;
  return ((long long)s * kQ + dir) * cells_per_block() + loc;
}

void refinement_boxes(const Tree& t, int levels, int block, double margin, int boxes[6][6]) {
  for (int l = 0; l < 6; ++l)
    for (int q = 0; q < 6; ++q) boxes[l][q] = 0;
  if (levels < 2) return;
  double lo[3], hi[3];
  tree_bounds(t, lo, hi);
  const int B = block;
  for (int a = 0; a < 3; ++a) {
    double ext = hi[a] - lo[a];
    double glo = lo[a] - margin * ext, ghi = hi[a] + margin * ext;
    // finest cells, rounded outward to whole finest blocks
    boxes[levels - 1][a] = (int)std::floor(glo / B) * B;
    boxes[levels - 1][3 + a] = (int)std::ceil(ghi / B) * B;
  }
  // each coarser box: the finer box's footprint rounded outward to whole
  // blocks of its own level, plus one block on every side
  for (int l = levels - 2; l >= 1; --l)
    for (int a = 0; a < 3; ++a) {
      boxes[l][a] = floordiv(boxes[l + 1][a], 2 * B) * B - B;
      boxes[l][3 + a] = -floordiv(-boxes[l + 1][3 + a], 2 * B) * B + B;
    }
}

namespace {

// cell of level l is updated by level l (inside its real region, not covered by l+1)
bool live(const Mesh& m, int l, int x, int y, int z) {
  const Level& v = m.lv[l];
  int c[3] = {x, y, z};
  for (int a = 0; a < 3; ++a)
    if (v.wrap[a]) c[a] = wrapmod(c[a], v.dom[a]);
  if (!v.in_real(c[0], c[1], c[2])) return false;
  if (l + 1 < m.L) {
    const Level& f = m.lv[l + 1];
    if (f.in_real(2 * c[0], 2 * c[1], 2 * c[2])) return false;
  }
  return true;
}

CellType base_type(const Mesh& m, int l, int x, int y, int z) {
  const Level& v = m.lv[l];
  if (!v.in_real(x, y, z)) return OUTSIDE;
  if (l + 1 < m.L && m.lv[l + 1].in_real(2 * x, 2 * y, 2 * z)) return COVERED;
  return FLUID;
}

void block_origin(const Level& v, int gi, int o[3]) {
  int bx = gi % v.nb[0], by = (gi / v.nb[0]) % v.nb[1], bz = gi / (v.nb[0] * v.nb[1]);
  o[0] = v.org[0] + bx * v.B;
  o[1] = v.org[1] + by * v.B;
  o[2] = v.org[2] + bz * v.B;
}

int layout_level(Mesh& m, int l) {
  Level& v = m.lv[l];
  const int B = v.B;
  size_t ng = (size_t)v.nb[0] * v.nb[1] * v.nb[2];
  std::vector<int8_t> state(ng, ABSENT);
  parallel_for((long long)ng, [&](long long gi) {
    const int bx = (int)(gi % v.nb[0]), by = (int)((gi / v.nb[0]) % v.nb[1]), bz = (int)(gi / ((size_t)v.nb[0] * v.nb[1]));
    int o[3] = {v.org[0] + bx * B, v.org[1] + by * B, v.org[2] + bz * B};
    bool any = false;
    for (int z = 0; z < B && !any; ++z)
      for (int y = 0; y < B && !any; ++y)
        for (int x = 0; x < B && !any; ++x)
          if (live(m, l, o[0] + x, o[1] + y, o[2] + z)) any = true;
    if (any) state[gi] = ACTIVE;
  }, 64);
  std::vector<int8_t> ghost(ng, 0);
  parallel_for((long long)ng, [&](long long gi) {
    if (state[gi] != ABSENT) return;
    const int bx = (int)(gi % v.nb[0]), by = (int)((gi / v.nb[0]) % v.nb[1]), bz = (int)(gi / ((size_t)v.nb[0] * v.nb[1]));
    bool near = false;
    for (int dz = -1; dz <= 1 && !near; ++dz)
      for (int dy = -1; dy <= 1 && !near; ++dy)
        for (int dx = -1; dx <= 1 && !near; ++dx) {
          int n[3] = {bx + dx, by + dy, bz + dz};
          bool ok = true;
          for (int a = 0; a < 3; ++a) {
            if (v.wrap[a]) n[a] = wrapmod(n[a], v.nb[a]);
            if (n[a] < 0 || n[a] >= v.nb[a]) ok = false;
          }
          if (ok && state[((size_t)n[2] * v.nb[1] + n[1]) * v.nb[0] + n[0]] == ACTIVE) near = true;
        }
    if (near) ghost[gi] = 1;
  }, 256);
  for (size_t gi = 0; gi < ng; ++gi)
    if (ghost[gi]) state[gi] = GHOST;
  std::vector<std::pair<uint64_t, int>> act, gho;
  for (size_t gi = 0; gi < ng; ++gi) {
    int bx = (int)(gi % v.nb[0]), by = (int)((gi / v.nb[0]) % v.nb[1]), bz = (int)(gi / ((size_t)v.nb[0] * v.nb[1]));
    if (state[gi] == ACTIVE) act.push_back({morton(bx, by, bz), (int)gi});
    if (state[gi] == GHOST) gho.push_back({morton(bx, by, bz), (int)gi});
  }
  std::sort(act.begin(), act.end());
  std::sort(gho.begin(), gho.end());
  v.slot.assign(ng, -1);
  v.grid_of.clear();
  for (auto& p : act) { v.slot[p.second] = (int)v.grid_of.size(); v.grid_of.push_back(p.second); }
  for (auto& p : gho) { v.slot[p.second] = (int)v.grid_of.size(); v.grid_of.push_back(p.second); }
  v.n_active = (int)act.size();
  v.n_storage = (int)v.grid_of.size();
  const long long cpb = v.cells_per_block();
  v.type.assign((size_t)v.n_storage * cpb, OUTSIDE);
  parallel_for(v.n_storage, [&](long long s) {
    int o[3];
    block_origin(v, v.grid_of[s], o);
    for (int z = 0; z < B; ++z)
      for (int y = 0; y < B; ++y)
        for (int x = 0; x < B; ++x) {
          int gx = o[0] + x, gy = o[1] + y, gz = o[2] + z;
          v.type[(size_t)s * cpb + (z * B + y) * B + x] = base_type(m, l, gx, gy, gz);
        }
  }, 16);
  // neighbour table of active blocks
  v.nbr.assign((size_t)v.n_active * kQ, -1);
  for (int s = 0; s < v.n_active; ++s) {
    int gi = v.grid_of[s];
    int b[3] = {gi % v.nb[0], (gi / v.nb[0]) % v.nb[1], gi / (v.nb[0] * v.nb[1])};
    for (int d = 0; d < kQ; ++d) {
      int n[3] = {b[0] + cx(d), b[1] + cy(d), b[2] + cz(d)};
      for (int a = 0; a < 3; ++a) {
        if (v.wrap[a]) n[a] = wrapmod(n[a], v.nb[a]);
        if (n[a] < 0 || n[a] >= v.nb[a]) {
          m.error = "active block without neighbour storage";
          return LBM_EINVAL;
        }
      }
      int t = v.slot[((size_t)n[2] * v.nb[1] + n[1]) * v.nb[0] + n[0]];
      if (t < 0) {
        m.error = "active block without neighbour storage";
        return LBM_EINVAL;
      }
      v.nbr[(size_t)s * kQ + d] = t;
    }
  }
  return LBM_OK;
}

int classify_solids(Mesh& m, int l, const std::vector<Prim>& prims) {
  Level& v = m.lv[l];
  const int B = v.B;
  const long long cpb = v.cells_per_block();
  const double h = std::ldexp(1.0, m.L - 1 - l);
  std::vector<double> plo(prims.size() * 3), phi(prims.size() * 3);
  for (size_t k = 0; k < prims.size(); ++k) prim_bounds(prims[k], &plo[3 * k], &phi[3 * k]);
  parallel_for(v.n_active, [&](long long s) {
    int o[3];
    block_origin(v, v.grid_of[s], o);
    std::vector<int> cand;
    for (size_t k = 0; k < prims.size(); ++k) {
      bool hit = true;
      for (int a = 0; a < 3; ++a) {
        double lo = o[a] * h - h, hi = (o[a] + B) * h + h;
        if (phi[3 * k + a] < lo || plo[3 * k + a] > hi) hit = false;
      }
      if (hit) cand.push_back((int)k);
    }
    if (cand.empty()) return;
    for (int z = 0; z < B; ++z)
      for (int y = 0; y < B; ++y)
        for (int x = 0; x < B; ++x) {
          uint8_t& t = v.type[(size_t)s * cpb + (z * B + y) * B + x];
          if (t != FLUID) continue;
          double c[3] = {(o[0] + x + 0.5) * h, (o[1] + y + 0.5) * h, (o[2] + z + 0.5) * h};
          for (int k : cand)
            if (prim_contains(prims[k], c)) {
              t = SOLID;
              break;
            }
        }
  }, 4);
  return LBM_OK;
}

int build_links(Mesh& m, int l, const std::vector<Prim>& prims) {
  Level& v = m.lv[l];
  const int B = v.B;
  const long long cpb = v.cells_per_block();
  const double h = std::ldexp(1.0, m.L - 1 - l);
  v.links.clear();
  std::vector<double> plo(prims.size() * 3), phi(prims.size() * 3);
  for (size_t k = 0; k < prims.size(); ++k) prim_bounds(prims[k], &plo[3 * k], &phi[3 * k]);
  std::vector<std::vector<Link>> per_block(v.n_active);
  parallel_for(v.n_active, [&](long long s) {
    int o[3];
    block_origin(v, v.grid_of[s], o);
    // primitives that can hold the entry point of a link of this block: the
    // link segment lies within one cell of the block
    std::vector<int> cand;
    for (size_t k = 0; k < prims.size(); ++k) {
      bool hit = true;
      for (int a = 0; a < 3; ++a) {
        double lo = o[a] * h - h, hi = (o[a] + B) * h + h;
        if (phi[3 * k + a] < lo || plo[3 * k + a] > hi) hit = false;
      }
      if (hit) cand.push_back((int)k);
    }
    std::vector<Link>& out = per_block[s];
    for (int z = 0; z < B; ++z)
      for (int y = 0; y < B; ++y)
        for (int x = 0; x < B; ++x) {
          if (v.type[(size_t)s * cpb + (z * B + y) * B + x] != SOLID) continue;
          int sx = o[0] + x, sy = o[1] + y, sz = o[2] + z;
          for (int i = 0; i < kQ; ++i) {
            if (i == 13) continue;
            int fx = sx - cx(i), fy = sy - cy(i), fz = sz - cz(i);
            if (v.cell_type(fx, fy, fz) != FLUID) continue;
            double p0[3] = {(fx + 0.5) * h, (fy + 0.5) * h, (fz + 0.5) * h};
            double dd[3] = {cx(i) * h, cy(i) * h, cz(i) * h};
            double q = std::numeric_limits<double>::infinity();
            int seg = -1;
            for (int k : cand) {
              const double t = prim_entry(prims[k], p0, dd);
              if (t < q) {
                q = t;
                seg = k;
              }
            }
            if (seg < 0) {  // the solid cell's centre lies inside: first primitive containing it
              double sc[3] = {(sx + 0.5) * h, (sy + 0.5) * h, (sz + 0.5) * h};
              for (size_t k = 0; k < prims.size() && seg < 0; ++k)
                if (prim_contains(prims[k], sc)) seg = (int)k;
            }
            if (!(q <= 1.0)) q = 1.0;
            if (q < 1e-6) q = 1e-6;
            int c[3] = {fx, fy, fz};
            for (int a = 0; a < 3; ++a)
              if (v.wrap[a]) c[a] = wrapmod(c[a], v.dom[a]);
            out.push_back({c[0], c[1], c[2], i, q, seg < 0 ? 0 : seg});
          }
        }
  }, 4);
  size_t nlinks = 0;
  for (const auto& b : per_block) nlinks += b.size();
  v.links.reserve(nlinks);
  for (auto& b : per_block) {
    v.links.insert(v.links.end(), b.begin(), b.end());
    std::vector<Link>().swap(b);
  }
  std::sort(v.links.begin(), v.links.end(), [&](const Link& a, const Link& b) {
    if (a.seg != b.seg) return a.seg < b.seg;
    long long ka = v.addr(a.x, a.y, a.z, 0), kb = v.addr(b.x, b.y, b.z, 0);
    return ka != kb ? ka < kb : a.dir < b.dir;
  });
  v.seg_begin.assign(prims.size() + 1, 0);
  for (const Link& k : v.links) v.seg_begin[k.seg + 1]++;
  for (size_t k = 0; k < prims.size(); ++k) v.seg_begin[k + 1] += v.seg_begin[k];
  for (int p = 0; p < 2; ++p) v.wall[p].assign(v.links.size(), WallEntry{});
  std::atomic<int> bad{0};  // 1: touches an interface, 2: link without storage
  parallel_for((long long)v.links.size(), [&](long long n) {
    const Link& k = v.links[n];
    int i = k.dir, ib = opposite(i);
    int x = k.x, y = k.y, z = k.z;
    // the link cell must not touch another level (its value would be overwritten)
    for (int d = 0; d < kQ; ++d) {
      CellType t = v.cell_type(x + cx(d), y + cy(d), z + cz(d));
      if (t == COVERED || (t == OUTSIDE && l > 0)) {
        bad.store(1);
        return;
      }
    }
    bool back = v.cell_type(x - cx(i), y - cy(i), z - cz(i)) == FLUID;
    WallEntry e0, e1;
    e0.dst = v.addr(x + cx(i), y + cy(i), z + cz(i), i);
    e0.a = v.addr(x, y, z, ib);
    e0.b = back ? v.addr(x - cx(i), y - cy(i), z - cz(i), ib) : -1;
    e0.c = v.addr(x, y, z, i);
    e1.dst = v.addr(x, y, z, ib);
    e1.a = v.addr(x + cx(i), y + cy(i), z + cz(i), i);
    e1.b = back ? v.addr(x, y, z, i) : -1;
    e1.c = v.addr(x - cx(i), y - cy(i), z - cz(i), ib);
    e0.q = e1.q = (float)k.q;
    e0.dir = e1.dir = i;
    e0.seg = e1.seg = k.seg;
    e0.pad = e1.pad = 0;
    if (e0.dst < 0 || e0.a < 0 || e0.c < 0 || e1.a < 0 || e1.c < 0) {
      bad.store(2);
      return;
    }
    v.wall[0][n] = e0;
    v.wall[1][n] = e1;
  }, 1024);
  if (bad.load() == 1) {
    m.error = "the geometry touches a refinement interface";
    return LBM_EINVAL;
  }
  if (bad.load() == 2) {
    m.error = "cut link without storage";
    return LBM_EINVAL;
  }
  return LBM_OK;
}

// Sec. 2.3 faces of level 0: the source a boundary cell pulls from outside.
// Returns false for the inflow equilibrium, else the cell and direction.
bool face_source(const Mesh& m, int gx, int gy, int gz, int i, int* sx, int* sy, int* sz, int* sj) {
  const int* n = m.n0;
  int g[3] = {gx, gy, gz};
  int c[3] = {cx(i), cy(i), cz(i)};
  for (int a = 0; a < 3; ++a)
    if (m.bc[a] == LBM_BC_PERIODIC) g[a] = wrapmod(g[a], n[a]);
  if (g[0] < 0) return false;
  for (int a = 1; a < 3; ++a) {
    if (g[a] >= 0 && g[a] < n[a]) continue;
    if (m.bc[a] == LBM_BC_INFLOW) return false;
    g[a] = g[a] < 0 ? -1 - g[a] : 2 * n[a] - 1 - g[a];
    c[a] = -c[a];
  }
  if (g[0] >= n[0]) g[0] = n[0] - 1;
  *sx = g[0];
  *sy = g[1];
  *sz = g[2];
  *sj = dir_index(c[0], c[1], c[2]);
  return true;
}

int build_faces(Mesh& m) {
  Level& v = m.lv[0];
  const int B = v.B;
  const long long cpb = v.cells_per_block();
  for (int p = 0; p < 2; ++p) v.face[p].clear();
  std::vector<std::vector<FaceEntry>> part0(v.n_active), part1(v.n_active);
  std::vector<std::vector<int>> partp(v.n_active);
  std::atomic<bool> bad{false};
  parallel_for(v.n_active, [&](long long s) {
    int o[3];
    block_origin(v, v.grid_of[s], o);
    bool touches = false;  // only blocks holding a cell on a non-periodic domain face
    for (int a = 0; a < 3; ++a)
      if (m.bc[a] != LBM_BC_PERIODIC && ((o[a] <= 0 && 0 < o[a] + B) || (o[a] <= m.n0[a] - 1 && m.n0[a] - 1 < o[a] + B)))
        touches = true;
    if (!touches) return;
    std::vector<FaceEntry>& f0 = part0[s];
    std::vector<FaceEntry>& f1 = part1[s];
    std::vector<int>& fp = partp[s];
    for (int z = 0; z < B; ++z)
      for (int y = 0; y < B; ++y)
        for (int x = 0; x < B; ++x) {
          if (v.type[(size_t)s * cpb + (z * B + y) * B + x] != FLUID) continue;
          int X = o[0] + x, Y = o[1] + y, Z = o[2] + z;
          bool edge = false;
          for (int a = 0; a < 3; ++a) {
            int c = a == 0 ? X : (a == 1 ? Y : Z);
            if (m.bc[a] != LBM_BC_PERIODIC && (c == 0 || c == m.n0[a] - 1)) edge = true;
          }
          if (!edge) continue;
          for (int i = 0; i < kQ; ++i) {
            int gx = X - cx(i), gy = Y - cy(i), gz = Z - cz(i);
            bool out = false;
            int g[3] = {gx, gy, gz};
            for (int a = 0; a < 3; ++a)
              if (m.bc[a] != LBM_BC_PERIODIC && (g[a] < 0 || g[a] >= m.n0[a])) out = true;
            if (!out) continue;
            int sx, sy, sz, sj;
            bool cell = face_source(m, gx, gy, gz, i, &sx, &sy, &sz, &sj);
            FaceEntry e0{}, e1{};
            e0.dir = e1.dir = i;
            e0.dst = v.addr(gx, gy, gz, opposite(i));
            e1.dst = v.addr(X, Y, Z, i);
            if (cell) {
              e0.src = v.addr(sx, sy, sz, opposite(sj));
              e1.src = v.addr(sx + cx(sj), sy + cy(sj), sz + cz(sj), sj);
            } else {
              e0.src = e1.src = -1;
            }
            if (e0.dst < 0 || e1.dst < 0 || (cell && (e0.src < 0 || e1.src < 0))) {
              bad.store(true);
              return;
            }
            f0.push_back(e0);
            f1.push_back(e1);
            int w[3] = {gx, gy, gz};
            for (int a = 0; a < 3; ++a)
              if (m.bc[a] == LBM_BC_PERIODIC) w[a] = wrapmod(w[a], m.n0[a]);
            fp.insert(fp.end(), {w[0], w[1], w[2], 0});
          }
        }
  }, 8);
  if (bad.load()) {
    m.error = "face slot without storage";
    return LBM_EINVAL;
  }
  v.face_pos.clear();
  for (int s = 0; s < v.n_active; ++s) {
    v.face[0].insert(v.face[0].end(), part0[s].begin(), part0[s].end());
    v.face[1].insert(v.face[1].end(), part1[s].begin(), part1[s].end());
    v.face_pos.insert(v.face_pos.end(), partp[s].begin(), partp[s].end());
  }
  return LBM_OK;
}

// Interface between level l (coarse) and l+1 (fine).  The exchange is the
// exact advection, at fine resolution, of the coarse post-collision field
// held constant over the coarse step by virtual fine cells outside the fine
// region (see the oracle's description of the same scheme); it reduces to:
//  * before the second fine step, a fine cell x whose neighbour x - c_i lies
//    outside receives the coarse post-collision f*_i of parent(x - c_i);
//  * before the next first fine step it receives f*_i of x - 2c_i, which
//    for a box region lies outside too: the coarse value of parent(x - 2c_i);
//  * a coarse cell W next to the fine region receives, per direction, the
//    mean over its 8 children p of: fine f*_i(p - c_i) of the second fine
//    step, or fine f*_i(p - 2c_i) of the first, or coarse f*_i(W - c_i).
int build_interface(Mesh& m, int l) {
  Level& C = m.lv[l];
  Level& F = m.lv[l + 1];
  C.expl.clear();
  C.save.clear();
  C.infl.clear();
  C.coal.clear();
  // errors, reported for the first plane (in z order) that has one
  static const char* const kErr[] = {"", "refinement interface crosses a solid",
                                     "refinement box too close to the coarser level's edge",
                                     "interface slot without storage",
                                     "refinement box too close to a solid or an edge",
                                   "refinement region is not a box"};
  // one part per z plane, concatenated in z order: the tables come out in
  // the order of a sequential z, y, x sweep.  Saved slots are requested by
  // key (per-part request numbers) and numbered at the end, distinct keys in
  // increasing order.
  struct Part {
    std::vector<ExplodeEntry> expl;
    std::vector<InflowEntry> infl;
    std::vector<CoalesceEntry> coal;
    std::vector<long long> want;
    int err = 0;
  };
  auto coarse_post = [&](int X, int Y, int Z, int i, int parity) -> long long {
    if (parity == 0) return C.addr(X, Y, Z, opposite(i));
    return C.addr(X + cx(i), Y + cy(i), Z + cz(i), i);
  };
  const int* lo = F.rlo;
  const int* hi = F.rhi;
  std::vector<Part> fine((size_t)(hi[2] - lo[2]));
  parallel_for(hi[2] - lo[2], [&](long long zi) {
    Part& P = fine[(size_t)zi];
    const int z = lo[2] + (int)zi;
    for (int y = lo[1]; y < hi[1]; ++y) {
      // cells of the box's outer shell only: all of x on the y/z faces, else the two x ends
      const bool face = y == lo[1] || y == hi[1] - 1 || z == lo[2] || z == hi[2] - 1;
      for (int x = lo[0]; x < hi[0]; x = (face || x >= hi[0] - 1) ? x + 1 : hi[0] - 1) {
        for (int i = 0; i < kQ; ++i) {
          int ax = x - cx(i), ay = y - cy(i), az = z - cz(i);
          if (in_box(lo, hi, ax, ay, az)) continue;
          if (F.cell_type(x, y, z) != FLUID) {
            P.err = 1;
            return;
          }
          int px = floordiv(ax, 2), py = floordiv(ay, 2), pz = floordiv(az, 2);
          if (C.cell_type(px, py, pz) != FLUID) {
            P.err = 2;
            return;
          }
          ExplodeEntry e{};
          e.dst = F.addr(ax, ay, az, opposite(i));
          e.src[0] = coarse_post(px, py, pz, i, 0);
          e.src[1] = coarse_post(px, py, pz, i, 1);
          // the value x pulls at the next first sub-step left x - 2 c_i
          // two fine steps before: outside a box (x - c_i is outside, and
          // so is every point further along -c_i), hence the coarse value
          // of its parent
          InflowEntry f{};
          f.dst = F.addr(x, y, z, i);
          f.sv = -1;
          int bx = x - 2 * cx(i), by = y - 2 * cy(i), bz = z - 2 * cz(i);
          if (in_box(lo, hi, bx, by, bz)) {
            P.err = 5;
            return;
          }
          int qx = floordiv(bx, 2), qy = floordiv(by, 2), qz = floordiv(bz, 2);
          if (C.cell_type(qx, qy, qz) != FLUID) {
            P.err = 2;
            return;
          }
          f.csrc[0] = coarse_post(qx, qy, qz, i, 0);
          f.csrc[1] = coarse_post(qx, qy, qz, i, 1);
          if (e.dst < 0 || e.src[0] < 0 || e.src[1] < 0 || f.dst < 0 || f.csrc[0] < 0 || f.csrc[1] < 0) {
            P.err = 3;
            return;
          }
          P.expl.push_back(e);
          P.infl.push_back(f);
        }
      }
    }
  });
  // coarse cells around the footprint [lo/2, hi/2)
  int clo[3], chi[3];
  for (int a = 0; a < 3; ++a) {
    clo[a] = lo[a] / 2;
    chi[a] = hi[a] / 2;
  }
  std::vector<Part> coarse((size_t)(chi[2] - clo[2] + 2));
  parallel_for(chi[2] - clo[2] + 2, [&](long long zi) {
    Part& P = coarse[(size_t)zi];
    const int Z = clo[2] - 1 + (int)zi;
    for (int Y = clo[1] - 1; Y <= chi[1]; ++Y) {
      const bool face = Y == clo[1] - 1 || Y == chi[1] || Z == clo[2] - 1 || Z == chi[2];
      for (int X = clo[0] - 1; X <= chi[0]; X = (face || X >= chi[0]) ? X + 1 : chi[0]) {
        if (C.cell_type(X, Y, Z) != FLUID) {
          P.err = 4;
          return;
        }
        for (int i = 0; i < kQ; ++i) {
          CoalesceEntry e{};
          for (int s = 0; s < 8; ++s) {
            int px = 2 * X + (s & 1), py = 2 * Y + ((s >> 1) & 1), pz = 2 * Z + (s >> 2);
            int ax = px - cx(i), ay = py - cy(i), az = pz - cz(i);
            int bx = px - 2 * cx(i), by = py - 2 * cy(i), bz = pz - 2 * cz(i);
            if (in_box(lo, hi, ax, ay, az)) {
              long long a = F.addr(px, py, pz, i);
              if (a < 0) {
                P.err = 3;
                return;
              }
              e.fsrc[e.nfine++] = a;
            } else if (in_box(lo, hi, bx, by, bz)) {
              P.want.push_back(F.addr(bx, by, bz, opposite(i)));
              e.fsrc[e.nfine++] = -(long long)(P.want.size() - 1) - 1;
            } else {
              e.ncoarse++;
            }
          }
          if (e.nfine == 0) continue;
          e.dst[0] = C.addr(X - cx(i), Y - cy(i), Z - cz(i), opposite(i));
          e.dst[1] = C.addr(X, Y, Z, i);
          if (e.dst[0] < 0 || e.dst[1] < 0) {
            P.err = 3;
            return;
          }
          P.coal.push_back(e);
        }
      }
    }
  });
  for (const auto* parts : {&fine, &coarse})
    for (const Part& P : *parts)
      if (P.err) {
        m.error = kErr[P.err];
        return LBM_EINVAL;
      }
  // concatenate in plane order (parallel copies into pre-sized tables),
  // turning per-part request numbers into global ones
  std::vector<size_t> eo(fine.size() + 1, 0), wo(fine.size() + coarse.size() + 1, 0), co(coarse.size() + 1, 0);
  for (size_t k = 0; k < fine.size(); ++k) {
    eo[k + 1] = eo[k] + fine[k].expl.size();
    wo[k + 1] = wo[k] + fine[k].want.size();
  }
  for (size_t k = 0; k < coarse.size(); ++k) {
    co[k + 1] = co[k] + coarse[k].coal.size();
    wo[fine.size() + k + 1] = wo[fine.size() + k] + coarse[k].want.size();
  }
  C.expl.resize(eo.back());
  C.infl.resize(eo.back());
  C.coal.resize(co.back());
  std::vector<long long> want(wo.back());
  parallel_for((long long)(fine.size() + coarse.size()), [&](long long k) {
    if (k < (long long)fine.size()) {
      Part& P = fine[k];
      std::copy(P.expl.begin(), P.expl.end(), C.expl.begin() + eo[k]);
      std::copy(P.infl.begin(), P.infl.end(), C.infl.begin() + eo[k]);
      std::copy(P.want.begin(), P.want.end(), want.begin() + wo[k]);
    } else {
      const size_t c = (size_t)k - fine.size();
      Part& P = coarse[c];
      for (CoalesceEntry& e : P.coal)
        for (int q = 0; q < e.nfine; ++q)
          if (e.fsrc[q] < 0) e.fsrc[q] -= (long long)wo[k];
      std::copy(P.coal.begin(), P.coal.end(), C.coal.begin() + co[c]);
      std::copy(P.want.begin(), P.want.end(), want.begin() + wo[k]);
    }
  });
  std::vector<Part>().swap(fine);
  std::vector<Part>().swap(coarse);
  std::vector<long long> keys(want);
  parallel_sort(keys);
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  C.save.resize(keys.size());
  for (size_t k = 0; k < keys.size(); ++k) C.save[k].src = keys[k];
  auto resolve = [&](long long req) {
    return (long long)(std::lower_bound(keys.begin(), keys.end(), want[req]) - keys.begin());
  };
  // a saved slot that an inflow entry overwrites (every slot (b, ibar) with
  // b + c_i outside the box is an inflow destination) is saved by that
  // entry's thread just before its write; the save entry itself is skipped
  C.save_dev = C.save;
  parallel_for((long long)C.infl.size(), [&](long long n) {
    InflowEntry& f = C.infl[n];
    auto it = std::lower_bound(keys.begin(), keys.end(), f.dst);
    if (it != keys.end() && *it == f.dst) {
      f.sv = (int)(it - keys.begin());
      C.save_dev[(size_t)f.sv].src = -1;
    }
  }, 4096);
  parallel_for((long long)C.coal.size(), [&](long long n) {
    CoalesceEntry& e = C.coal[n];
    for (int k = 0; k < e.nfine; ++k)
      if (e.fsrc[k] < 0) e.fsrc[k] = -resolve(-e.fsrc[k] - 1) - 1;
  }, 4096);
  return LBM_OK;
}

}  // namespace

// Order of [0, n) by ascending (key(i), i), keys non-negative: a parallel
// sort of 64-bit words key << b | i when they fit (b = bits of n - 1), else of
// key / index pairs.
template <class K>
std::vector<long long> sorted_order(long long n, K&& key) {
  std::vector<long long> perm((size_t)n);
  int b = 1;
  while ((1LL << b) < n) ++b;
  std::atomic<long long> kmax{0};
  parallel_for((n + 65535) / 65536, [&](long long c) {
    long long mx = 0;
    for (long long i = c * 65536; i < std::min(n, (c + 1) * 65536); ++i) mx = std::max(mx, key(i));
    long long cur = kmax.load();
    while (mx > cur && !kmax.compare_exchange_weak(cur, mx)) {
    }
  });
  if (b < 62 && kmax.load() < (1LL << (62 - b))) {
    std::vector<unsigned long long> w((size_t)n);
    parallel_for(n, [&](long long i) { w[(size_t)i] = ((unsigned long long)key(i) << b) | (unsigned long long)i; }, 4096);
    parallel_sort(w);
    const unsigned long long mask = (1ULL << b) - 1;
    parallel_for(n, [&](long long i) { perm[(size_t)i] = (long long)(w[(size_t)i] & mask); }, 4096);
    return perm;
  }
  std::vector<std::pair<long long, long long>> kv((size_t)n);
  parallel_for(n, [&](long long i) { kv[(size_t)i] = {key(i), i}; }, 4096);
  parallel_sort(kv);
  parallel_for(n, [&](long long i) { perm[(size_t)i] = kv[(size_t)i].second; }, 4096);
  return perm;
}
template <class T>
void permute(std::vector<T>& v, const std::vector<long long>& perm, int stride = 1) {
  std::vector<T> out(v.size());
  parallel_for((long long)perm.size(), [&](long long i) {
    for (int k = 0; k < stride; ++k) out[(size_t)i * stride + k] = v[(size_t)perm[i] * stride + k];
  }, 4096);
  v.swap(out);
}

// Table order for the device: entries sorted by destination address, so that
// a warp's threads write neighbouring cells of one population plane instead
// of the 27 planes of one cell (every entry has its own destination, so the
// order changes no result).  Cut links stay grouped by branch (contiguous
// per-branch ranges) and are sorted by destination inside each branch; the
// two parity tables of the faces and of the links share one order with their
// per-entry companions (face positions, links).
// The distinct outside cells the level-0 face entries pull the inflow
// equilibrium from: several entries pull the same cell (along different
// directions), so a turbulent inflow velocity is evaluated once per cell.
static void turbulence_cells(Mesh& m) {
  Level& v = m.lv[0];
  v.turb_cells.clear();
  v.turb_idx.assign(v.face[0].size(), -1);
  if (v.face_pos.size() != 4 * v.face[0].size()) return;
  const long long sx = (long long)m.n0[0] + 2, sy = (long long)m.n0[1] + 2;
  std::unordered_map<long long, int> at;
  at.reserve(v.face[0].size() / 4 + 16);
  for (size_t t = 0; t < v.face[0].size(); ++t) {
    if (v.face[0][t].src >= 0) continue;
    const int* p = &v.face_pos[4 * t];
    const long long key = ((long long)(p[2] + 1) * sy + (p[1] + 1)) * sx + (p[0] + 1);
    auto it = at.emplace(key, (int)(v.turb_cells.size() / 4));
    if (it.second) v.turb_cells.insert(v.turb_cells.end(), {p[0], p[1], p[2], 0});
    v.turb_idx[t] = it.first->second;
  }
}

static void order_tables(Mesh& m) {
  for (int l = 0; l < m.L; ++l) {
    Level& v = m.lv[l];
    if (!v.links.empty()) {
      // links come grouped by branch; sort inside each branch's range
      std::vector<long long> perm(v.links.size());
      for (size_t sg = 0; sg + 1 < v.seg_begin.size(); ++sg) {
        const long long b0 = v.seg_begin[sg], n = v.seg_begin[sg + 1] - b0;
        if (n <= 0) continue;
        const auto local = sorted_order(n, [&](long long i) { return v.wall[0][(size_t)(b0 + i)].dst; });
        for (long long i = 0; i < n; ++i) perm[(size_t)(b0 + i)] = b0 + local[(size_t)i];
      }
      permute(v.links, perm);
      for (int p = 0; p < 2; ++p) permute(v.wall[p], perm);
    }
    if (!v.face[0].empty()) {
      const auto perm = sorted_order((long long)v.face[0].size(),
                                     [&](long long i) { return v.face[0][(size_t)i].dst; });
      for (int p = 0; p < 2; ++p) permute(v.face[p], perm);
      if (v.face_pos.size() == 4 * v.face[0].size()) permute(v.face_pos, perm, 4);
    }
    if (!v.expl.empty())
      permute(v.expl, sorted_order((long long)v.expl.size(),
                                   [&](long long i) { return v.expl[(size_t)i].dst; }));
    if (!v.infl.empty())
      permute(v.infl, sorted_order((long long)v.infl.size(),
                                   [&](long long i) { return v.infl[(size_t)i].dst; }));
    if (!v.coal.empty())
      permute(v.coal, sorted_order((long long)v.coal.size(),
                                   [&](long long i) { return v.coal[(size_t)i].dst[0]; }));
  }
}

// Which boundary kernels may run beside others (as parallel branches of the
// step): a kernel may overlap a sequence of others when no slot it writes is
// read or written by them and no slot it reads is written by them.  Slots are
// keyed (element offset, level); the sets are sorted and probed in parallel.
namespace {
using KeySet = std::vector<long long>;
long long slot_key(int l, long long off) { return off * 8 + l; }
void finish(KeySet& k) {
  parallel_sort(k);
  k.erase(std::unique(k.begin(), k.end()), k.end());
}
bool disjoint(const KeySet& a, const KeySet& b) {
  const KeySet& small = a.size() < b.size() ? a : b;
  const KeySet& large = a.size() < b.size() ? b : a;
  if (small.empty()) return true;
  std::atomic<bool> hit{false};
  const long long n = (long long)small.size(), chunk = 1 << 15;
  parallel_for((n + chunk - 1) / chunk, [&](long long c) {
    for (long long i = c * chunk; i < std::min(n, (c + 1) * chunk) && !hit.load(std::memory_order_relaxed); ++i)
      if (std::binary_search(large.begin(), large.end(), small[(size_t)i])) hit.store(true);
  });
  return !hit.load();
}
}  // namespace

// fill `out` with f(entry k, slot j) for the n entries of `tab`, `per` slots
// each (negative values skipped), in parallel, then sort and deduplicate
template <class T, class F>
void key_set(const std::vector<T>& tab, int per, F&& f, KeySet* out) {
  const size_t base = out->size();
  out->resize(base + tab.size() * (size_t)per, -1);
  parallel_for((long long)tab.size(), [&](long long k) {
    for (int j = 0; j < per; ++j) (*out)[base + (size_t)k * per + j] = f(tab[(size_t)k], j);
  }, 4096);
}
void finish_keys(KeySet& k) {
  k.erase(std::remove(k.begin(), k.end(), -1LL), k.end());
  finish(k);
}

// the exact test at slot level, for the pairs whose block sets met
static void slot_checks(Mesh& m, std::vector<char>* walls_ok, bool* faces_ok) {
  const int L = m.L;
  std::vector<KeySet> iw(L), ir(L), ww(L), wr(L);
  for (int l = 0; l < L; ++l) {
    const Level& v = m.lv[l];
    for (int p = 0; p < 2; ++p) {
      key_set(v.wall[p], 1, [&](const WallEntry& w, int) { return slot_key(l, w.dst); }, &ww[l]);
      key_set(v.wall[p], 3, [&](const WallEntry& w, int j) {
        const long long o = j == 0 ? w.a : (j == 1 ? w.b : w.c);
        return o >= 0 ? slot_key(l, o) : -1LL;
      }, &wr[l]);
    }
    finish_keys(ww[l]);
    finish_keys(wr[l]);
  }
  const Level& v0 = m.lv[0];
  const bool faces = !v0.face[0].empty();
  for (int l = 0; l + 1 < L; ++l) {
    if (!((l == 0 && faces) || !ww[l + 1].empty())) continue;
    const Level& v = m.lv[l];
    const int fl = l + 1;
    key_set(v.expl, 1, [&](const ExplodeEntry& e, int) { return slot_key(fl, e.dst); }, &iw[l]);
    key_set(v.infl, 1, [&](const InflowEntry& e, int) { return slot_key(fl, e.dst); }, &iw[l]);
    key_set(v.coal, 2, [&](const CoalesceEntry& e, int j) { return slot_key(l, e.dst[j]); }, &iw[l]);
    key_set(v.expl, 2, [&](const ExplodeEntry& e, int j) { return slot_key(l, e.src[j]); }, &ir[l]);
    key_set(v.save, 1, [&](const SaveEntry& e, int) { return slot_key(fl, e.src); }, &ir[l]);
    key_set(v.infl, 2, [&](const InflowEntry& e, int j) { return slot_key(l, e.csrc[j]); },
            &ir[l]);
    key_set(v.coal, 8, [&](const CoalesceEntry& e, int j) {
      return j < e.nfine && e.fsrc[j] >= 0 ? slot_key(fl, e.fsrc[j]) : -1LL;
    }, &ir[l]);
    finish_keys(iw[l]);
    finish_keys(ir[l]);
  }
  for (int l = 1; l < L; ++l)
    if (!(*walls_ok)[l])
      (*walls_ok)[l] = !ww[l].empty() && disjoint(ww[l], iw[l - 1]) && disjoint(ww[l], ir[l - 1]) &&
                       disjoint(wr[l], iw[l - 1]);
  if (faces && !*faces_ok) {
    KeySet fw, fr;
    for (int p = 0; p < 2; ++p) {
      key_set(v0.face[p], 1, [&](const FaceEntry& e, int) { return slot_key(0, e.dst); }, &fw);
      key_set(v0.face[p], 1, [&](const FaceEntry& e, int) { return e.src >= 0 ? slot_key(0, e.src) : -1LL; },
              &fr);
    }
    finish_keys(fw);
    finish_keys(fr);
    *faces_ok = disjoint(fw, iw[0]) && disjoint(fw, ir[0]) && disjoint(fw, ww[0]) && disjoint(fw, wr[0]) &&
                disjoint(fr, iw[0]) && disjoint(fr, ww[0]);
  }
}

// Storage blocks a set of slots touches, per level (a slot's block is its
// element offset over 27 B^3): disjoint block sets prove disjoint slot sets
// cheaply, the usual case (tree links deep inside the finest level, faces at
// the domain boundary, interface tables at the refinement boxes).
struct BlockMarks {
  std::vector<std::vector<char>> on;
  explicit BlockMarks(const Mesh& m) : on(m.L) {
    for (int l = 0; l < m.L; ++l) on[l].assign((size_t)std::max(1, m.lv[l].n_storage), 0);
  }
  // block of an element offset: offset / (27 B^3), by a constant divisor
  void mark(const Mesh& m, int l, long long off) {
    if (off < 0) return;
    const long long b = m.B == 16 ? off / (27LL * 4096) : (m.B == 8 ? off / (27LL * 512) : off / (27LL * m.B * m.B * m.B));
    on[l][(size_t)b] = 1;
  }
};
bool blocks_disjoint(const BlockMarks& a, const BlockMarks& b) {
  for (size_t l = 0; l < a.on.size(); ++l)
    for (size_t k = 0; k < a.on[l].size(); ++k)
      if (a.on[l][k] && b.on[l][k]) return false;
  return true;
}

static void overlap_checks(Mesh& m) {
  const int L = m.L;
  // block-level pass: one task per mark set (each writes only its own)
  std::vector<BlockMarks> ww(L, BlockMarks(m)), wr(L, BlockMarks(m)), iwr(L, BlockMarks(m)), iw(L, BlockMarks(m));
  const Level& v0 = m.lv[0];
  BlockMarks fw(m), fr(m);
  std::vector<std::function<void()>> tasks;
  for (int l = 0; l < L; ++l) {
    const Level& v = m.lv[l];
    tasks.push_back([&, l] {
      for (int p = 0; p < 2; ++p)
        for (const WallEntry& w : v.wall[p]) ww[l].mark(m, l, w.dst);
    });
    tasks.push_back([&, l] {
      for (int p = 0; p < 2; ++p)
        for (const WallEntry& w : v.wall[p]) {
          wr[l].mark(m, l, w.a);
          wr[l].mark(m, l, w.b);
          wr[l].mark(m, l, w.c);
        }
    });
    if (l + 1 == L) continue;
    const int fl = l + 1;
    // iw: slots the interface writes; iwr: slots it reads or writes
    tasks.push_back([&, l, fl] {
      for (const ExplodeEntry& e : v.expl) iw[l].mark(m, fl, e.dst);
      for (const InflowEntry& e : v.infl) iw[l].mark(m, fl, e.dst);
      for (const CoalesceEntry& e : v.coal)
        for (int j = 0; j < 2; ++j) iw[l].mark(m, l, e.dst[j]);
    });
    tasks.push_back([&, l, fl] {
      for (const ExplodeEntry& e : v.expl) {
        iwr[l].mark(m, fl, e.dst);
        iwr[l].mark(m, l, e.src[0]);
        iwr[l].mark(m, l, e.src[1]);
      }
      for (const SaveEntry& e : v.save) iwr[l].mark(m, fl, e.src);
      for (const InflowEntry& e : v.infl) {
        iwr[l].mark(m, fl, e.dst);
        iwr[l].mark(m, l, e.csrc[0]);
        iwr[l].mark(m, l, e.csrc[1]);
      }
      for (const CoalesceEntry& e : v.coal) {
        for (int j = 0; j < 2; ++j) iwr[l].mark(m, l, e.dst[j]);
        for (int k = 0; k < e.nfine; ++k) iwr[l].mark(m, fl, e.fsrc[k]);
      }
    });
  }
  tasks.push_back([&] {
    for (int p = 0; p < 2; ++p)
      for (const FaceEntry& e : v0.face[p]) fw.mark(m, 0, e.dst);
  });
  tasks.push_back([&] {
    for (int p = 0; p < 2; ++p)
      for (const FaceEntry& e : v0.face[p]) fr.mark(m, 0, e.src);
  });
  parallel_for((long long)tasks.size(), [&](long long k) { tasks[(size_t)k](); });
  std::vector<char> walls_ok(L, 0);
  for (int l = 1; l < L; ++l)
    walls_ok[l] = !m.lv[l].wall[0].empty() && blocks_disjoint(ww[l], iwr[l - 1]) && blocks_disjoint(wr[l], iw[l - 1]);
  const bool faces = !v0.face[0].empty();
  bool faces_ok = faces && blocks_disjoint(fw, iwr[0]) && blocks_disjoint(fw, ww[0]) && blocks_disjoint(fw, wr[0]) &&
                  blocks_disjoint(fr, iw[0]) && blocks_disjoint(fr, ww[0]);
  bool exact = false;
  for (int l = 1; l < L; ++l) exact |= !walls_ok[l] && !m.lv[l].wall[0].empty();
  exact |= faces && !faces_ok;
  if (exact) slot_checks(m, &walls_ok, &faces_ok);
  for (int l = 0; l < L; ++l) m.lv[l].ovl_walls = walls_ok[l] != 0;
  m.ovl_faces = faces_ok;
}

// Per collide parity p, the active blocks whose update touches no slot the
// wall kernel of the step before (table wall[1 - p]) reads or writes, then
// the others.  An even step touches the own slots of its cells; an odd step
// touches slot (y, m) only from cell y - c_m (its pull of f_mbar and its push
// of f_m), so each wall slot names exactly one updating cell.
static void wall_blocks(Mesh& m) {
  for (int l = 0; l < m.L; ++l) {
    Level& v = m.lv[l];
    for (int p = 0; p < 2; ++p) {
      v.wblocks[p].clear();
      v.n_windep[p] = 0;
    }
    if (v.wall[0].empty()) continue;
    const long long C3 = v.cells_per_block();
    const int B = v.B;
    for (int p = 0; p < 2; ++p) {
      std::vector<char> dep(v.n_active, 0);
      auto touch = [&](long long off) {
        if (off < 0) return;
        const long long sb = off / (kQ * C3);
        if (p == 0) {
          if (sb < v.n_active) dep[(size_t)sb] = 1;
          return;
        }
        const int dir = (int)((off / C3) % kQ), cell = (int)(off % C3);
        int o[3];
        block_origin(v, v.grid_of[(size_t)sb], o);
        int local;
        const int s = v.locate(o[0] + cell % B - cx(dir), o[1] + (cell / B) % B - cy(dir),
                               o[2] + cell / (B * B) - cz(dir), &local);
        if (s >= 0 && s < v.n_active) dep[(size_t)s] = 1;
      };
      for (const WallEntry& w : v.wall[1 - p]) {
        touch(w.dst);
        touch(w.a);
        touch(w.b);
        touch(w.c);
      }
      for (int s = 0; s < v.n_active; ++s)
        if (!dep[(size_t)s]) v.wblocks[p].push_back(s);
      v.n_windep[p] = (int)v.wblocks[p].size();
      for (int s = 0; s < v.n_active; ++s)
        if (dep[(size_t)s]) v.wblocks[p].push_back(s);
    }
  }
}

int build_mesh(const lbm_domain_desc& d, const int boxes[6][6], const std::vector<Prim>& prims, Mesh* out) {
  Mesh& m = *out;
  m.L = d.levels;
  m.B = d.block;
  m.n0[0] = d.nx;
  m.n0[1] = d.ny;
  m.n0[2] = d.nz;
  for (int a = 0; a < 3; ++a) m.bc[a] = d.bc[a];
  std::memcpy(m.boxes, boxes, sizeof(m.boxes));
  m.lv.assign(m.L, Level());
  const int B = m.B;
  for (int l = 0; l < m.L; ++l) {
    Level& v = m.lv[l];
    v.l = l;
    v.B = B;
    if (l == 0) {
      for (int a = 0; a < 3; ++a) {
        v.rlo[a] = 0;
        v.rhi[a] = m.n0[a];
        if (m.bc[a] == LBM_BC_PERIODIC) {
          if (m.n0[a] % B) {
            m.error = "periodic axes must be multiples of the block size";
            return LBM_EINVAL;
          }
          v.wrap[a] = true;
          v.dom[a] = m.n0[a];
          v.org[a] = 0;
          v.nb[a] = m.n0[a] / B;
        } else {
          v.org[a] = -B;
          v.nb[a] = (m.n0[a] + B - 1) / B + 2;
        }
      }
    } else {
      const Level& p = m.lv[l - 1];
      for (int a = 0; a < 3; ++a) {
        v.rlo[a] = boxes[l][a];
        v.rhi[a] = boxes[l][3 + a];
        if (v.rlo[a] % B || v.rhi[a] % B || v.rhi[a] <= v.rlo[a]) {
          m.error = "refinement boxes must be aligned to whole blocks of their level";
          return LBM_EINVAL;
        }
        // footprint inside the parent's real region, two parent cells to spare
        if (v.rlo[a] / 2 < p.rlo[a] + 2 || v.rhi[a] / 2 > p.rhi[a] - 2) {
          m.error = "refinement box leaves less than two cells of margin inside its parent level";
          return LBM_EINVAL;
        }
        v.org[a] = v.rlo[a] - B;
        v.nb[a] = (v.rhi[a] - v.rlo[a]) / B + 2;
      }
    }
  }
  for (int l = 0; l < m.L; ++l) {
    int rc = layout_level(m, l);
    if (rc) return rc;
  }
  for (int l = 0; l < m.L; ++l) {
    classify_solids(m, l, prims);
    Level& v = m.lv[l];
    // collide masks and counts
    const long long cpb = v.cells_per_block();
    std::vector<long long> nf(v.n_active, 0);
    std::atomic<bool> solid{false};
    parallel_for(v.n_active, [&](long long s) {
      const uint8_t* t = &v.type[(size_t)s * cpb];
      long long n = 0;
      bool sol = false;
      for (long long c = 0; c < cpb; ++c) {
        n += t[c] == FLUID;
        sol |= t[c] == SOLID;
      }
      nf[s] = n;
      if (sol) solid.store(true);
    }, 64);
    if (l + 1 < m.L && solid.load()) {
      m.error = "the tree must lie inside the finest level's box";
      return LBM_EINVAL;
    }
    v.maskoff.assign(v.n_active, -1);
    v.n_fluid = 0;
    int nmask = 0;
    for (int s = 0; s < v.n_active; ++s) {
      v.n_fluid += nf[s];
      if (nf[s] != cpb) v.maskoff[s] = nmask++;
    }
    v.masks.assign((size_t)nmask * cpb, 0);
    parallel_for(v.n_active, [&](long long s) {
      if (v.maskoff[s] < 0) return;
      const uint8_t* t = &v.type[(size_t)s * cpb];
      uint8_t* mk = &v.masks[(size_t)v.maskoff[s] * cpb];
      for (long long c = 0; c < cpb; ++c) mk[c] = t[c] == FLUID ? 1 : 0;
    }, 16);
  }
  for (int l = 0; l < m.L; ++l) {
    int rc = build_links(m, l, prims);
    if (rc) return rc;
  }
  int rc = build_faces(m);
  if (rc) return rc;
  for (int l = 0; l + 1 < m.L; ++l) {
    rc = build_interface(m, l);
    if (rc) return rc;
  }
  order_tables(m);
  turbulence_cells(m);
  overlap_checks(m);
  wall_blocks(m);
  return LBM_OK;
}

// 32-bit copies of the boundary and interface tables of every level whose
// own array and (for the interface) finer array hold fewer than 2^31 elements
template <class Wide, class Narrow, class F>
void narrow_copy(const std::vector<Wide>& in, std::vector<Narrow>* out, F&& conv) {
  out->resize(in.size());
  const long long n = (long long)in.size(), chunk = 1 << 16;
  parallel_for((n + chunk - 1) / chunk, [&](long long c) {
    for (long long k = c * chunk; k < std::min(n, (c + 1) * chunk); ++k) (*out)[k] = conv(in[k]);
  });
}

void narrow_tables(Mesh* m) {
  const long long lim = (1LL << 31) - 1;
  for (int l = 0; l < m->L; ++l) {
    Level& v = m->lv[l];
    v.narrow_ok = v.f_elems() <= lim && (l + 1 == m->L || m->lv[l + 1].f_elems() <= lim);
    if (!v.narrow_ok) {
      for (int p = 0; p < 2; ++p) {
        v.wall_n[p].clear();
        v.face_n[p].clear();
      }
      v.expl_n.clear();
      v.save_n.clear();
      v.infl_n.clear();
      v.coal_n.clear();
      continue;
    }
    for (int p = 0; p < 2; ++p) {
      narrow_copy(v.wall[p], &v.wall_n[p], [](const WallEntry& w) {
        return WallEntryN{(int)w.dst, (int)w.a, (int)w.b, (int)w.c, w.q, w.dir};
      });
      narrow_copy(v.face[p], &v.face_n[p],
                  [](const FaceEntry& e) { return FaceEntryN{(int)e.dst, (int)e.src, e.dir}; });
    }
    narrow_copy(v.expl, &v.expl_n,
                [](const ExplodeEntry& e) { return ExplodeEntryN{(int)e.dst, {(int)e.src[0], (int)e.src[1]}}; });
    narrow_copy(v.save_dev, &v.save_n, [](const SaveEntry& e) { return SaveEntryN{(int)e.src}; });
    narrow_copy(v.infl, &v.infl_n, [](const InflowEntry& e) {
      return InflowEntryN{(int)e.dst, {(int)e.csrc[0], (int)e.csrc[1]}, e.sv};
    });
    narrow_copy(v.coal, &v.coal_n, [](const CoalesceEntry& e) {
      CoalesceEntryN o;
      o.dst[0] = (int)e.dst[0];
      o.dst[1] = (int)e.dst[1];
      for (int j = 0; j < 8; ++j) o.fsrc[j] = (int)e.fsrc[j];
      o.nfine = (short)e.nfine;
      o.ncoarse = (short)e.ncoarse;
      return o;
    });
  }
}

}  // namespace lbm
