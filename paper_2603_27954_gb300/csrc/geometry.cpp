// Tree geometry of Sec. 2.1: the parametric L-system of Eq. (1) rewritten as
// a module string and drawn by a turtle; placement helpers; solid
// primitives with ray entry points; projected frontal area (Eq. 7).
#include <algorithm>
#include <cmath>
#include <limits>
#include <vector>

#include "internal.h"
#include "parallel.h"

namespace lbm {

// SplitMix64 (Steele, Lea & Flood 2014), counter form: output number k of
// a generator seeded with `seed`.
uint64_t splitmix(uint64_t seed, uint64_t k) {
  uint64_t z = seed + 0x9E3779B97F4A7C15ULL * (k + 1);
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ULL;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

namespace {

constexpr double kPi = 3.14159265358979323846;

struct Module {
  char sym;     // 'A' apex, '!' width, 'F' segment, '[' ']', '+' about U, '/' about H
  double a, b;  // A: s, w; '!': w; 'F': s; '+': angle; '/': angle
  int child;    // '/': child index when the angle is drawn from the seed, else -1
};

struct Turtle {
  double p[3], h[3], l[3], u[3];
  double width;
  int depth;
  int last_f;
};

void turn_u(Turtle& t, double deg) {  // "+": frame [H L U] times R_U
  double a = deg * kPi / 180.0, c = std::cos(a), s = std::sin(a);
  for (int k = 0; k < 3; ++k) {
    double h = t.h[k], l = t.l[k];
    t.h[k] = h * c - l * s;
    t.l[k] = h * s + l * c;
  }
}
void roll_h(Turtle& t, double deg) {  // "/": frame [H L U] times R_H
  double a = deg * kPi / 180.0, c = std::cos(a), s = std::sin(a);
  for (int k = 0; k < 3; ++k) {
    double l = t.l[k], u = t.u[k];
    t.l[k] = l * c + u * s;
    t.u[k] = -l * s + u * c;
  }
}

double seg_unit_axis(const double* r, double a[3]) {
  double d[3] = {r[3] - r[0], r[4] - r[1], r[5] - r[2]};
  double len = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  for (int k = 0; k < 3; ++k) a[k] = d[k] / len;
  return len;
}

// Interval [t0, t1] of the line x + t d inside a flat-capped cylinder
// (intersection of the infinite cylinder and the slab between the caps).
bool cylinder_span(const double* r, const double x[3], const double d[3], double* t0, double* t1) {
  double a[3];
  double len = seg_unit_axis(r, a);
  double rad2 = 0.25 * r[6] * r[6];
  double rel[3] = {x[0] - r[0], x[1] - r[1], x[2] - r[2]};
  double ra = rel[0] * a[0] + rel[1] * a[1] + rel[2] * a[2];
  double da = d[0] * a[0] + d[1] * a[1] + d[2] * a[2];
  double pr[3], pd[3];
  for (int k = 0; k < 3; ++k) {
    pr[k] = rel[k] - ra * a[k];
    pd[k] = d[k] - da * a[k];
  }
  double qa = pd[0] * pd[0] + pd[1] * pd[1] + pd[2] * pd[2];
  double qb = pr[0] * pd[0] + pr[1] * pd[1] + pr[2] * pd[2];
  double qc = pr[0] * pr[0] + pr[1] * pr[1] + pr[2] * pr[2] - rad2;
  double lo = -std::numeric_limits<double>::infinity(), hi = -lo;
  if (qa < 1e-300) {
    if (qc > 0) return false;
  } else {
    double disc = qb * qb - qa * qc;
    if (disc < 0) return false;
    double sq = std::sqrt(disc);
    lo = (-qb - sq) / qa;
    hi = (-qb + sq) / qa;
  }
  if (std::fabs(da) < 1e-300) {
    if (ra < 0 || ra > len) return false;
  } else {
    double e0 = -ra / da, e1 = (len - ra) / da;
    if (e0 > e1) std::swap(e0, e1);
    lo = std::max(lo, e0);
    hi = std::min(hi, e1);
  }
  if (lo > hi) return false;
  *t0 = lo;
  *t1 = hi;
  return true;
}

}  // namespace

int build_lsystem(const lbm_tree_desc& t, Tree* out) {
  if (t.n < 0 || t.n > 12 || t.children < 1 || t.children > 4 || !(t.s0 > 0) || !(t.w0 > 0))
    return LBM_EINVAL;
  // rewriting: rule p1 applied n times to every apex with s >= min
  std::vector<Module> str{{'A', t.s0, t.w0, -1}};
  for (int it = 0; it < t.n; ++it) {
    std::vector<Module> next;
    next.reserve(str.size() * 8);
    for (const Module& m : str) {
      if (m.sym != 'A' || m.a < t.min_len) {
        next.push_back(m);
        continue;
      }
      next.push_back({'!', m.b, 0, -1});
      next.push_back({'F', m.a, 0, -1});
      for (int k = 0; k < t.children; ++k) {
        next.push_back({'[', 0, 0, -1});
        if (t.azimuth_mode == 0) {
          next.push_back({'+', t.alpha_deg[k], 0, -1});
          next.push_back({'/', t.phi_deg[k], 0, -1});
        } else {
          next.push_back({'/', 0, 0, k});
          next.push_back({'+', t.alpha_deg[k], 0, -1});
        }
        next.push_back({'A', m.a * t.r[k], m.b * t.dfac[k], -1});
        next.push_back({']', 0, 0, -1});
      }
    }
    str.swap(next);
    if (str.size() > (size_t)50'000'000) return LBM_EINVAL;
  }
  // interpretation
  out->seg.clear();
  Turtle tu{{0, 0, 0}, {0, 0, 1}, {1, 0, 0}, {0, 1, 0}, t.w0, 0, -1};
  std::vector<Turtle> stack;
  int nf = 0;
  for (const Module& m : str) {
    switch (m.sym) {
      case '!': tu.width = m.a; break;
      case 'F': {
        double e[3];
        for (int k = 0; k < 3; ++k) e[k] = tu.p[k] + m.a * tu.h[k];
        double row[8] = {tu.p[0], tu.p[1], tu.p[2], e[0], e[1], e[2], tu.width, (double)tu.depth};
        out->seg.insert(out->seg.end(), row, row + 8);
        for (int k = 0; k < 3; ++k) tu.p[k] = e[k];
        tu.last_f = nf++;
        break;
      }
      case '[':
        stack.push_back(tu);
        tu.depth += 1;
        break;
      case ']':
        tu = stack.back();
        stack.pop_back();
        break;
      case '+': turn_u(tu, m.a); break;
      case '/': {
        double ang = m.a;
        if (m.child >= 0) {
          uint64_t z = splitmix(t.seed, (uint64_t)tu.last_f * (uint64_t)t.children + (uint64_t)m.child);
          ang = 360.0 * (double)(z >> 11) * (1.0 / 9007199254740992.0);
        }
        roll_h(tu, ang);
        break;
      }
      default: break;
    }
  }
  return LBM_OK;
}

void tree_bounds(const Tree& t, double lo[3], double hi[3]) {
  for (int k = 0; k < 3; ++k) {
    lo[k] = std::numeric_limits<double>::infinity();
    hi[k] = -lo[k];
  }
  for (int s = 0; s < t.count(); ++s) {
    Prim p{0, {}};
    std::copy(&t.seg[8 * s], &t.seg[8 * s] + 8, p.p);
    double a[3], b[3];
    prim_bounds(p, a, b);
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::min(lo[k], a[k]);
      hi[k] = std::max(hi[k], b[k]);
    }
  }
}

double tree_height(const Tree& t) {
  double lo[3], hi[3];
  tree_bounds(t, lo, hi);
  return hi[2] - lo[2];
}

void tree_centroid(const Tree& t, double c[3]) {
  double vol = 0, acc[3] = {0, 0, 0};
  for (int s = 0; s < t.count(); ++s) {
    const double* r = &t.seg[8 * s];
    double a[3];
    double len = seg_unit_axis(r, a);
    double v = kPi * 0.25 * r[6] * r[6] * len;
    vol += v;
    for (int k = 0; k < 3; ++k) acc[k] += v * 0.5 * (r[k] + r[k + 3]);
  }
  for (int k = 0; k < 3; ++k) c[k] = acc[k] / vol;
}

void tree_affine(Tree* t, double scale, const double shift[3]) {
  for (int s = 0; s < t->count(); ++s) {
    double* r = &t->seg[8 * s];
    for (int k = 0; k < 3; ++k) {
      r[k] = r[k] * scale + shift[k];
      r[k + 3] = r[k + 3] * scale + shift[k];
    }
    r[6] *= scale;
  }
}

// Eq. (7) needs A_x: the union of the cylinders' shadows on the y-z plane,
// sampled at pixel centres ((j+1/2)h, (k+1/2)h).
double frontal_area(const Tree& t, double pitch) {
  if (t.count() == 0) return 0.0;
  double lo[3], hi[3];
  tree_bounds(t, lo, hi);
  long j0 = (long)std::floor(lo[1] / pitch) - 1, j1 = (long)std::ceil(hi[1] / pitch) + 1;
  long k0 = (long)std::floor(lo[2] / pitch) - 1, k1 = (long)std::ceil(hi[2] / pitch) + 1;
  long nj = j1 - j0 + 1, nk = k1 - k0 + 1;
  const double dir[3] = {1, 0, 0};
  const int n = t.count();
  std::vector<long> box((size_t)4 * n);  // pixel ranges ja, jb, ka, kb per branch
  for (int s = 0; s < n; ++s) {
    Prim p{0, {}};
    std::copy(&t.seg[8 * s], &t.seg[8 * s] + 8, p.p);
    double a[3], b[3];
    prim_bounds(p, a, b);
    box[4 * s] = std::max(j0, (long)std::floor(a[1] / pitch) - 1);
    box[4 * s + 1] = std::min(j1, (long)std::ceil(b[1] / pitch) + 1);
    box[4 * s + 2] = std::max(k0, (long)std::floor(a[2] / pitch) - 1);
    box[4 * s + 3] = std::min(k1, (long)std::ceil(b[2] / pitch) + 1);
  }
  // one pixel row (fixed k) per task; a pixel counts once whatever covers it
  std::vector<long> row_count((size_t)nk, 0);
  parallel_for(nk, [&](long long kr) {
    const long k = k0 + (long)kr;
    std::vector<uint8_t> hit((size_t)nj, 0);
    for (int s = 0; s < n; ++s) {
      if (k < box[4 * s + 2] || k > box[4 * s + 3]) continue;
      const double* r = &t.seg[8 * s];
      for (long j = box[4 * s]; j <= box[4 * s + 1]; ++j) {
        uint8_t& h = hit[(size_t)(j - j0)];
        if (h) continue;
        double x[3] = {0.0, (j + 0.5) * pitch, (k + 0.5) * pitch};
        double t0, t1;
        if (cylinder_span(r, x, dir, &t0, &t1)) h = 1;
      }
    }
    long c = 0;
    for (uint8_t h : hit) c += h;
    row_count[(size_t)kr] = c;
  }, 4);
  long count = 0;
  for (long c : row_count) count += c;
  return (double)count * pitch * pitch;
}

bool prim_contains(const Prim& p, const double x[3]) {
  switch (p.kind) {
    case 0: {
      double a[3];
      double len = seg_unit_axis(p.p, a);
      double rel[3] = {x[0] - p.p[0], x[1] - p.p[1], x[2] - p.p[2]};
      double along = rel[0] * a[0] + rel[1] * a[1] + rel[2] * a[2];
      if (along < 0 || along > len) return false;
      double perp2 = 0;
      for (int k = 0; k < 3; ++k) {
        double c = rel[k] - along * a[k];
        perp2 += c * c;
      }
      return perp2 <= 0.25 * p.p[6] * p.p[6];
    }
    case 1:
      return p.p[0] * x[0] + p.p[1] * x[1] + p.p[2] * x[2] <= p.p[3];
    default:
      return x[0] >= p.p[0] && x[0] <= p.p[3] && x[1] >= p.p[1] && x[1] <= p.p[4] && x[2] >= p.p[2] &&
             x[2] <= p.p[5];
  }
}

double prim_entry(const Prim& p, const double x[3], const double d[3]) {
  const double inf = std::numeric_limits<double>::infinity();
  switch (p.kind) {
    case 0: {
      double t0, t1;
      if (!cylinder_span(p.p, x, d, &t0, &t1) || t1 < 0) return inf;
      return std::max(t0, 0.0);
    }
    case 1: {
      double nx = p.p[0] * x[0] + p.p[1] * x[1] + p.p[2] * x[2];
      double nd = p.p[0] * d[0] + p.p[1] * d[1] + p.p[2] * d[2];
      if (nx <= p.p[3]) return 0.0;
      if (nd >= 0) return inf;
      return (p.p[3] - nx) / nd;
    }
    default: {
      double lo = -inf, hi = inf;
      for (int k = 0; k < 3; ++k) {
        if (std::fabs(d[k]) < 1e-300) {
          if (x[k] < p.p[k] || x[k] > p.p[k + 3]) return inf;
          continue;
        }
        double e0 = (p.p[k] - x[k]) / d[k], e1 = (p.p[k + 3] - x[k]) / d[k];
        if (e0 > e1) std::swap(e0, e1);
        lo = std::max(lo, e0);
        hi = std::min(hi, e1);
      }
      if (lo > hi || hi < 0) return inf;
      return std::max(lo, 0.0);
    }
  }
}

void prim_bounds(const Prim& p, double lo[3], double hi[3]) {
  const double inf = std::numeric_limits<double>::infinity();
  switch (p.kind) {
    case 0: {
      double a[3];
      seg_unit_axis(p.p, a);
      for (int k = 0; k < 3; ++k) {
        double env = 0.5 * p.p[6] * std::sqrt(std::max(0.0, 1.0 - a[k] * a[k]));
        lo[k] = std::min(p.p[k], p.p[k + 3]) - env;
        hi[k] = std::max(p.p[k], p.p[k + 3]) + env;
      }
      return;
    }
    case 1:
      for (int k = 0; k < 3; ++k) {
        lo[k] = -inf;
        hi[k] = inf;
      }
      return;
    default:
      for (int k = 0; k < 3; ++k) {
        lo[k] = p.p[k];
        hi[k] = p.p[k + 3];
      }
  }
}

// Branch-wise description of the tree (Sec. 2.4): per cylinder its length L,
// diameter D, the angle alpha between its axis and the flow (x), and the
// inputs of the sectional-drag surrogate.  Shielding depth: the mean, over 16
// points along the axis, of the number of other cylinders that the
// x-parallel line through the point meets upstream of it.
void branch_table(const Tree& t, double u, double nu, double height, double i_u, std::vector<double>* out) {
  const int n = t.count();
  out->assign((size_t)n * LBM_BRANCH_COLS, 0.0);
  const double dir[3] = {1, 0, 0};
  // does the stream-wise line through p meet another branch m != k that it
  // enters at x < xmax?  (the line starts on the x = 0 plane)
  auto upstream = [&](int k, const double p[3], double xmax, int* count) {
    const double x0[3] = {0.0, p[1], p[2]};
    int c = 0;
    for (int m = 0; m < n; ++m) {
      if (m == k) continue;
      double t0, t1;
      if (cylinder_span(&t.seg[8 * m], x0, dir, &t0, &t1) && t0 < xmax) ++c;
    }
    if (count) *count = c;
    return c > 0;
  };
  for (int k = 0; k < n; ++k) {
    const double* r = &t.seg[8 * k];
    double a[3];
    const double len = seg_unit_axis(r, a);
    const double D = r[6];
    const double cosa = a[0];  // signed: the axis points from the branch's base to its tip
    const double sina = std::sqrt(std::max(0.0, 1.0 - cosa * cosa));
    // shielding depth: other branches entered upstream along 16 axis points
    double shield = 0;
    for (int j = 0; j < 16; ++j) {
      const double s = (j + 0.5) / 16.0;
      const double p[3] = {r[0] + s * (r[3] - r[0]), r[1] + s * (r[4] - r[1]), r[2] + s * (r[5] - r[2])};
      int c = 0;
      upstream(k, p, p[0], &c);
      shield += c;
    }
    // shadowed fraction of the silhouette: 16 axial x 5 lateral points across
    // the projected width (lateral direction normal to the axis and the flow)
    double w[3] = {0.0, a[2], -a[1]};  // a x e_x
    const double wn = std::sqrt(w[1] * w[1] + w[2] * w[2]);
    if (wn > 1e-9) {
      w[1] /= wn;
      w[2] /= wn;
    } else {
      w[1] = 1.0;
      w[2] = 0.0;
    }
    int shadowed = 0;
    for (int j = 0; j < 16; ++j) {
      const double s = (j + 0.5) / 16.0;
      for (int l = -2; l <= 2; ++l) {
        const double o = 0.2 * l * D;
        const double p[3] = {r[0] + s * (r[3] - r[0]) + o * w[0], r[1] + s * (r[4] - r[1]) + o * w[1],
                             r[2] + s * (r[5] - r[2]) + o * w[2]};
        if (upstream(k, p, p[0] - 0.5 * D, nullptr)) ++shadowed;
      }
    }
    // leaf: no other branch starts at this branch's tip
    bool leaf = true;
    for (int m = 0; m < n && leaf; ++m) {
      if (m == k) continue;
      const double* q = &t.seg[8 * m];
      if (std::fabs(q[0] - r[3]) + std::fabs(q[1] - r[4]) + std::fabs(q[2] - r[5]) < 1e-9 * (1.0 + len)) leaf = false;
    }
    double* row = &(*out)[(size_t)LBM_BRANCH_COLS * k];
    row[0] = std::log10(u * D / nu);  // local Reynolds number of the branch
    row[1] = r[7];                    // generation
    row[2] = D / height;
    row[3] = cosa;  // cosine of the angle to the flow
    row[4] = i_u;
    row[5] = shield / 16.0;
    row[6] = len;
    row[7] = D;
    row[8] = sina * sina * sina;
    row[9] = shadowed / 80.0;
    row[10] = leaf ? 1.0 : 0.0;
  }
}

}  // namespace lbm
