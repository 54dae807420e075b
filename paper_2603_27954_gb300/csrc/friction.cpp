// Surface quadrature for the friction force (C_F, Sec. 3: the wall shear
// stress integrated over the whole tree surface).  The paper does not say how
// the shear is taken from the lattice; here every primitive's surface is
// covered by quadrature points (spacing 1/2 finest cell), each with its
// outward normal n and area dA.  The stress at a point is extrapolated
// linearly to the wall from two fluid cells along the normal: A, the
// finest-level cell containing x + delta n for the first delta in {1, 1.5, 2}
// that is fluid, and B, the cell containing x + (delta + 1) n when it is fluid
// and lies at least 1/4 cell farther out (else the stress of A alone).
// Points inside another primitive (junctions, overlaps) are not part of the
// wetted surface and are dropped.
//
// Cylinders: lateral points on N_s x N_t lines (N_s = ceil(L / h), N_t =
// max(8, ceil(2 pi r / h)), s = (i + 1/2) L / N_s, theta = 2 pi (j + 1/2) / N_t,
// radial direction cos(theta) e1 + sin(theta) e2 with e1 = a x z / |a x z|
// (a x x when |a x z| < 0.1) and e2 = a x e1); each end cap on N_r
// equal-width rings (N_r = ceil(r / h)), ring m with max(4, ceil(2 pi rho_m /
// h)) points at rho_m = (m + 1/2) r / N_r.  Half-spaces n . x <= d: a grid of
// spacing h over the two axes other than n's largest component, across the
// finest level's real region, each point projected onto the plane along that
// axis, dA = h^2 / |n_max|.  Boxes carry no points.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"
#include "parallel.h"

namespace lbm {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kSpacing = 0.5;

void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

double norm3(const double a[3]) { return std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }

struct Point {
  double x[3], n[3], area;
};

void cylinder_points(const double* r, std::vector<Point>* out) {
  double a[3] = {r[3] - r[0], r[4] - r[1], r[5] - r[2]};
  const double len = norm3(a);
  for (double& v : a) v /= len;
  const double rad = 0.5 * r[6];
  double e1[3], e2[3];
  const double z[3] = {0, 0, 1}, xx[3] = {1, 0, 0};
  cross3(a, z, e1);
  if (norm3(e1) < 0.1) cross3(a, xx, e1);
  const double n1 = norm3(e1);
  for (double& v : e1) v /= n1;
  cross3(a, e1, e2);
  const int ns = std::max(1, (int)std::ceil(len / kSpacing));
  const int nt = std::max(8, (int)std::ceil(2 * kPi * rad / kSpacing));
  const double dA = (2 * kPi * rad / nt) * (len / ns);
  for (int i = 0; i < ns; ++i)
    for (int j = 0; j < nt; ++j) {
      const double s = (i + 0.5) * len / ns, th = 2 * kPi * (j + 0.5) / nt;
      Point p;
      for (int k = 0; k < 3; ++k) {
        p.n[k] = std::cos(th) * e1[k] + std::sin(th) * e2[k];
        p.x[k] = r[k] + s * a[k] + rad * p.n[k];
      }
      p.area = dA;
      out->push_back(p);
    }
  const int nr = std::max(1, (int)std::ceil(rad / kSpacing));
  for (int end = 0; end < 2; ++end) {
    const double* c = end ? r + 3 : r;
    const double sgn = end ? 1.0 : -1.0;
    for (int m = 0; m < nr; ++m) {
      const double rho = (m + 0.5) * rad / nr;
      const int nphi = std::max(4, (int)std::ceil(2 * kPi * rho / kSpacing));
      const double ring = kPi * rad * rad * (2 * m + 1) / ((double)nr * nr);
      for (int j = 0; j < nphi; ++j) {
        const double ph = 2 * kPi * (j + 0.5) / nphi;
        Point p;
        for (int k = 0; k < 3; ++k) {
          p.n[k] = sgn * a[k];
          p.x[k] = c[k] + rho * (std::cos(ph) * e1[k] + std::sin(ph) * e2[k]);
        }
        p.area = ring / nphi;
        out->push_back(p);
      }
    }
  }
}

void plane_points(const double* pl, const Level& v, std::vector<Point>* out) {
  const double nn = norm3(pl);
  if (nn < 1e-12) return;
  const double n[3] = {pl[0] / nn, pl[1] / nn, pl[2] / nn};
  const double dist = pl[3] / nn;
  int ax = 0;
  for (int k = 1; k < 3; ++k)
    if (std::fabs(n[k]) > std::fabs(n[ax])) ax = k;
  const int u = (ax + 1) % 3, w = (ax + 2) % 3;
  const int nu = (int)std::ceil((v.rhi[u] - v.rlo[u]) / kSpacing);
  const int nw = (int)std::ceil((v.rhi[w] - v.rlo[w]) / kSpacing);
  const double dA = kSpacing * kSpacing / std::fabs(n[ax]);
  for (int i = 0; i < nu; ++i)
    for (int j = 0; j < nw; ++j) {
      Point p;
      p.x[u] = v.rlo[u] + (i + 0.5) * kSpacing;
      p.x[w] = v.rlo[w] + (j + 0.5) * kSpacing;
      p.x[ax] = (dist - n[u] * p.x[u] - n[w] * p.x[w]) / n[ax];
      for (int k = 0; k < 3; ++k) p.n[k] = n[k];
      p.area = dA;
      out->push_back(p);
    }
}

}  // namespace

int build_friction_samples(const Mesh& m, const std::vector<Prim>& prims, std::vector<FrictionSample>* out,
                           std::vector<int>* seg_begin) {
  const Level& v = m.lv[m.L - 1];
  out->clear();
  seg_begin->assign(prims.size() + 1, 0);
  std::vector<std::vector<FrictionSample>> per(prims.size());
  parallel_for((long long)prims.size(), [&](long long k) {
    std::vector<Point> pts;
    if (prims[k].kind == 0) cylinder_points(prims[k].p, &pts);
    else if (prims[k].kind == 1) plane_points(prims[k].p, v, &pts);
    for (const Point& p : pts) {
      bool inside = false;
      for (size_t o = 0; o < prims.size() && !inside; ++o)
        if (o != (size_t)k && prim_contains(prims[o], p.x)) inside = true;
      if (inside) continue;
      auto cell_at = [&](double delta, int c[3]) {
        for (int q = 0; q < 3; ++q) c[q] = (int)std::floor(p.x[q] + delta * p.n[q]);
        return v.cell_type(c[0], c[1], c[2]) == FLUID;
      };
      auto dist = [&](const int c[3]) {
        double d = 0;
        for (int q = 0; q < 3; ++q) d += (c[q] + 0.5 - p.x[q]) * p.n[q];
        return d;
      };
      for (double delta : {1.0, 1.5, 2.0}) {
        int ca[3], cb[3];
        if (!cell_at(delta, ca)) continue;
        FrictionSample s{};
        s.slot[0] = v.locate(ca[0], ca[1], ca[2], &s.cell[0]);
        s.dist[0] = (float)dist(ca);
        s.slot[1] = -1;
        s.cell[1] = 0;
        s.dist[1] = 0;
        if (cell_at(delta + 1.0, cb) && dist(cb) > dist(ca) + 0.25) {
          s.slot[1] = v.locate(cb[0], cb[1], cb[2], &s.cell[1]);
          s.dist[1] = (float)dist(cb);
        }
        for (int q = 0; q < 3; ++q) s.n[q] = (float)p.n[q];
        s.area = (float)p.area;
        s.seg = (int)k;
        per[k].push_back(s);
        break;
      }
    }
  });
  for (size_t k = 0; k < prims.size(); ++k) {
    (*seg_begin)[k + 1] = (*seg_begin)[k] + (int)per[k].size();
    out->insert(out->end(), per[k].begin(), per[k].end());
  }
  return LBM_OK;
}

}  // namespace lbm
