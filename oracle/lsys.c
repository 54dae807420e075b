/*
 * Oracle: L-system tree, placement, solid primitives and frontal area.
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 */
#include <math.h>
#include <string.h>
#include "orc.h"

#define DEG (3.14159265358979323846 / 180.0)

/* SplitMix64 (Steele, Lea & Flood 2014): the k-th output of a generator
   seeded with `seed` is the mix of seed + (k+1)*gamma. */
static uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

typedef struct { double h[3], l[3], u[3]; } frame;

/* "+" (Table of symbols): rotation about U, frame columns [H L U] times R_U(a) */
static frame rot_u(frame f, double a) {
  frame g = f;
  double c = cos(a), s = sin(a);
  for (int k = 0; k < 3; ++k) {
    g.h[k] = f.h[k] * c - f.l[k] * s;
    g.l[k] = f.h[k] * s + f.l[k] * c;
  }
  return g;
}
/* "/" : rotation about H, frame columns [H L U] times R_H(a) */
static frame rot_h(frame f, double a) {
  frame g = f;
  double c = cos(a), s = sin(a);
  for (int k = 0; k < 3; ++k) {
    g.l[k] = f.l[k] * c + f.u[k] * s;
    g.u[k] = -f.l[k] * s + f.u[k] * c;
  }
  return g;
}

typedef struct { const orc_tree* t; double* seg; int n, max; } lctx;

/* Rule p1 of Eq. (1): A(s,w): s >= min -> !(w) F(s) [child 1] [child 2] ...
   applied to an apex of generation g; after n rewritings apices of
   generation n remain unexpanded and draw nothing. */
static void apex(lctx* c, int g, double s, double w, const double p[3], frame f) {
  const orc_tree* t = c->t;
  if (g >= t->n || s < t->min_len) return;
  if (c->n >= c->max) { c->n = c->max + 1; return; }
  int id = c->n++;
  double e[3];
  for (int k = 0; k < 3; ++k) e[k] = p[k] + s * f.h[k];
  double* row = c->seg + 8 * (long)id;
  row[0] = p[0]; row[1] = p[1]; row[2] = p[2];
  row[3] = e[0]; row[4] = e[1]; row[5] = e[2];
  row[6] = w; row[7] = g;
  for (int k = 0; k < t->children; ++k) {
    frame cf;
    if (t->azimuth_mode == 0) {
      cf = rot_h(rot_u(f, t->alpha_deg[k] * DEG), t->phi_deg[k] * DEG);
    } else {
      uint64_t z = splitmix64_at(t->seed, (uint64_t)id * (uint64_t)t->children + (uint64_t)k);
      double phi = 360.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0));
      cf = rot_u(rot_h(f, phi * DEG), t->alpha_deg[k] * DEG);
    }
    apex(c, g + 1, s * t->r[k], w * t->dfac[k], e, cf);
  }
}

int orc_lsystem(const orc_tree* t, double* seg, int max_seg) {
  if (t->children < 1 || t->children > 4 || t->n < 0) return -1;
  lctx c = {t, seg, 0, max_seg};
  frame f0 = {{0, 0, 1}, {1, 0, 0}, {0, 1, 0}}; /* H up (+z), L = +x, U = H x L = +y */
  double p0[3] = {0, 0, 0};
  apex(&c, 0, t->s0, t->w0, p0, f0);
  return c.n > max_seg ? -2 : c.n;
}

static void seg_axis(const double* r, double a[3], double* len) {
  double d[3] = {r[3] - r[0], r[4] - r[1], r[5] - r[2]};
  double l = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  for (int k = 0; k < 3; ++k) a[k] = d[k] / l;
  *len = l;
}

/* exact axis-aligned bounding box of the union of flat-capped cylinders */
void orc_tree_bbox(const double* seg, int n, double lo[3], double hi[3]) {
  for (int k = 0; k < 3; ++k) { lo[k] = INFINITY; hi[k] = -INFINITY; }
  for (int i = 0; i < n; ++i) {
    const double* r = seg + 8 * i;
    double a[3], len;
    seg_axis(r, a, &len);
    for (int k = 0; k < 3; ++k) {
      double env = 0.5 * r[6] * sqrt(fmax(0.0, 1.0 - a[k] * a[k]));
      double mn = fmin(r[k], r[3 + k]) - env, mx = fmax(r[k], r[3 + k]) + env;
      if (mn < lo[k]) lo[k] = mn;
      if (mx > hi[k]) hi[k] = mx;
    }
  }
}

/* tree height H (Table 2): vertical extent of the cylinders, envelope included */
double orc_tree_height(const double* seg, int n) {
  double lo[3], hi[3];
  orc_tree_bbox(seg, n, lo, hi);
  return hi[2] - lo[2];
}

/* centre of mass (Sec. 2.3): volume-weighted centroid of the cylinders */
void orc_tree_com(const double* seg, int n, double com[3]) {
  double vs = 0, m[3] = {0, 0, 0};
  for (int i = 0; i < n; ++i) {
    const double* r = seg + 8 * i;
    double a[3], len;
    seg_axis(r, a, &len);
    double v = 0.25 * 3.14159265358979323846 * r[6] * r[6] * len;
    vs += v;
    for (int k = 0; k < 3; ++k) m[k] += v * 0.5 * (r[k] + r[3 + k]);
  }
  for (int k = 0; k < 3; ++k) com[k] = m[k] / vs;
}

void orc_transform(double* seg, int n, double scale, const double shift[3]) {
  for (int i = 0; i < n; ++i) {
    double* r = seg + 8 * i;
    for (int k = 0; k < 3; ++k) {
      r[k] = r[k] * scale + shift[k];
      r[3 + k] = r[3 + k] * scale + shift[k];
    }
    r[6] *= scale;
  }
}

/* ---- primitives ---- */

/* parameter interval [t0,t1] of the line x + t d inside an infinite solid
   cylinder / slab; returns 0 if empty */
static int cyl_interval(const double* r, const double x[3], const double d[3], double* t0, double* t1) {
  double a[3], len;
  seg_axis(r, a, &len);
  double rad = 0.5 * r[6];
  double w[3] = {x[0] - r[0], x[1] - r[1], x[2] - r[2]};
  double wa = w[0] * a[0] + w[1] * a[1] + w[2] * a[2];
  double da = d[0] * a[0] + d[1] * a[1] + d[2] * a[2];
  double wp[3], dp[3];
  for (int k = 0; k < 3; ++k) { wp[k] = w[k] - wa * a[k]; dp[k] = d[k] - da * a[k]; }
  double A = dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2];
  double B = wp[0] * dp[0] + wp[1] * dp[1] + wp[2] * dp[2];
  double C = wp[0] * wp[0] + wp[1] * wp[1] + wp[2] * wp[2] - rad * rad;
  double lo = -INFINITY, hi = INFINITY;
  if (A < 1e-300) {
    if (C > 0) return 0;
  } else {
    double disc = B * B - A * C;
    if (disc < 0) return 0;
    double sq = sqrt(disc);
    lo = (-B - sq) / A;
    hi = (-B + sq) / A;
  }
  /* slab 0 <= (w + t d).a <= len */
  if (fabs(da) < 1e-300) {
    if (wa < 0 || wa > len) return 0;
  } else {
    double s0 = (0.0 - wa) / da, s1 = (len - wa) / da;
    if (s0 > s1) { double tmp = s0; s0 = s1; s1 = tmp; }
    if (s0 > lo) lo = s0;
    if (s1 < hi) hi = s1;
  }
  if (lo > hi) return 0;
  *t0 = lo; *t1 = hi;
  return 1;
}

static int prim_inside1(const orc_prim* p, const double x[3]) {
  if (p->kind == 0) {
    double a[3], len;
    seg_axis(p->p, a, &len);
    double w[3] = {x[0] - p->p[0], x[1] - p->p[1], x[2] - p->p[2]};
    double wa = w[0] * a[0] + w[1] * a[1] + w[2] * a[2];
    if (wa < 0 || wa > len) return 0;
    double q2 = 0;
    for (int k = 0; k < 3; ++k) { double c = w[k] - wa * a[k]; q2 += c * c; }
    return q2 <= 0.25 * p->p[6] * p->p[6];
  } else if (p->kind == 1) {
    return p->p[0] * x[0] + p->p[1] * x[1] + p->p[2] * x[2] <= p->p[3];
  } else {
    for (int k = 0; k < 3; ++k)
      if (x[k] < p->p[k] || x[k] > p->p[3 + k]) return 0;
    return 1;
  }
}

int orc_prim_inside(const orc_prim* pr, int n, const double x[3]) {
  for (int i = 0; i < n; ++i)
    if (prim_inside1(pr + i, x)) return 1;
  return 0;
}

/* smallest t >= 0 at which x + t d enters any primitive; INFINITY if none */
double orc_prim_ray(const orc_prim* pr, int n, const double x[3], const double d[3]) {
  double best = INFINITY;
  for (int i = 0; i < n; ++i) {
    const orc_prim* p = pr + i;
    double t = INFINITY;
    if (p->kind == 0) {
      double t0, t1;
      if (cyl_interval(p->p, x, d, &t0, &t1) && t1 >= 0) t = t0 > 0 ? t0 : 0;
    } else if (p->kind == 1) {
      double nx = p->p[0] * x[0] + p->p[1] * x[1] + p->p[2] * x[2];
      double nd = p->p[0] * d[0] + p->p[1] * d[1] + p->p[2] * d[2];
      if (nx <= p->p[3]) t = 0;
      else if (nd < 0) t = (p->p[3] - nx) / nd;
    } else {
      double lo = -INFINITY, hi = INFINITY;
      int ok = 1;
      for (int k = 0; k < 3 && ok; ++k) {
        if (fabs(d[k]) < 1e-300) {
          if (x[k] < p->p[k] || x[k] > p->p[3 + k]) ok = 0;
        } else {
          double a = (p->p[k] - x[k]) / d[k], b = (p->p[3 + k] - x[k]) / d[k];
          if (a > b) { double tmp = a; a = b; b = tmp; }
          if (a > lo) lo = a;
          if (b < hi) hi = b;
        }
      }
      if (ok && lo <= hi && hi >= 0) t = lo > 0 ? lo : 0;
    }
    if (t < best) best = t;
  }
  return best;
}

/* projected frontal area A_x (Sec. 3, Eq. 7): pixels of pitch h on the y-z
   plane, centred at ((j+1/2)h, (k+1/2)h), counted when the line parallel to
   x through the pixel centre meets any cylinder */
double orc_frontal_area(const double* seg, int n, double pitch) {
  double lo[3], hi[3];
  orc_tree_bbox(seg, n, lo, hi);
  long j0 = (long)floor(lo[1] / pitch) - 1, j1 = (long)ceil(hi[1] / pitch) + 1;
  long k0 = (long)floor(lo[2] / pitch) - 1, k1 = (long)ceil(hi[2] / pitch) + 1;
  long count = 0;
  double d[3] = {1, 0, 0};
  for (long k = k0; k <= k1; ++k)
    for (long j = j0; j <= j1; ++j) {
      double x[3] = {0.0, (j + 0.5) * pitch, (k + 0.5) * pitch};
      for (int i = 0; i < n; ++i) {
        double t0, t1;
        if (cyl_interval(seg + 8 * i, x, d, &t0, &t1)) { ++count; break; }
      }
    }
  return (double)count * pitch * pitch;
}

/* exported for the generator's published test vector */
uint64_t orc_splitmix64(uint64_t seed, uint64_t k) { return splitmix64_at(seed, k); }
