/*
 * Oracle: lattice Boltzmann time stepping on nested refinement levels.
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 *
 * One time step of a level is "collide, then stream" with two plain arrays
 * (A holds the current values, B receives the streamed ones).
 *
 *  - Streaming, Sec. 2.2: f_i(x, t+1) = f*_i(x - c_i, t).
 *  - Domain faces, Sec. 2.3: uniform inflow U along +x (equilibrium at
 *    rho = 1), zero-gradient outflow, lateral faces periodic, specular slip
 *    or inflow.  The value a fluid cell pulls from outside the domain is
 *    resolved by: wrap periodic axes; x below 0 -> inflow equilibrium;
 *    y, z outside -> inflow equilibrium or mirror the cell and flip that
 *    velocity component (slip); x beyond the outlet -> the last interior
 *    plane.
 *  - Interpolated bounce-back on cut links (Bouzidi et al. 2001, Sec. 2.2),
 *    linear form, with simple bounce-back when the second fluid node is
 *    missing; momentum-exchange force (Wen et al. 2014) for a resting wall:
 *    F = sum over links c_i (f*_i(x_f, t) + f_ibar(x_f, t+1)).
 *  - Refinement (Sec. 2.2 octree AMR, refinement ratio 2, acoustic scaling
 *    nu_{l+1} = 2 nu_l): level l+1 covers the box R_{l+1}; around it the
 *    level-(l+1) array keeps a margin of "virtual" cells.  A level-l step
 *    collides level l, copies every virtual cell's parent post-collision
 *    populations into it, advances level l+1 twice (virtual cells are
 *    streamed like the others but never collided), then streams level l;
 *    each level-l cell next to R_{l+1} instead receives, per direction, the
 *    mean of its 8 children after those two fine steps.  This is the exact
 *    advection at fine resolution of the piecewise-constant coarse field,
 *    hence conserves mass and momentum (volumetric explode / coalesce).
 */
#include <math.h>
#include <omp.h>
#include <stdlib.h>
#include <string.h>
#include "orc.h"

enum { T_FLUID = 0, T_SOLID = 1, T_COVERED = 2, T_VIRTUAL = 3 };
#define MARGIN 4

static int cx(int i) { return i % 3 - 1; }
static int cy(int i) { return (i / 3) % 3 - 1; }
static int cz(int i) { return i / 9 - 1; }
static int opp(int i) { return 26 - i; }
static int dir_of(int x, int y, int z) { return (x + 1) + 3 * (y + 1) + 9 * (z + 1); }

typedef struct {
  int lo[3], n[3];
  int rlo[3], rhi[3];
  long ncell;
  double *A, *B;
  unsigned char* type;
  unsigned char* ring;
  long nlink;
  long* lcell;
  int* ldir;
  double* lq;
  long* lback; /* index of x_f - c_i if it is a fluid cell, else -1 */
  int* lseg;   /* primitive whose surface the link enters first */
  orc_rates rates;
  double F[3];
} lev;

struct orc_sim {
  orc_desc d;
  int L;
  lev lv[6];
  double feq_in[27];
  double Fsum[3];
  long nF;
  int nprim;
  double* Fseg; /* per-primitive running sum of the finest level's force */
  long t;       /* coarse steps done */
  int nturb;    /* random Fourier modes of a turbulent inflow (0: uniform) */
  double* turb; /* per mode: k (3), a (3), psi */
  double u_in;
};

static long lidx(const lev* v, int x, int y, int z) {
  int a = x - v->lo[0], b = y - v->lo[1], c = z - v->lo[2];
  if (a < 0 || b < 0 || c < 0 || a >= v->n[0] || b >= v->n[1] || c >= v->n[2]) return -1;
  return a + (long)v->n[0] * (b + (long)v->n[1] * c);
}
static void lcoord(const lev* v, long id, int* x, int* y, int* z) {
  *x = (int)(id % v->n[0]) + v->lo[0];
  *y = (int)((id / v->n[0]) % v->n[1]) + v->lo[1];
  *z = (int)(id / ((long)v->n[0] * v->n[1])) + v->lo[2];
}
static int in_real(const lev* v, int x, int y, int z) {
  return x >= v->rlo[0] && x < v->rhi[0] && y >= v->rlo[1] && y < v->rhi[1] && z >= v->rlo[2] && z < v->rhi[2];
}
static int wrapi(int a, int n) { a %= n; return a < 0 ? a + n : a; }

/* cell types of every level of the refinement hierarchy (Sec. 2.2's octree
   refinement, boxes per reading 12): fluid, covered by the next finer level,
   or virtual (the margin around a finer level's box), and the ring of coarse
   cells next to a finer box that receive its coalesced populations */
static void classify_levels(orc_sim* s) {
  for (int l = 0; l < s->L; ++l) {
    lev* v = &s->lv[l];
    for (long id = 0; id < v->ncell; ++id) {
      int x, y, z;
      lcoord(v, id, &x, &y, &z);
      unsigned char t = in_real(v, x, y, z) ? T_FLUID : T_VIRTUAL;
      if (t == T_FLUID && l + 1 < s->L) {
        const lev* f = &s->lv[l + 1];
        if (2 * x >= f->rlo[0] && 2 * x < f->rhi[0] && 2 * y >= f->rlo[1] && 2 * y < f->rhi[1] &&
            2 * z >= f->rlo[2] && 2 * z < f->rhi[2])
          t = T_COVERED;
      }
      v->type[id] = t;
    }
  }
  for (int l = 0; l + 1 < s->L; ++l) {
    lev* v = &s->lv[l];
    for (long id = 0; id < v->ncell; ++id) {
      v->ring[id] = 0;
      if (v->type[id] != T_FLUID) continue;
      int x, y, z;
      lcoord(v, id, &x, &y, &z);
      for (int i = 0; i < 27; ++i) {
        long nb = lidx(v, x + cx(i), y + cy(i), z + cz(i));
        if (nb >= 0 && v->type[nb] == T_COVERED) v->ring[id] = 1;
      }
    }
  }
}

orc_sim* orc_create(const orc_desc* d) {
  orc_init();
  if (d->levels < 1 || d->levels > 6 || d->nx < 1 || d->ny < 1 || d->nz < 1) return NULL;
  if (d->bc[0] != ORC_BC_PERIODIC && d->bc[0] != ORC_BC_INOUT) return NULL;
  for (int a = 1; a < 3; ++a)
    if (d->bc[a] == ORC_BC_INOUT) return NULL;
  orc_sim* s = calloc(1, sizeof(orc_sim));
  s->d = *d;
  s->L = d->levels;
  for (int l = 0; l < s->L; ++l) {
    lev* v = &s->lv[l];
    if (l == 0) {
      int n0[3] = {d->nx, d->ny, d->nz};
      for (int a = 0; a < 3; ++a) { v->lo[a] = 0; v->n[a] = n0[a]; v->rlo[a] = 0; v->rhi[a] = n0[a]; }
    } else {
      for (int a = 0; a < 3; ++a) {
        v->rlo[a] = d->box[l][a];
        v->rhi[a] = d->box[l][3 + a];
        if (v->rlo[a] % 2 || v->rhi[a] % 2 || v->rhi[a] <= v->rlo[a]) { orc_destroy(s); return NULL; }
        v->lo[a] = v->rlo[a] - MARGIN;
        v->n[a] = v->rhi[a] - v->rlo[a] + 2 * MARGIN;
      }
    }
    v->ncell = (long)v->n[0] * v->n[1] * v->n[2];
    v->A = calloc(v->ncell * 27, sizeof(double));
    v->B = calloc(v->ncell * 27, sizeof(double));
    v->type = calloc(v->ncell, 1);
    v->ring = calloc(v->ncell, 1);
    double nu = d->nu0 * ldexp(1.0, l);
    v->rates.omega1 = 1.0 / (3.0 * nu + 0.5);
    v->rates.omega2 = d->omega2;
    for (int q = 0; q < 8; ++q) v->rates.omega_hi[q] = d->omega_hi[q];
    v->rates.galilean = d->galilean;
  }
  classify_levels(s);
  /* virtual cells must have fluid parents */
  for (int l = 1; l < s->L; ++l) {
    lev* v = &s->lv[l];
    const lev* p = &s->lv[l - 1];
    for (long id = 0; id < v->ncell; ++id) {
      if (v->type[id] != T_VIRTUAL) continue;
      int x, y, z;
      lcoord(v, id, &x, &y, &z);
      long pid = lidx(p, x >> 1, y >> 1, z >> 1);
      if (pid < 0 || p->type[pid] != T_FLUID || !in_real(p, x >> 1, y >> 1, z >> 1)) {
        orc_destroy(s);
        return NULL;
      }
    }
  }
  double uin[3] = {d->u_in, 0, 0};
  orc_equilibrium(1.0, uin, s->feq_in);
  orc_init_uniform(s, 1.0, uin);
  return s;
}

void orc_destroy(orc_sim* s) {
  if (!s) return;
  for (int l = 0; l < 6; ++l) {
    lev* v = &s->lv[l];
    free(v->A); free(v->B); free(v->type); free(v->ring);
    free(v->lcell); free(v->ldir); free(v->lq); free(v->lback); free(v->lseg);
  }
  free(s->Fseg);
  free(s->turb);
  free(s);
}

void orc_init_uniform(orc_sim* s, double rho, const double u[3]) {
  double feq[27];
  s->t = 0;
  orc_equilibrium(rho, u, feq);
  for (int l = 0; l < s->L; ++l) {
    lev* v = &s->lv[l];
    for (long id = 0; id < v->ncell; ++id) memcpy(v->A + 27 * id, feq, sizeof feq);
    v->F[0] = v->F[1] = v->F[2] = 0;
  }
  s->Fsum[0] = s->Fsum[1] = s->Fsum[2] = 0;
  s->nF = 0;
  if (s->Fseg) memset(s->Fseg, 0, 3 * sizeof(double) * (size_t)s->nprim);
}

int orc_init_field(orc_sim* s, int level, const double* rho, const double* u) {
  if (level < 0 || level >= s->L) return -1;
  lev* v = &s->lv[level];
  long k = 0;
  for (int z = v->rlo[2]; z < v->rhi[2]; ++z)
    for (int y = v->rlo[1]; y < v->rhi[1]; ++y)
      for (int x = v->rlo[0]; x < v->rhi[0]; ++x, ++k) {
        long id = lidx(v, x, y, z);
        orc_equilibrium(rho[k], u + 3 * k, v->A + 27 * id);
      }
  return 0;
}

/* fluid cell index of level-0 coordinates after periodic wrapping, -1 outside */
static long level0_cell(const orc_sim* s, int x, int y, int z) {
  const lev* v = &s->lv[0];
  int g[3] = {x, y, z};
  for (int a = 0; a < 3; ++a) {
    if (s->d.bc[a] == ORC_BC_PERIODIC) g[a] = wrapi(g[a], v->n[a]);
    if (g[a] < 0 || g[a] >= v->n[a]) return -1;
  }
  return lidx(v, g[0], g[1], g[2]);
}

/* solid cells (cell centre inside a primitive, inclusive) and the cut links
   of Sec. 2.2's interpolated bounce-back: for every fluid cell and direction
   c_i reaching a solid cell, the wall fraction q (first entry of the ray,
   clamped to [1e-6, 1]), the second fluid node x_f - c_i and the branch the
   link belongs to (reading 17) */
int orc_set_prims(orc_sim* s, const orc_prim* pr, int np) {
  int L = s->L;
  classify_levels(s); /* fresh cell types and ring flags */
  for (int l = 0; l < L; ++l) {
    lev* v = &s->lv[l];
    double h = ldexp(1.0, L - 1 - l);
    for (long id = 0; id < v->ncell; ++id) {
      if (v->type[id] != T_FLUID) continue;
      int x, y, z;
      lcoord(v, id, &x, &y, &z);
      double c[3] = {(x + 0.5) * h, (y + 0.5) * h, (z + 0.5) * h};
      if (orc_prim_inside(pr, np, c)) v->type[id] = T_SOLID;
    }
    free(v->lcell); free(v->ldir); free(v->lq); free(v->lback); free(v->lseg);
    long cap = 1024, nl = 0;
    v->lcell = malloc(cap * sizeof(long));
    v->ldir = malloc(cap * sizeof(int));
    v->lq = malloc(cap * sizeof(double));
    v->lback = malloc(cap * sizeof(long));
    v->lseg = malloc(cap * sizeof(int));
    for (long id = 0; id < v->ncell; ++id) {
      if (v->type[id] != T_FLUID) continue;
      int x, y, z;
      lcoord(v, id, &x, &y, &z);
      for (int i = 0; i < 27; ++i) {
        if (i == 13) continue;
        long nb = l == 0 ? level0_cell(s, x + cx(i), y + cy(i), z + cz(i))
                         : lidx(v, x + cx(i), y + cy(i), z + cz(i));
        if (nb < 0 || v->type[nb] != T_SOLID) continue;
        double p0[3] = {(x + 0.5) * h, (y + 0.5) * h, (z + 0.5) * h};
        double dd[3] = {cx(i) * h, cy(i) * h, cz(i) * h};
        /* the link's branch: the primitive its ray enters first (ties: lowest index),
           or, if no ray entry is found, the first primitive holding the solid centre */
        double q = INFINITY;
        int seg = -1;
        for (int k = 0; k < np; ++k) {
          double tk = orc_prim_ray(pr + k, 1, p0, dd);
          if (tk < q) { q = tk; seg = k; }
        }
        if (seg < 0) {
          long sid = l == 0 ? level0_cell(s, x + cx(i), y + cy(i), z + cz(i)) : lidx(v, x + cx(i), y + cy(i), z + cz(i));
          int sx, sy, sz;
          lcoord(v, sid, &sx, &sy, &sz);
          double sc[3] = {(sx + 0.5) * h, (sy + 0.5) * h, (sz + 0.5) * h};
          for (int k = 0; k < np && seg < 0; ++k)
            if (orc_prim_inside(pr + k, 1, sc)) seg = k;
          if (seg < 0) seg = 0;
        }
        if (!(q <= 1.0)) q = 1.0;
        if (q < 1e-6) q = 1e-6;
        long bk = l == 0 ? level0_cell(s, x - cx(i), y - cy(i), z - cz(i))
                         : lidx(v, x - cx(i), y - cy(i), z - cz(i));
        if (bk >= 0 && v->type[bk] != T_FLUID) bk = -1;
        if (l > 0 && bk >= 0) {
          int bx, by, bz;
          lcoord(v, bk, &bx, &by, &bz);
          if (!in_real(v, bx, by, bz)) bk = -1;
        }
        if (v->ring[id]) return -3; /* the tree must stay clear of refinement interfaces */
        if (nl == cap) {
          cap *= 2;
          v->lcell = realloc(v->lcell, cap * sizeof(long));
          v->ldir = realloc(v->ldir, cap * sizeof(int));
          v->lq = realloc(v->lq, cap * sizeof(double));
          v->lback = realloc(v->lback, cap * sizeof(long));
          v->lseg = realloc(v->lseg, cap * sizeof(int));
        }
        v->lcell[nl] = id; v->ldir[nl] = i; v->lq[nl] = q; v->lback[nl] = bk; v->lseg[nl] = seg;
        ++nl;
      }
    }
    v->nlink = nl;
  }
  free(s->Fseg);
  s->nprim = np;
  s->Fseg = calloc(3 * (size_t)(np > 0 ? np : 1), sizeof(double));
  return 0;
}

/* value of f*_i pulled from level-0 position g (possibly outside the domain) */
/* inflow equilibrium pulled from level-0 cell g (periodic axes wrapped):
   uniform, or at u = U e_x + sum_n a_n cos(k_n . (p - U t e_x) + psi_n), p the
   cell centre, t the coarse steps done (frozen synthetic turbulence) */
static double inflow_value(const orc_sim* s, const int g[3], int i) {
  if (s->nturb == 0) return s->feq_in[i];
  double p[3] = {g[0] + 0.5 - s->u_in * (double)s->t, g[1] + 0.5, g[2] + 0.5};
  double u[3] = {s->u_in, 0, 0};
  for (int n = 0; n < s->nturb; ++n) {
    const double* m = s->turb + 7 * n;
    double c = cos(m[0] * p[0] + m[1] * p[1] + m[2] * p[2] + m[6]);
    for (int a = 0; a < 3; ++a) u[a] += m[3 + a] * c;
  }
  double feq[27];
  orc_equilibrium(1.0, u, feq);
  return feq[i];
}

/* Sec. 2.3's domain faces: the value a level-0 cell pulls from position g,
   inside or outside the domain (inflow face, lateral inflow or slip faces,
   zero-gradient outflow; periodic axes wrap) */
static double pull0(const orc_sim* s, const double* A, int gx, int gy, int gz, int i) {
  const lev* v = &s->lv[0];
  int g[3] = {gx, gy, gz};
  for (int a = 0; a < 3; ++a)
    if (s->d.bc[a] == ORC_BC_PERIODIC) g[a] = wrapi(g[a], v->n[a]);
  if (g[0] < 0) return inflow_value(s, g, i); /* inflow face */
  int c[3] = {cx(i), cy(i), cz(i)};
  for (int a = 1; a < 3; ++a) {
    if (g[a] < 0 || g[a] >= v->n[a]) {
      if (s->d.bc[a] == ORC_BC_INFLOW) return inflow_value(s, g, i);
      /* specular slip: mirror the cell across the face, flip that component */
      g[a] = g[a] < 0 ? -1 - g[a] : 2 * v->n[a] - 1 - g[a];
      c[a] = -c[a];
    }
  }
  if (g[0] >= v->n[0]) g[0] = v->n[0] - 1; /* zero-gradient outflow */
  int j = dir_of(c[0], c[1], c[2]);
  return A[27 * lidx(v, g[0], g[1], g[2]) + j];
}

/* the cumulant collision (Sec. 2.2, Geier et al. 2015) of every fluid cell
   of level l, in place, at the level's rates (omega1 from nu_l) */
static void collide_level(orc_sim* s, int l) {
  lev* v = &s->lv[l];
  const double* F = (l == 0 && s->L == 1) ? s->d.force : NULL;
#pragma omp parallel for schedule(static)
  for (long id = 0; id < v->ncell; ++id) {
    if (v->type[id] != T_FLUID) continue;
    double out[27];
    orc_collide(v->A + 27 * id, out, &v->rates, F);
    memcpy(v->A + 27 * id, out, sizeof out);
  }
}

/* streaming f_i(x, t+1) = f*_i(x - c_i, t) of level l into the second array
   (Sec. 2.2), the faces of Sec. 2.3 on level 0, then the interpolated
   bounce-back of every cut link (Bouzidi et al. 2001) with its
   momentum-exchange force (Wen et al. 2014), and the coalesce transfer from
   the next finer level into the ring cells */
static void stream_level(orc_sim* s, int l) {
  lev* v = &s->lv[l];
  const double* A = v->A;
  double* B = v->B;
#pragma omp parallel for schedule(static)
  for (long id = 0; id < v->ncell; ++id) {
    unsigned char t = v->type[id];
    if (t != T_FLUID && t != T_VIRTUAL) continue;
    int x, y, z;
    lcoord(v, id, &x, &y, &z);
    for (int i = 0; i < 27; ++i) {
      int gx = x - cx(i), gy = y - cy(i), gz = z - cz(i);
      if (l == 0) {
        B[27 * id + i] = pull0(s, A, gx, gy, gz, i);
      } else {
        long g = lidx(v, gx, gy, gz);
        B[27 * id + i] = g >= 0 ? A[27 * g + i] : NAN; /* edge of the margin: never used */
      }
    }
  }
  /* interpolated bounce-back and momentum exchange */
  double F[3] = {0, 0, 0};
  /* per-branch forces take the gauge form: the rest state (rho = 1, u = 0,
     f = w) is subtracted from every link, since one branch's links do not
     close a surface and the uniform reference pressure would not cancel */
  double wrest[27];
  const double zero[3] = {0, 0, 0};
  orc_equilibrium(1.0, zero, wrest);
  for (long k = 0; k < v->nlink; ++k) {
    long id = v->lcell[k];
    int i = v->ldir[k], ib = opp(i);
    double q = v->lq[k];
    double fa = A[27 * id + i];   /* f*_i(x_f, t), toward the wall */
    double fc = A[27 * id + ib];  /* f*_ibar(x_f, t) */
    double out;
    if (v->lback[k] < 0) out = fa; /* second fluid node missing: simple bounce-back */
    else if (q < 0.5) out = 2 * q * fa + (1 - 2 * q) * A[27 * v->lback[k] + i];
    else out = fa / (2 * q) + (2 * q - 1) / (2 * q) * fc;
    B[27 * id + ib] = out;
    F[0] += cx(i) * (fa + out);
    F[1] += cy(i) * (fa + out);
    F[2] += cz(i) * (fa + out);
    if (l == s->L - 1 && s->Fseg) {
      double* g = s->Fseg + 3 * v->lseg[k];
      const double gs = fa + out - 2.0 * wrest[i];
      g[0] += cx(i) * gs;
      g[1] += cy(i) * gs;
      g[2] += cz(i) * gs;
    }
  }
  v->F[0] = F[0]; v->F[1] = F[1]; v->F[2] = F[2];
  if (l == s->L - 1) {
    for (int a = 0; a < 3; ++a) s->Fsum[a] += F[a];
    s->nF++;
  }
  /* coalesce: level-l cells next to R_{l+1} take the mean of their children */
  if (l + 1 < s->L) {
    const lev* f = &s->lv[l + 1];
#pragma omp parallel for schedule(static)
    for (long id = 0; id < v->ncell; ++id) {
      if (!v->ring[id]) continue;
      int x, y, z;
      lcoord(v, id, &x, &y, &z);
      for (int i = 0; i < 27; ++i) {
        double sum = 0;
        for (int c = 0; c < 8; ++c) {
          long ch = lidx(f, 2 * x + (c & 1), 2 * y + ((c >> 1) & 1), 2 * z + (c >> 2));
          sum += f->A[27 * ch + i];
        }
        B[27 * id + i] = sum / 8.0;
      }
    }
  }
  v->A = B;
  v->B = (double*)A;
}

/* one step of level l with recursive sub-cycling (acoustic scaling): collide
   level l, explode its post-collision populations into the next finer
   level's virtual cells, advance that level twice, then stream level l */
static void step_level(orc_sim* s, int l) {
  collide_level(s, l);
  if (l + 1 < s->L) {
    lev* v = &s->lv[l];
    lev* f = &s->lv[l + 1];
    /* explode: virtual cells take their parent's post-collision populations */
#pragma omp parallel for schedule(static)
    for (long id = 0; id < f->ncell; ++id) {
      if (f->type[id] != T_VIRTUAL) continue;
      int x, y, z;
      lcoord(f, id, &x, &y, &z);
      long p = lidx(v, x >> 1, y >> 1, z >> 1);
      memcpy(f->A + 27 * id, v->A + 27 * p, 27 * sizeof(double));
    }
    step_level(s, l + 1);
    step_level(s, l + 1);
  }
  stream_level(s, l);
}

void orc_step(orc_sim* s, int ncoarse) {
  for (int n = 0; n < ncoarse; ++n) {
    step_level(s, 0);
    s->t++;
  }
}

int orc_set_turbulence(orc_sim* s, const double* modes, int n, double u_in) {
  if (n < 0) return -1;
  free(s->turb);
  s->turb = NULL;
  s->nturb = 0;
  if (n > 0) {
    s->turb = malloc(7 * sizeof(double) * (size_t)n);
    if (!s->turb) return -1;
    memcpy(s->turb, modes, 7 * sizeof(double) * (size_t)n);
  }
  s->nturb = n;
  s->u_in = u_in;
  return 0;
}

void orc_level_box(const orc_sim* s, int level, int lo[3], int hi[3]) {
  const lev* v = &s->lv[level];
  for (int a = 0; a < 3; ++a) { lo[a] = v->rlo[a]; hi[a] = v->rhi[a]; }
}

void orc_get_f(const orc_sim* s, int level, double* out) {
  const lev* v = &s->lv[level];
  long k = 0;
  for (int z = v->rlo[2]; z < v->rhi[2]; ++z)
    for (int y = v->rlo[1]; y < v->rhi[1]; ++y)
      for (int x = v->rlo[0]; x < v->rhi[0]; ++x, ++k) {
        long id = lidx(v, x, y, z);
        for (int i = 0; i < 27; ++i)
          out[27 * k + i] = v->type[id] == T_FLUID ? v->A[27 * id + i] : NAN;
      }
}

void orc_get_macro(const orc_sim* s, int level, double* rho, double* u) {
  const lev* v = &s->lv[level];
  const double* F = (level == 0 && s->L == 1) ? s->d.force : NULL;
  long k = 0;
  for (int z = v->rlo[2]; z < v->rhi[2]; ++z)
    for (int y = v->rlo[1]; y < v->rhi[1]; ++y)
      for (int x = v->rlo[0]; x < v->rhi[0]; ++x, ++k) {
        long id = lidx(v, x, y, z);
        if (v->type[id] != T_FLUID) {
          rho[k] = NAN; u[3 * k] = u[3 * k + 1] = u[3 * k + 2] = NAN;
          continue;
        }
        double r = 0, j[3] = {0, 0, 0};
        for (int i = 0; i < 27; ++i) {
          double f = v->A[27 * id + i];
          r += f; j[0] += f * cx(i); j[1] += f * cy(i); j[2] += f * cz(i);
        }
        rho[k] = r;
        for (int a = 0; a < 3; ++a) u[3 * k + a] = (j[a] + (F ? 0.5 * F[a] : 0.0)) / r;
      }
}

int orc_level_links(const orc_sim* s, int level, long* cell, int* dir, double* q, int max) {
  const lev* v = &s->lv[level];
  if (!cell) return (int)v->nlink;
  int n = 0;
  for (long k = 0; k < v->nlink && n < max; ++k, ++n) {
    int x, y, z;
    lcoord(v, v->lcell[k], &x, &y, &z);
    /* report the cell as a linear index over the level's real box */
    long rx = x - v->rlo[0], ry = y - v->rlo[1], rz = z - v->rlo[2];
    long nxr = v->rhi[0] - v->rlo[0], nyr = v->rhi[1] - v->rlo[1];
    cell[n] = rx + nxr * (ry + nyr * rz);
    dir[n] = v->ldir[k];
    q[n] = v->lq[k];
  }
  return n;
}

/* the primitive (branch) each cut link of a level is attributed to, in the
   order of orc_level_links */
int orc_level_link_segs(const orc_sim* s, int level, int* seg, int max) {
  const lev* v = &s->lv[level];
  int n = 0;
  for (long k = 0; k < v->nlink && n < max; ++k, ++n) seg[n] = v->lseg[k];
  return n;
}

void orc_force(const orc_sim* s, double last[3], double sum[3], long* nsum) {
  const lev* v = &s->lv[s->L - 1];
  for (int a = 0; a < 3; ++a) { last[a] = v->F[a]; sum[a] = s->Fsum[a]; }
  *nsum = s->nF;
}

void orc_mass(const orc_sim* s, double* mass, double mom[3]) {
  double m = 0, p[3] = {0, 0, 0};
  for (int l = 0; l < s->L; ++l) {
    const lev* v = &s->lv[l];
    double w = ldexp(1.0, -3 * l), ml = 0, pl[3] = {0, 0, 0};
    for (long id = 0; id < v->ncell; ++id) {
      if (v->type[id] != T_FLUID) continue;
      for (int i = 0; i < 27; ++i) {
        double f = v->A[27 * id + i];
        ml += f; pl[0] += f * cx(i); pl[1] += f * cy(i); pl[2] += f * cz(i);
      }
    }
    m += w * ml;
    for (int a = 0; a < 3; ++a) p[a] += w * pl[a];
  }
  *mass = m;
  for (int a = 0; a < 3; ++a) mom[a] = p[a];
}

int orc_cell_type(const orc_sim* s, int level, unsigned char* out) {
  const lev* v = &s->lv[level];
  long k = 0;
  for (int z = v->rlo[2]; z < v->rhi[2]; ++z)
    for (int y = v->rlo[1]; y < v->rhi[1]; ++y)
      for (int x = v->rlo[0]; x < v->rhi[0]; ++x, ++k) out[k] = v->type[lidx(v, x, y, z)];
  return (int)k;
}

/* per-branch mean force of the finest level since the last initialisation */
int orc_branch_forces(const orc_sim* s, double* mean, int n) {
  if (n < s->nprim) return -1;
  for (int k = 0; k < s->nprim; ++k)
    for (int a = 0; a < 3; ++a) mean[3 * k + a] = s->nF > 0 ? s->Fseg[3 * k + a] / (double)s->nF : 0.0;
  return s->nprim;
}

int orc_set_threads(int n) {
  int prev = omp_get_max_threads();
  if (n >= 1) omp_set_num_threads(n);
  return prev;
}
