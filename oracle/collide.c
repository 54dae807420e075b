/*
 * Oracle: D3Q27 velocity set, equilibrium and the cumulant collision of
 * Geier et al. (2015), the collision model named in Sec. 2.2.
 * TEST INFRASTRUCTURE ONLY (see orc.h).
 *
 * Conventions of this file:
 *   population index i = (cx+1) + 3 (cy+1) + 9 (cz+1)
 *   moment / cumulant multi-index (a,b,c), a,b,c in {0,1,2}, index a + 3b + 9c
 *   k_abc are the cumulants of the normalised distribution f/rho (derivatives
 *   of log sum_i f_i exp(Xi.c_i) at Xi = 0); Geier's C_abc = rho * k_abc.
 * The collision computes central moments by their definition, converts them
 * to cumulants with the set-partition formula of joint cumulants, relaxes
 * each cumulant group toward its equilibrium, converts back with the inverse
 * partition formula and recovers populations from the 27 central moments by
 * inverting the moment map (a Kronecker product of three 3x3 matrices).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "orc.h"

static int CX[27], CY[27], CZ[27];

/* ---- set partitions of the multiset behind each multi-index ---- */
typedef struct { int nblk; int blk[3]; double coef; } term;
static term TERMS[27][64];
static int NTERMS[27];
static int INIT_DONE = 0;

static void record_partition(int t, const int* lab, int n, const int* g, int nb) {
  int cnt[6][3];
  int size[6] = {0};
  memset(cnt, 0, sizeof cnt);
  for (int e = 0; e < n; ++e) { cnt[g[e]][lab[e]]++; size[g[e]]++; }
  if (nb > 3) return;
  for (int b = 0; b < nb; ++b) if (size[b] < 2) return; /* first central moments vanish */
  term* tm = &TERMS[t][NTERMS[t]++];
  tm->nblk = nb;
  for (int b = 0; b < nb; ++b) tm->blk[b] = cnt[b][0] + 3 * cnt[b][1] + 9 * cnt[b][2];
  double fact = 1;
  for (int q = 2; q < nb; ++q) fact *= q;
  tm->coef = ((nb - 1) % 2 ? -1.0 : 1.0) * fact; /* (-1)^(k-1) (k-1)! */
}

/* every set partition of the n labelled elements, as restricted growth strings */
static void partitions(int t, const int* lab, int n, int e, int* g, int nb) {
  if (e == n) { record_partition(t, lab, n, g, nb); return; }
  for (int b = 0; b <= nb; ++b) {
    g[e] = b;
    partitions(t, lab, n, e + 1, g, b == nb ? nb + 1 : nb);
  }
}

static void add_partitions(int t, const int* lab, int n) {
  int g[6] = {0};
  NTERMS[t] = 0;
  if (n < 2) return;
  partitions(t, lab, n, 1, g, 1);
}

void orc_init(void) {
  if (INIT_DONE) return;
  for (int i = 0; i < 27; ++i) {
    CX[i] = i % 3 - 1;
    CY[i] = (i / 3) % 3 - 1;
    CZ[i] = i / 9 - 1;
  }
  for (int t = 0; t < 27; ++t) {
    int a = t % 3, b = (t / 3) % 3, c = t / 9;
    int lab[6], n = 0;
    for (int q = 0; q < a; ++q) lab[n++] = 0;
    for (int q = 0; q < b; ++q) lab[n++] = 1;
    for (int q = 0; q < c; ++q) lab[n++] = 2;
    add_partitions(t, lab, n);
  }
  INIT_DONE = 1;
}

/* textbook equilibrium: rho times a product of 1-D three-point distributions,
   each with mean u_a and variance 1/3 (all higher lattice cumulants zero) */
static double phi1(int c, double u) {
  if (c == 0) return 2.0 / 3.0 - u * u;
  return 0.5 * (1.0 / 3.0 + u * u + c * u);
}
void orc_equilibrium(double rho, const double u[3], double* feq) {
  orc_init();
  for (int i = 0; i < 27; ++i)
    feq[i] = rho * phi1(CX[i], u[0]) * phi1(CY[i], u[1]) * phi1(CZ[i], u[2]);
}

/* central moments (normalised by rho) about velocity u: definition */
static void central_moments(const double* f, double rho, const double u[3], double* m) {
  double px[3][3], py[3][3], pz[3][3];
  for (int c = 0; c < 3; ++c) {
    double dx = (c - 1) - u[0], dy = (c - 1) - u[1], dz = (c - 1) - u[2];
    px[c][0] = 1; px[c][1] = dx; px[c][2] = dx * dx;
    py[c][0] = 1; py[c][1] = dy; py[c][2] = dy * dy;
    pz[c][0] = 1; pz[c][1] = dz; pz[c][2] = dz * dz;
  }
  for (int t = 0; t < 27; ++t) {
    int a = t % 3, b = (t / 3) % 3, c = t / 9;
    double s = 0;
    for (int i = 0; i < 27; ++i)
      s += f[i] * px[CX[i] + 1][a] * py[CY[i] + 1][b] * pz[CZ[i] + 1][c];
    m[t] = s / rho;
  }
}

/* cumulants from central moments by the set-partition formula of joint
   cumulants (the definition behind Geier et al. 2015's cumulants): k_t is
   the sum over partitions of the multiset of t into blocks of size >= 2 of
   (-1)^(b-1) (b-1)! times the product of the blocks' central moments */
static void cum_from_mom(const double* m, double* k) {
  for (int t = 0; t < 27; ++t) {
    double s = 0;
    for (int q = 0; q < NTERMS[t]; ++q) {
      const term* tm = &TERMS[t][q];
      double p = tm->coef;
      for (int b = 0; b < tm->nblk; ++b) p *= m[tm->blk[b]];
      s += p;
    }
    k[t] = s;
  }
}

/* the inverse: central moments as the sum over the same partitions of the
   product of the blocks' cumulants */
static void mom_from_cum(const double* k, double* m) {
  for (int t = 0; t < 27; ++t) {
    double s = 0;
    for (int q = 0; q < NTERMS[t]; ++q) {
      const term* tm = &TERMS[t][q];
      double p = 1;
      for (int b = 0; b < tm->nblk; ++b) p *= k[tm->blk[b]];
      s += p;
    }
    m[t] = s;
  }
}

/* cumulants of one cell's populations (Sec. 2.2 names the cumulant LBM of
   Geier et al. 2015): rho, the mean velocity, then the cumulants of orders
   2 to 6 from the central moments */
void orc_cumulants(const double* f, double* k) {
  orc_init();
  double rho = 0, j[3] = {0, 0, 0};
  for (int i = 0; i < 27; ++i) {
    rho += f[i];
    j[0] += f[i] * CX[i]; j[1] += f[i] * CY[i]; j[2] += f[i] * CZ[i];
  }
  double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
  double m[27];
  central_moments(f, rho, u, m);
  cum_from_mom(m, k);
  k[0] = rho;          /* k_000 slot carries rho */
  k[1] = u[0]; k[3] = u[1]; k[9] = u[2]; /* first cumulants: mean velocity */
}

/* 3x3 inverse by Gauss-Jordan elimination with partial pivoting */
static void inv3(const double A_in[3][3], double X[3][3]) {
  double A[3][6];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 6; ++c) A[r][c] = c < 3 ? A_in[r][c] : (c - 3 == r);
  for (int c = 0; c < 3; ++c) {
    int p = c;
    for (int r = c + 1; r < 3; ++r) if (fabs(A[r][c]) > fabs(A[p][c])) p = r;
    if (p != c) for (int q = 0; q < 6; ++q) { double tmp = A[c][q]; A[c][q] = A[p][q]; A[p][q] = tmp; }
    double piv = A[c][c];
    for (int q = 0; q < 6; ++q) A[c][q] /= piv;
    for (int r = 0; r < 3; ++r)
      if (r != c) {
        double fct = A[r][c];
        for (int q = 0; q < 6; ++q) A[r][q] -= fct * A[c][q];
      }
  }
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) X[r][c] = A[r][c + 3];
}

/* populations from 27 central moments (not normalised) about u */
static void populations_from_central(const double* kap, const double u[3], double* f) {
  double V[3][3][3], I[3][3][3]; /* per axis: V[a][c] = (c-1-u)^a */
  for (int ax = 0; ax < 3; ++ax) {
    for (int c = 0; c < 3; ++c) {
      double d = (c - 1) - u[ax];
      V[ax][0][c] = 1; V[ax][1][c] = d; V[ax][2][c] = d * d;
    }
    inv3((const double(*)[3])V[ax], I[ax]);
  }
  for (int i = 0; i < 27; ++i) {
    double s = 0;
    for (int t = 0; t < 27; ++t) {
      int a = t % 3, b = (t / 3) % 3, c = t / 9;
      s += I[0][CX[i] + 1][a] * I[1][CY[i] + 1][b] * I[2][CZ[i] + 1][c] * kap[t];
    }
    f[i] = s;
  }
}

#define K(a, b, c) k[(a) + 3 * (b) + 9 * (c)]
#define KS(a, b, c) ks[(a) + 3 * (b) + 9 * (c)]

/* Relaxation of the cumulants (Geier et al. 2015): the deviatoric second-order
   cumulants with omega1, their trace with omega2 toward rho c_s^2 (c_s^2 = 1/3),
   third order in the groups (k120 +- k102), (k210 +- k012), (k201 +- k021) with
   omega3 / omega4 and k111 with omega5, fourth order as
   (k220 - 2k202 + k022), (k220 + k202 - 2k022) with omega6, their sum with
   omega7 and k211, k121, k112 with omega8, fifth order with omega9, sixth
   with omega10, all higher equilibria zero.  With `galilean` the diagonal
   second-order relaxation carries the correction for the D3Q27 lattice's
   missing u^3 term, using velocity-gradient estimates from the second-order
   cumulants themselves. */
static void relax(const double* k, double* ks, const double u[3], const orc_rates* r) {
  double w1 = r->omega1, w2 = r->omega2;
  const double* wh = r->omega_hi; /* wh[0] = omega3 ... wh[7] = omega10 */
  memcpy(ks, k, 27 * sizeof(double));
  double dxu = -0.5 * w1 * (2 * K(2,0,0) - K(0,2,0) - K(0,0,2))
               - 0.5 * w2 * (K(2,0,0) + K(0,2,0) + K(0,0,2) - 1.0);
  double dyv = dxu + 1.5 * w1 * (K(2,0,0) - K(0,2,0));
  double dzw = dxu + 1.5 * w1 * (K(2,0,0) - K(0,0,2));
  double g = r->galilean ? 1.0 : 0.0;
  double ux2 = u[0] * u[0], uy2 = u[1] * u[1], uz2 = u[2] * u[2];
  double A = (1 - w1) * (K(2,0,0) - K(0,2,0)) - g * 3 * (1 - 0.5 * w1) * (ux2 * dxu - uy2 * dyv);
  double B = (1 - w1) * (K(2,0,0) - K(0,0,2)) - g * 3 * (1 - 0.5 * w1) * (ux2 * dxu - uz2 * dzw);
  double T = w2 * 1.0 + (1 - w2) * (K(2,0,0) + K(0,2,0) + K(0,0,2))
             - g * 3 * (1 - 0.5 * w2) * (ux2 * dxu + uy2 * dyv + uz2 * dzw);
  KS(2,0,0) = (A + B + T) / 3.0;
  KS(0,2,0) = KS(2,0,0) - A;
  KS(0,0,2) = KS(2,0,0) - B;
  KS(1,1,0) = (1 - w1) * K(1,1,0);
  KS(1,0,1) = (1 - w1) * K(1,0,1);
  KS(0,1,1) = (1 - w1) * K(0,1,1);
  /* third order */
  {
    double w3 = wh[0], w4 = wh[1], w5 = wh[2];
    double p, m;
    p = (1 - w3) * (K(1,2,0) + K(1,0,2)); m = (1 - w4) * (K(1,2,0) - K(1,0,2));
    KS(1,2,0) = 0.5 * (p + m); KS(1,0,2) = 0.5 * (p - m);
    p = (1 - w3) * (K(2,1,0) + K(0,1,2)); m = (1 - w4) * (K(2,1,0) - K(0,1,2));
    KS(2,1,0) = 0.5 * (p + m); KS(0,1,2) = 0.5 * (p - m);
    p = (1 - w3) * (K(2,0,1) + K(0,2,1)); m = (1 - w4) * (K(2,0,1) - K(0,2,1));
    KS(2,0,1) = 0.5 * (p + m); KS(0,2,1) = 0.5 * (p - m);
    KS(1,1,1) = (1 - w5) * K(1,1,1);
  }
  /* fourth order */
  {
    double w6 = wh[3], w7 = wh[4], w8 = wh[5];
    double d1 = (1 - w6) * (K(2,2,0) - 2 * K(2,0,2) + K(0,2,2));
    double d2 = (1 - w6) * (K(2,2,0) + K(2,0,2) - 2 * K(0,2,2));
    double s = (1 - w7) * (K(2,2,0) + K(2,0,2) + K(0,2,2));
    /* solve x - 2y + z = d1, x + y - 2z = d2, x + y + z = s */
    double z = (s - d2) / 3.0;
    double y = (s - d1) / 3.0;
    double x = s - y - z;
    KS(2,2,0) = x; KS(2,0,2) = y; KS(0,2,2) = z;
    KS(2,1,1) = (1 - w8) * K(2,1,1);
    KS(1,2,1) = (1 - w8) * K(1,2,1);
    KS(1,1,2) = (1 - w8) * K(1,1,2);
  }
  KS(2,2,1) = (1 - wh[6]) * K(2,2,1);
  KS(2,1,2) = (1 - wh[6]) * K(2,1,2);
  KS(1,2,2) = (1 - wh[6]) * K(1,2,2);
  KS(2,2,2) = (1 - wh[7]) * K(2,2,2);
}

/* One collision.  `force` (may be NULL) is a body-force density: the
   velocity seen by the relaxation is (j + F/2)/rho and the post-collision
   momentum is j + F. */
void orc_collide(const double* fin, double* fout, const orc_rates* r, const double force[3]) {
  orc_init();
  double rho = 0, j[3] = {0, 0, 0};
  for (int i = 0; i < 27; ++i) {
    rho += fin[i];
    j[0] += fin[i] * CX[i]; j[1] += fin[i] * CY[i]; j[2] += fin[i] * CZ[i];
  }
  double F[3] = {0, 0, 0};
  if (force) { F[0] = force[0]; F[1] = force[1]; F[2] = force[2]; }
  double umean[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
  double uphys[3], upost[3];
  for (int a = 0; a < 3; ++a) {
    uphys[a] = (j[a] + 0.5 * F[a]) / rho;
    upost[a] = (j[a] + F[a]) / rho;
  }
  double m[27], k[27], ks[27], ms[27], kap[27];
  central_moments(fin, rho, umean, m);
  cum_from_mom(m, k);
  relax(k, ks, uphys, r);
  mom_from_cum(ks, ms);
  ms[0] = 1.0; ms[1] = 0.0; ms[3] = 0.0; ms[9] = 0.0;
  for (int t = 0; t < 27; ++t) kap[t] = rho * ms[t];
  populations_from_central(kap, upost, fout);
}
