/*
 * Plain FP64 CPU oracle for the D3Q27 cumulant lattice Boltzmann step on a
 * block-refined mesh around an L-system tree.
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, obviously-correct
 * restatement of the method that the CUDA library is checked against.  Only
 * the test-suite, the smoke check and the CPU-baseline leg of the benchmark
 * load it; the product path never does.  It shares no code, header, table or
 * constant with the CUDA library.
 *
 * Section / equation references are to the paper "Drag Crisis in Fractal
 * Trees Revealed by Simulation and Theory" (Tokiwa, Yin, Onishi):
 *   Sec. 2.1 Eq. (1)  parametric L-system and turtle symbols (Table "symbols")
 *   Sec. 2.1 Table 1/2 tree parameters and derived D0/H, L0/H
 *   Sec. 2.2          D3Q27 cumulant LBM (Geier et al. 2015), octree AMR,
 *                     interpolated bounce-back (Bouzidi et al. 2001),
 *                     momentum-exchange force (Wen et al. 2014)
 *   Sec. 2.3          domain, inflow/outflow, centre of mass placement
 *   Sec. 3 Eq. (7)    C_D = F_D / (1/2 rho U^2 A_x)
 */
#ifndef ORC_H
#define ORC_H
#include <stdint.h>

/* ---------------- tree (Sec. 2.1, Eq. 1) ---------------- */
typedef struct {
  int n;             /* number of rewritings of rule p1: F generations 0..n-1 */
  int children;      /* apices created per application of p1 (paper: 2), <= 4 */
  double s0, w0;     /* axiom A(s0, w0): trunk length and diameter */
  double min_len;    /* rule p1 fires only while s >= min */
  double r[4];       /* length factor per child (r1, r2, ...) */
  double dfac[4];    /* diameter factor per child (paper: q^e and (1-q)^e) */
  double alpha_deg[4]; /* "+" rotation about U, per child */
  double phi_deg[4];   /* "/" rotation about H, per child (azimuth_mode 0) */
  int azimuth_mode;  /* 0: child frame = F * R_U(alpha) * R_H(phi)   (the rule as printed)
                        1: child frame = F * R_H(phi) * R_U(alpha), phi drawn per child
                           uniformly in [0,360) from a SplitMix64 counter stream */
  uint64_t seed;
} orc_tree;

/* segments are rows of 8 doubles: x0 y0 z0 x1 y1 z1 diameter generation */
int orc_lsystem(const orc_tree* t, double* seg, int max_seg);
uint64_t orc_splitmix64(uint64_t seed, uint64_t k);
void orc_tree_bbox(const double* seg, int n, double lo[3], double hi[3]);
double orc_tree_height(const double* seg, int n);
void orc_tree_com(const double* seg, int n, double com[3]);
void orc_transform(double* seg, int n, double scale, const double shift[3]);

/* ---------------- solid primitives ---------------- */
/* kind 0: finite flat-capped cylinder  p[0..7] = x0 y0 z0 x1 y1 z1 D gen
   kind 1: half-space  n.x <= d         p[0..3] = nx ny nz d
   kind 2: axis-aligned box             p[0..5] = lo(3) hi(3)            */
typedef struct { int kind; double p[8]; } orc_prim;
int orc_prim_inside(const orc_prim* pr, int n, const double x[3]);
double orc_prim_ray(const orc_prim* pr, int n, const double x[3], const double d[3]);
double orc_frontal_area(const double* seg, int n, double pitch);

/* ---------------- collision (Sec. 2.2; Geier et al. 2015) ---------------- */
typedef struct {
  double omega1;      /* shear rate 1/(3 nu + 1/2) */
  double omega2;      /* bulk rate */
  double omega_hi[8]; /* omega3 .. omega10 */
  int galilean;       /* 1: include the Galilean-invariance correction of the
                         diagonal second-order cumulants */
} orc_rates;
void orc_init(void);
void orc_equilibrium(double rho, const double u[3], double* feq);
void orc_cumulants(const double* f, double* k);   /* 27 normalised cumulants */
void orc_collide(const double* fin, double* fout, const orc_rates* r, const double force[3]);

/* ---------------- simulation ---------------- */
enum { ORC_BC_PERIODIC = 0, ORC_BC_INOUT = 1, ORC_BC_SLIP = 2, ORC_BC_INFLOW = 3 };
typedef struct {
  int levels;              /* 1..6 */
  int nx, ny, nz;          /* level-0 cells */
  int box[6][6];           /* for l>=1: real region R_l in level-l cells: lo xyz, hi xyz (exclusive) */
  int bc[3];               /* per axis, ORC_BC_* (x: periodic or in/out) */
  double u_in;             /* inlet velocity along +x, lattice units */
  double nu0;              /* level-0 lattice kinematic viscosity */
  double omega2;
  double omega_hi[8];
  int galilean;
  double force[3];         /* body force density (single-level runs only) */
} orc_desc;

typedef struct orc_sim orc_sim;
orc_sim* orc_create(const orc_desc* d);
void orc_destroy(orc_sim* s);
/* solid primitives in finest-level cell units; classifies every level and builds links */
int orc_set_prims(orc_sim* s, const orc_prim* pr, int n);
void orc_init_uniform(orc_sim* s, double rho, const double u[3]);
/* per-cell equilibrium initialisation of one level from rho[n], u[3n] over its real box */
int orc_init_field(orc_sim* s, int level, const double* rho, const double* u);
void orc_step(orc_sim* s, int ncoarse);
/* turbulent inflow: n modes of 7 doubles (k, a, psi), mean speed u_in */
int orc_set_turbulence(orc_sim* s, const double* modes, int n, double u_in);
/* real box of a level and its populations f_i(x) (NaN for non-fluid cells), x fastest */
void orc_level_box(const orc_sim* s, int level, int lo[3], int hi[3]);
void orc_get_f(const orc_sim* s, int level, double* out);
void orc_get_macro(const orc_sim* s, int level, double* rho, double* u);
int orc_level_links(const orc_sim* s, int level, long* cell, int* dir, double* q, int max);
int orc_level_link_segs(const orc_sim* s, int level, int* seg, int max);
void orc_force(const orc_sim* s, double last[3], double sum[3], long* nsum);
void orc_mass(const orc_sim* s, double* mass, double mom[3]);
int orc_cell_type(const orc_sim* s, int level, unsigned char* out);
int orc_branch_forces(const orc_sim* s, double* mean, int n);

/* host threads of the OpenMP loops (n >= 1); returns the previous count */
int orc_set_threads(int n);

#endif
