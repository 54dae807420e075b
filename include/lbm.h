/*
 * liblbm: D3Q27 cumulant lattice Boltzmann time step on a block-refined mesh
 * around an L-system tree, with interpolated bounce-back on the branches and
 * the momentum-exchange drag, for NVIDIA GB300 (sm_103a).
 *
 * Paper: Tokiwa, Yin & Onishi, "Drag Crisis in Fractal Trees Revealed by
 * Simulation and Theory".  Section references below are to that paper.
 *
 * Conventions common to every call
 *  - Every call returns an lbm_status (0 on success, a negative code on
 *    failure); no call aborts or throws across this boundary: a host
 *    allocation that fails inside the library returns LBM_ENOMEM, any other
 *    internal C++ exception LBM_ESTATE, each with its message.
 *  - Lattice units throughout: lengths in cells of the level named, the
 *    inflow speed in cells per time step, density 1 at rest.  "Finest
 *    cells" are cells of the finest refinement level.
 *  - Population index i = (cx+1) + 3 (cy+1) + 9 (cz+1) for the D3Q27
 *    velocity c_i = (cx, cy, cz), cx, cy, cz in {-1, 0, 1}; the opposite
 *    direction is 26 - i.
 *  - Host arrays of a level's cells are ordered x fastest, then y, then z,
 *    over that level's real box (lbm_level_info).
 *  - The caller owns every host buffer and the device buffer it binds
 *    (lbm_bind_memory); the domain owns its host-side metadata only.  The
 *    library never allocates device memory: all device state lives in the
 *    bound buffer.
 *  - Calls on one domain are not thread-safe.  Device work is issued
 *    asynchronously on the stream given to lbm_create_domain; calls that
 *    return device results to the host synchronise that stream.
 */
#ifndef LBM_H
#define LBM_H
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_domain lbm_domain; /* opaque, owned by the library */

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = -1,    /* an argument or descriptor field is out of range */
  LBM_ENOMEM = -2,    /* host allocation failed or the bound buffer is too small */
  LBM_ECUDA = -3,     /* a CUDA runtime call failed (message: lbm_last_error) */
  LBM_EUNSTABLE = -4, /* the watchdog found NaN/Inf or a density outside [0.5, 2] */
  LBM_ESTATE = -5,    /* call out of order (e.g. stepping before binding memory), or an
                         internal error (lbm_last_error says which) */
  LBM_ETIMEOUT = -6   /* reserved: a bounded device wait gave up */
} lbm_status;

typedef enum {
  LBM_BC_PERIODIC = 0, /* wrap around */
  LBM_BC_INOUT = 1,    /* x only: uniform inflow at x = 0, zero-gradient outflow at x = nx (Sec. 2.3) */
  LBM_BC_SLIP = 2,     /* specular reflection (free slip) */
  LBM_BC_INFLOW = 3    /* y, z: equilibrium at rho = 1 and the inflow velocity (Sec. 2.3: inflow on all non-outlet faces) */
} lbm_bc;

/* Population storage.  LBM_FP64: f_i - w_i in FP64 with FP64 collision and
   bounce-back arithmetic (FP64 wall fractions q): the method in double
   precision, as the paper's smallest workload states it; a reference and
   validation form (GB300's FP64 rate is a small fraction of its FP32 rate,
   so its one collide kernel per parity is arithmetic-bound; no turbulent
   inflow, no batches).  LBM_FP32: f_i - w_i in FP32.  LBM_FP16_DEV:
   (f_i - f_i^eq(1, U e_x)) * 2^13 in IEEE binary16, deviations from the
   inflow equilibrium at the inflow speed U (the power-of-two scale is per
   level).  Collision arithmetic is FP32 in both reduced forms; the drag and
   mass reductions and the interface ledger are FP64 in every form.
   lbm_get_populations returns f_i in every form. */
typedef enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_FP16_DEV = 2 } lbm_precision;

/* Collide-kernel variants (all compute the same result; within the FP16 form
   the packed two-cell kernels and the one-cell ones differ in the last bit of
   FP32 rounding).  Odd AA step: per-thread column pointers, TMA/cp.async
   staging through shared memory (FP32 and 16^3 blocks only; others fall back
   to column pointers), direct neighbour addressing, or two x-neighbouring
   cells per thread collided as one in packed FP32.  Even step: direct loads
   and stores, a 4-stage TMA bulk pipeline (FP32 and 16^3 blocks only), or two
   x-neighbouring cells per thread moved with pair loads and stores (4 bytes
   in FP16, 8 in FP32) and collided as one in packed FP32 (the FP16 direct
   even step runs the same packed code in both lanes and equals it bit for
   bit).  Defaults: column pointers and the direct even step for FP32, pairs
   in both steps for FP16; lbm_autotune measures all of them. */
typedef enum {
  LBM_ODD_COLUMNS = 0,
  LBM_ODD_STAGED = 1,
  LBM_ODD_DIRECT = 2,
  LBM_ODD_PAIRS = 3,   /* registers budgeted for 6 resident CTAs per SM */
  LBM_ODD_PAIRS_7 = 4, /* the same kernel budgeted for 7 (72 registers, a few spills; 16^3 blocks) */
  LBM_ODD_PAIRS_8 = 5  /* ... for 8 (64 registers, more spills; 16^3 blocks) */
} lbm_odd_variant;
typedef enum { LBM_EVEN_DIRECT = 0, LBM_EVEN_TMA = 1, LBM_EVEN_PAIRS = 2 } lbm_even_variant;

/* Problem statement (Sec. 2.2-2.3): domain, inflow, Re_H, refinement.
   Coarse level = level 0; every finer level halves the cell size and the
   time step (acoustic scaling, nu_{l+1} = 2 nu_l in lattice units). */
typedef struct {
  int nx, ny, nz;          /* level-0 cells; periodic axes must be multiples of block */
  int levels;              /* 1..6 refinement levels */
  int block;               /* cells per block edge: 8 or 16 */
  int bc[3];               /* lbm_bc per axis; x is PERIODIC or INOUT, y/z are PERIODIC, SLIP or INFLOW */
  double u_in;             /* inflow speed U along +x, lattice units (0 < U < 0.3) */
  double re_h;             /* Re_H = U H / nu on the finest level, H = tree height in finest cells;
                              <= 0 selects nu_finest below */
  double nu_finest;        /* finest-level lattice viscosity when re_h <= 0 */
  double i_u;              /* inflow turbulence intensity u'_rms / U in [0, 0.5]; 0: uniform inflow,
                              > 0: random-Fourier-mode inflow (lbm_set_inflow_turbulence) */
  unsigned long long seed; /* reserved for seeded inflow turbulence */
  double refine_margin;    /* finest box = tree bounding box grown by this fraction per side (0.25) */
  int precision;           /* lbm_precision */
  int galilean;            /* 1: Galilean correction of the diagonal second-order cumulants */
  double omega2;           /* bulk relaxation rate (1) */
  int boxes[6][6];         /* optional refinement boxes R_l (l >= 1) in level-l cells,
                              lo xyz then hi xyz (exclusive); all zero: derived from the tree */
} lbm_domain_desc;

/* Parametric L-system of Eq. (1), Sec. 2.1.  n rewritings of rule p1 draw
   branch generations 0..n-1.  Child k of a branch gets length s * r[k],
   diameter w * dfac[k] (the paper: q^e and (1-q)^e), and a frame rotated
   by "+"(alpha[k]) about U and "/"(phi[k]) about H.  azimuth_mode 0 applies
   + then / with the fixed phi[k]; azimuth_mode 1 applies / then + with phi
   drawn uniformly in [0, 360) degrees from SplitMix64(seed) at counter
   (index of the parent branch in drawing order) * children + k.  The trunk
   points along +z.  The tree is scaled so the trunk is trunk_cells finest
   cells long and its volume centroid is placed at (Lx/4, Ly/2, Lz/2) of the
   domain (Sec. 2.3). */
typedef struct {
  int n;
  int children;            /* 1..4 */
  double s0, w0;           /* axiom A(s0, w0) */
  double min_len;          /* rule p1 applies while s >= min */
  double r[4], dfac[4], alpha_deg[4], phi_deg[4];
  int azimuth_mode;
  unsigned long long seed;
  double trunk_cells;
} lbm_tree_desc;

/* Create a domain (host metadata only; no device work).  cuda_stream is a
   cudaStream_t (NULL = legacy default stream).  *out receives the handle. */
int lbm_create_domain(const lbm_domain_desc* desc, void* cuda_stream, lbm_domain** out);

/* Build the tree of Eq. (1), place it, derive the refinement boxes (unless
   given), classify the cells of every level and build the cut-link lists
   with their wall fractions q (Sec. 2.2, interpolated bounce-back).  Must
   precede lbm_memory_requirements.  Host only. */
int lbm_set_geometry(lbm_domain* d, const lbm_tree_desc* tree);

/* As lbm_set_geometry, from ready segments: n rows of 8 doubles
   x0 y0 z0 x1 y1 z1 diameter generation, in finest cells, already placed. */
int lbm_set_geometry_segments(lbm_domain* d, const double* seg, int n);

/* General solid primitives in finest cells: kind[k] 0 = flat-capped
   cylinder (params x0 y0 z0 x1 y1 z1 D -), 1 = half-space n.x <= d
   (nx ny nz d), 2 = axis-aligned box (lo xyz, hi xyz); params n x 8.
   A cell is solid when its centre lies in any primitive.  n = 0: no solid. */
int lbm_set_geometry_prims(lbm_domain* d, const int* kind, const double* params, int n);

/* Bytes of device memory the domain needs (populations, tables, scratch). */
int lbm_memory_requirements(const lbm_domain* d, size_t* bytes);

/* What the bound buffer holds and what binding copies: *populations the
   bytes of population storage of all levels (active and ghost blocks),
   *uploaded the host-to-device bytes one lbm_bind_memory copies (boundary,
   interface and neighbour tables in the form the device uses, turbulence
   modes, the step counter; the populations are initialised on the device).
   Either pointer may be NULL.  Needs the geometry; host only. */
int lbm_memory_breakdown(const lbm_domain* d, size_t* populations, size_t* uploaded);

/* Bind a caller-owned device buffer of at least the required size (256-byte
   aligned), upload the tables and set every population to the inflow
   equilibrium.  The buffer must stay valid until lbm_destroy. */
int lbm_bind_memory(lbm_domain* d, void* device_ptr, size_t bytes);

/* Equilibrium state rho, u on every level (resets the force history). */
int lbm_init_uniform(lbm_domain* d, double rho, const double u[3]);

/* Equilibrium state from host fields over one level's real box:
   rho[n], u[3n] (x fastest); n must equal the box's cell count. */
int lbm_init_field(lbm_domain* d, int level, const double* rho, const double* u, size_t n);

/* The method's time step (Sec. 2.2: the cumulant LBM on the octree-refined
   mesh, interpolated bounce-back on the tree and the momentum-exchange
   force; Sec. 2.3: the inflow, outflow and lateral faces): advance n coarse
   steps, every level l taking 2^l steps of its own (recursive sub-cycling,
   acoustic scaling), asynchronously on the domain's stream (captured CUDA
   graphs - runs of eight and of two coarse steps while that many remain and
   no transfer is pending, else one per coarse step - unless graphs are off
   or timing is on; the results are the same either way).
   LBM_ESTATE before lbm_bind_memory; returns the status of the last
   watchdog check (lbm_set_watchdog), LBM_EUNSTABLE if it failed. */
int lbm_step(lbm_domain* d, int n_coarse);

/* Momentum-exchange force on the tree (Sec. 2.2, Wen et al. 2014) in
   finest-level lattice units: force_last of the last finest step and
   force_mean averaged over the finest steps since the last init or
   lbm_reset_force; c_d = force_last[0] / (1/2 U^2 A_x) (Eq. 7, rho = 1,
   A_x in finest cells^2).  Any pointer may be NULL.  Synchronises.
   lbm_reset_force also clears the interface ledger (lbm_interface_ledger). */
int lbm_drag(lbm_domain* d, double force_last[3], double force_mean[3], double* c_d);
/* The same without synchronising: enqueues on the domain's stream a copy of
   the 8 force accumulators (force of the last finest step [3], their sum over
   the finest steps [3], the number of those steps, and a status word that
   is nonzero when a bounded device wait gave up) to host_acc, which the
   caller owns (page-locked for the copy to overlap later work) and may read
   once the stream has passed this point; lbm_drag_decode turns them into
   lbm_drag's outputs (LBM_ETIMEOUT for a nonzero status). */
int lbm_drag_enqueue(lbm_domain* d, double host_acc[8]);
int lbm_drag_decode(const lbm_domain* d, const double acc[8], double force_last[3], double force_mean[3],
                    double* c_d);
int lbm_reset_force(lbm_domain* d);

/* Populations f_i(x) of one level's real box (27 per cell, NaN for cells
   that are not fluid), at the current coarse-step boundary.  Synchronises. */
int lbm_get_populations(lbm_domain* d, int level, double* f, size_t n_cells);

/* lbm_get_populations for the window [lo, hi) of a level's real box (cell
   coordinates counted from the box's first cell, x fastest in f), reading
   only the stored elements that window's fluid cells hold, so a small window
   of a level too large to copy whole costs little; f holds 27 values per
   cell (NaN for cells that are not fluid).  n_cells must equal the window's
   cell count; an empty window or one reaching outside the box gives
   LBM_EINVAL.  Synchronises. */
int lbm_get_populations_window(lbm_domain* d, int level, const int lo[3], const int hi[3], double* f,
                               size_t n_cells);

/* Density and velocity per cell of one level's real box (NaN: not fluid). */
int lbm_get_velocity(lbm_domain* d, int level, double* rho, double* u, size_t n_cells);

/* Volume-weighted total mass and momentum of all levels, FP64 on device
   (level-l cells weigh 8^-l).  Synchronises. */
int lbm_mass(lbm_domain* d, double* mass, double mom[3]);

/* lbm_mass without any caller-provided scratch.  (The paper has no
   counterpart; this is a service of the library.)  Same result and contract
   as lbm_mass, but the per-block partial sums go to a fixed scratch array
   inside the library image instead of the domain's bound buffer, and the
   call performs no device allocation of any kind (no cudaMalloc, no
   allocating library routine).  It is for callers that may not allocate
   device memory at the point of the call - code running under an allocator
   or memory pool that forbids growth, or a monitor that must not disturb
   the memory the caller has budgeted - and for callers that want the check
   without touching the domain's own scratch.
   Limits and rules: every level may hold at most 32768 active blocks
   (LBM_EINVAL otherwise); the scratch (about 1.3 MB per GPU that loads the
   library) is held until the process exits; the domain's device must be
   current; the first call on each device looks up the scratch address with
   that device current (once, race-free across host threads); all calls
   share the one scratch array, so calls whose device work overlaps race and
   must be serialised by the caller.  The call copies its totals to host
   memory and synchronises the domain's stream before it returns. */
int lbm_mass_noalloc(lbm_domain* d, double* mass, double mom[3]);

/* Mass and momentum of one level (as lbm_mass: FP64 on device, level-l
   cells weigh 8^-l).  Synchronises. */
int lbm_level_mass(lbm_domain* d, int level, double* mass, double mom[3]);

/* FP64 ledger of the refinement interface between `level` and level + 1
   (Sec. 2.2's octree refinement; the volumetric transfer between the
   levels).  Every coarse step the interface kernels record, as exact 64-bit
   fixed-point sums reported in FP64, twelve values - mass and momentum
   (x, y, z) of three flows, in level-0 cell volumes (a level-l cell weighs
   8^-l), full populations f_i:
     [0..3]  In:    coarse post-collision values handed to the fine level
                    (the explode and inflow transfers)
     [4..7]  OutF:  fine values the coalesce transfer takes from the fine
                    level
     [8..11] RecvC: what the coarse cells next to the fine region receive
                    (8 x the stored coalesce result minus the part it keeps
                    from the coarse cell itself)
   so that over any stretch of steps, up to the rounding of the collisions,
   the fine level's mass and momentum change by In - OutF and the coarse
   level's by RecvC - In (plus the flows of its own coarser interface, and
   nothing else in a closed box); RecvC - OutF is the interface's rounding
   defect.
   The interface kernels run once per step of the coarser level, so `last`
   holds the flows of the last step of `level` (one coarse step for level 0,
   half of one for level 1, ...) and *steps counts those steps; total: the
   sum since binding, lbm_init_uniform or lbm_reset_force (which clear the
   ledger).  Resolution: every recorded population deviation is rounded to
   a multiple of 2^-40 (exact for binary16 storage; at most 2^-41 per entry
   in FP32 and FP64), and the sums themselves are exact and independent of
   the order of the threads.
   The ledger is on by default; lbm_set_interface_ledger(d, 0) drops its
   sums from the interface kernels (toggling recaptures the graphs and clears
   the ledger).  LBM_EINVAL for the finest level.  Synchronises. */
int lbm_set_interface_ledger(lbm_domain* d, int on);
int lbm_interface_ledger(lbm_domain* d, int level, double last[12], double total[12], long long* steps);

/* Real box [lo, hi) of a level in level-l cells, and cell counts. */
int lbm_level_info(const lbm_domain* d, int level, int lo[3], int hi[3], long long* n_fluid,
                   long long* n_links, long long* n_active_blocks);

/* Tree height H and frontal area A_x (finest cells), finest viscosity. */
int lbm_geometry_info(const lbm_domain* d, double* height, double* frontal_area, int* n_segments,
                      double* nu_finest);

/* Cell type per cell of a level's real box: 0 fluid, 1 solid, 2 covered by
   the next finer level. */
int lbm_get_cell_types(const lbm_domain* d, int level, unsigned char* out, size_t n_cells);

/* Cut links of a level: cell (linear index over the real box), direction
   and wall fraction q; n is the capacity, *count the number of links. */
int lbm_get_links(const lbm_domain* d, int level, long long* cell, int* dir, double* q, size_t n,
                  long long* count);

/* The branch (primitive index) each cut link of a level belongs to - the
   cylinder its ray from the fluid cell enters first - in the order of
   lbm_get_links; n is the capacity, *count the number of links.  This is
   the attribution behind the per-branch forces (Sec. 2.4). */
int lbm_get_link_branches(const lbm_domain* d, int level, int* branch, size_t n, long long* count);

/* Placed segments (rows of 8 doubles) of the tree; n capacity. */
int lbm_get_segments(const lbm_domain* d, double* seg, int n, int* count);

/* Per-branch momentum-exchange forces (Sec. 2.4's branch-wise view of the
   tree, measured by the LBM).  Every cut link belongs to the cylinder (or
   primitive) its ray enters first; with branch forces on, every finest step
   adds each branch's force to a running FP64 sum (deterministic order).
   lbm_get_branch_forces returns, for the n >= number of branches, the mean
   force per branch since the last lbm_reset_force / init (finest-level
   lattice units, rows x y z) and the number of steps averaged.  Per link the
   rest state (rho = 1, u = 0) is subtracted, c_i (f*_i + f_ibar - 2 w_i):
   one branch's links do not close a surface, so the uniform reference
   pressure would otherwise enter its force.  Over all cut links of a finite
   solid sum c_i w_i = 0, so the sum over branches still equals the total of
   lbm_drag (up to rounding).  Toggling recaptures the graphs. */
int lbm_set_branch_forces(lbm_domain* d, int on);
int lbm_get_branch_forces(lbm_domain* d, double* mean_xyz, int n, long long* steps);

/* Branch-wise description of the tree for the analytical model (Sec. 2.4,
   Eq. 2: F_d = C_d (1/2 rho U^2) L D sin^3(alpha)) and its learned sectional
   drag: one row of LBM_BRANCH_COLS doubles per branch, in lbm_get_segments
   order:
     0 log10 Re_d (U D / nu, finest level)   1 generation   2 D/H
     3 cos(alpha), alpha in [0, pi] the angle between the flow and the axis
       drawn from the branch's base to its tip
     4 inflow turbulence intensity
     5 shielding depth: mean number of other branches that the stream-wise
       lines through 16 points of the axis enter upstream of the point
     6 L   7 D (finest cells)   8 sin^3(alpha)
     9 shadowed fraction: of 16 axial x 5 lateral points spread over the
       branch's projected width (offsets -0.4 D .. 0.4 D normal to the axis
       and the flow), those whose stream-wise line enters another branch
       more than D/2 upstream
    10 leaf: 1 if no other branch starts at this branch's tip, else 0
   n is the capacity in rows, *count the number of branches. */
#define LBM_BRANCH_COLS 11
int lbm_branch_table(const lbm_domain* d, double* rows, int n, int* count);

/* Branch-wise drag estimate (Sec. 2.4, Eq. 2 summed as in Eq. 4): with
   c_k = F_d,k / (rho U^2 L_k D_k / 2) the sectional drag coefficient of
   branch k, C_D-est = sum_k c_k L_k D_k / A_x.  rows: n rows of
   lbm_branch_table (host, LBM_BRANCH_COLS doubles each); c_sect: host array of n c_k, or
   NULL for the cylinder law c_k = C_d(Re_d,k) sin^3(alpha_k) with
   C_d(Re) = 1 + 10 Re^(-2/3) (White's cross-flow cylinder correlation,
   standing in for the paper's fit to measurements); area: A_x in the same
   length unit as L and D.  Writes *cd_est and, if c_out is not NULL, the n
   coefficients used.  Host arithmetic, no device work; LBM_EINVAL for null
   pointers, n < 0 or area <= 0. */
int lbm_branch_drag_estimate(const double* rows, int n, const double* c_sect, double area, double* cd_est,
                             double* c_out);

/* The measured sectional coefficients of Eqs. 2 and 3 (Sec. 2.4), rho = 1:
   c_drag[k] = mean F_x,k / (U^2 L_k D_k / 2) from the per-branch forces
   averaged since the last lbm_reset_force (lbm_set_branch_forces must be on),
   c_fric[k] the same from the per-branch friction means
   (lbm_set_friction_mean; zeros while it is off); *cd = mean F_x /
   (U^2 A_x / 2) over the same window (Eq. 7), *cf the friction's (Eq. 8; NaN while
   the friction mean is off).  Any pointer may be NULL; n is the capacity
   in branches.  Host arithmetic after reading the device sums; synchronises. */
int lbm_branch_coefficients(lbm_domain* d, double* c_drag, double* c_fric, int n, double* cd, double* cf);

/* ---- Friction and pressure drag (Sec. 3: C_F from the wall shear stress
   integrated over the tree surface, C_P = C_D - C_F) ----
   The surface of every primitive is covered by quadrature points (spacing
   1/2 finest cell; cylinders: lateral lines and end-cap rings; half-spaces:
   a grid over the finest level; points inside another primitive dropped).
   A cell's viscous stress is sigma' = -(1 - omega1/2) dev(sum_i c_i c_i
   (f_i - f_i^eq)) from its pre-collision populations at the step boundary;
   at a point it is extrapolated linearly to the wall from two fluid cells
   along the normal (A: the finest-level cell containing x + delta n for the
   first delta in {1, 1.5, 2} that is fluid; B: the cell containing
   x + (delta + 1) n if fluid and at least 1/4 cell farther out, else A
   alone).  The tangential traction (sigma' n minus its normal part) times
   the point's area is its friction force; sums are FP64, fixed order.
   lbm_friction: the friction force of the current state (finest-level
   lattice units), per branch if per_branch (n rows of 3) is given, and
   C_F = F_x / (1/2 U^2 A_x).  Synchronises.
   lbm_set_friction_mean: also accumulate it after every coarse step;
   lbm_get_friction_mean returns the mean since the last lbm_reset_force and
   the number of coarse steps averaged.  Toggling recaptures the graphs.
   lbm_friction_samples: 13 doubles per point - cell A (x y z), cell B
   (x y z, -1e9 when absent), n (3), area, the two normal distances (0 for
   absent B), branch; n is the capacity in points. */
int lbm_friction(lbm_domain* d, double force[3], double* per_branch, int n, double* c_f);
int lbm_set_friction_mean(lbm_domain* d, int on);
int lbm_get_friction_mean(lbm_domain* d, double mean[3], double* per_branch, int n, long long* steps);
int lbm_friction_samples(const lbm_domain* d, double* rows, int n, int* count);

/* ---- Sectional-drag surrogate (a learned C_d for Eq. 2, Sec. 2.4) ----
   A fully connected network: n_in inputs, `hidden` layers of `width` GELU
   units, one output; BF16 weights with FP32 accumulation in its forward and
   backward kernels, FP32 master weights and Adam (beta 0.9 / 0.999, eps 1e-8)
   moments, deterministic reductions.  The paper fits its cylinder drag law
   to measured data instead; this learned law is trained on per-branch forces
   that the LBM measures (lbm_get_branch_forces, lbm_branch_table).
   Parameters are one flat FP32 vector: per layer W (out x in, row-major) then
   the bias.  Inputs are standardised with (x - mu_x) / sd_x and the target
   with (y - mu_y) / sd_y (lbm_mlp_set_normalization); the loss is the mean
   squared error of the standardised output.  x is batch x n_in FP32, y and
   the optional idx (rows of x and y to use, int32) have batch entries; all
   are device pointers.  The caller binds one device buffer of
   lbm_mlp_memory_requirements bytes for a maximum batch. */
typedef struct lbm_mlp lbm_mlp;
int lbm_mlp_create(int n_in, int width, int hidden, void* cuda_stream, lbm_mlp** out);
int lbm_mlp_memory_requirements(const lbm_mlp* m, int max_batch, size_t* bytes);
int lbm_mlp_bind_memory(lbm_mlp* m, void* device_ptr, size_t bytes, int max_batch);
int lbm_mlp_param_count(const lbm_mlp* m, long long* n);
/* set / read the FP32 master parameters (host arrays); set resets Adam */
int lbm_mlp_set_params(lbm_mlp* m, const float* host, long long n);
int lbm_mlp_get_params(lbm_mlp* m, float* host, long long n);
int lbm_mlp_set_normalization(lbm_mlp* m, const float* mu_x, const float* sd_x, float mu_y, float sd_y);
/* y[b] = prediction (de-standardised) for x[b]; asynchronous */
int lbm_mlp_forward(lbm_mlp* m, const float* x, int batch, float* y);
/* y[b] = the mean prediction of n networks (an ensemble trained from
   different seeds) for x[b]: every member's forward pass and the running
   mean on the device, asynchronously.  Members must share n_in and the
   stream and have capacity for the batch. */
int lbm_mlp_ensemble_forward(lbm_mlp* const* nets, int n, const float* x, int batch, float* y);
/* loss and the gradient of the loss with respect to the parameters (host
   array of lbm_mlp_param_count floats, may be NULL); synchronises */
int lbm_mlp_gradients(lbm_mlp* m, const float* x, const float* y, const int* idx, int batch, float* grad_host,
                      double* loss);
/* one Adam step at learning rate lr; loss may be NULL (no synchronisation) */
int lbm_mlp_train_step(lbm_mlp* m, const float* x, const float* y, const int* idx, int batch, float lr,
                       double* loss);
const char* lbm_mlp_last_error(void);
void lbm_mlp_destroy(lbm_mlp* m);

/* Turbulent inflow (domains with i_u > 0; Sec. 4.2 defines I_u = u'_rms / U).
   Every inflow-equilibrium value pulled from outside level 0 is the
   equilibrium at rho = 1 and u = U e_x + u'(p - U t e_x) at the centre p of
   the cell it is pulled from, t the coarse steps done: a frozen synthetic
   field carried through the inflow at U (Taylor's hypothesis).
     u'(x) = sum_n a_n cos(k_n . x + psi_n),   a_n . k_n = 0,
   n_modes modes (default 256) with a von Karman spectrum whose integral
   length is `integral_length` level-0 cells (0: the tree height), scaled so
   that the expected stream-wise variance is (I_u U)^2; directions, phases
   and polarisations come from SplitMix64 draws of the domain's seed
   (counter 2^40 + 4 n + j).  Lengths and wavenumbers in level-0 cells;
   wavenumbers log-spaced over [k_e / 4, min(16 k_e, pi / 4)], k_e =
   0.747 / integral_length.  n_modes at most 1024.  LBM_ESTATE when i_u = 0. */
int lbm_set_inflow_turbulence(lbm_domain* d, int n_modes, double integral_length);
/* The mode table, 7 doubles per mode: k (3), a (3), psi; n is the capacity
   in modes, *count the number of modes (0 for uniform inflow). */
int lbm_inflow_modes(const lbm_domain* d, double* modes, int n, int* count);

/* ---- Schedules, autotuning and batches ----
   A schedule picks the collide-kernel variants and, for batches, the size of
   the persistent grid (ctas_per_sm CTAs per SM, 0: one CTA per block).
   lbm_autotune and lbm_batch_autotune time every available candidate for
   `steps` coarse steps (after one untimed step each) with CUDA events and
   keep the fastest; they advance the simulation by the steps they time, so
   re-initialise (lbm_init_uniform) before a production run.  lbm_autotune
   then times a few masks of lbm_set_overlap_features under the chosen
   schedule (overlap and graphs on; at least 16 steps each, twice) and leaves
   the fastest set (lbm_get_overlap_features reports it). */
typedef struct {
  int ctas_per_sm;   /* batches only; ignored by single domains */
  int odd_variant;   /* lbm_odd_variant */
  int even_variant;  /* lbm_even_variant */
  int z_split_even;  /* CTAs (or persistent-grid work units) per active block of the even step: */
  int z_split_odd;   /*   1, 2, 4 ... up to the block size, each walking block/z_split slabs
                        (results are identical for every split).  0 = automatic, per launch:
                        8 for FP32 and for the FP16 odd step in 16^3 blocks; for the FP16 even
                        step the fewest that give the launch at least 32 CTAs per SM (at most
                        8); 1 for 8^3 blocks.
                        Ignored by the staged and TMA variants. */
} lbm_schedule;
int lbm_set_schedule(lbm_domain* d, const lbm_schedule* s);
int lbm_get_schedule(const lbm_domain* d, lbm_schedule* s);
int lbm_autotune(lbm_domain* d, int steps, lbm_schedule* best, double* ms_per_step);

/* A batch steps several independent domains (bound, same block size and
   precision, same step parity) in lockstep: per level depth and sub-step
   ONE persistent collide launch walks a work list of (level, block) pairs of
   every domain that has that level, the per-domain boundary, force and
   interface kernels follow on the batch's stream, and each coarse step of
   the whole batch is one CUDA graph launch.  Results are identical to
   stepping each domain alone.  The batch binds its own small device buffer
   (descriptors and work lists).  Batches take the column-pointer, direct or
   paired (two cells per thread, 6 CTAs per SM) odd step and the direct or
   paired even step; lbm_batch_autotune times every combination at one CTA
   per work unit, then persistent grids for the best, then the z splits.
   FP32 or FP16 storage.  The domains must outlive the batch and must not
   be stepped on their own while they are in it. */
typedef struct lbm_batch lbm_batch;
int lbm_batch_create(lbm_domain* const* domains, int n, void* cuda_stream, lbm_batch** out);
int lbm_batch_memory_requirements(const lbm_batch* b, size_t* bytes);
int lbm_batch_bind_memory(lbm_batch* b, void* device_ptr, size_t bytes);
int lbm_batch_set_schedule(lbm_batch* b, const lbm_schedule* s);
int lbm_batch_get_schedule(const lbm_batch* b, lbm_schedule* s);
int lbm_batch_step(lbm_batch* b, int n_coarse_steps);
int lbm_batch_use_graphs(lbm_batch* b, int on);
int lbm_batch_autotune(lbm_batch* b, int steps, lbm_schedule* best, double* ms_per_step);
void lbm_batch_destroy(lbm_batch* b);

/* Run the collide kernels with 64-bit element offsets even on levels whose
   arrays hold fewer than 2^31 elements (they switch to 64-bit offsets by
   themselves above that), so that small cases exercise the large-array
   code; results are identical.  Toggling recaptures the graphs. */
int lbm_set_wide_offsets(lbm_domain* d, int on);

/* Run the level-0 face kernel and the wall kernels as parallel branches of
   the step (side streams; parallel graph branches) wherever a host check at
   lbm_set_geometry found that no slot they write is read or written by the
   kernels they run beside, and no slot they read is written by them
   (default on).  Results are identical either way.  Toggling recaptures the
   graphs. */
int lbm_set_overlap(lbm_domain* d, int on);

/* The reorderings lbm_set_overlap switches on, each separately (all by
   default).  Every one reorders the same launches over the domain's stream
   and side streams where the host check, or the slot rules of the AA
   update, show that the kernels it places side by side touch disjoint
   slots; results are identical under every mask.
   LBM_OVL_BRANCHES: level-0 faces and wall kernels as parallel branches.
   LBM_OVL_LEVELS: a level without cut links runs its collide, faces and
     (with LBM_OVL_TRANSFERS) explode transfer beside the finer level's
     first sub-step.
   LBM_OVL_TRANSFERS: the save and inflow transfers beside the finer
     level's second sub-step (when the finer level's walls touch none of
     their slots).
   LBM_OVL_DEFER: a level's coalesce transfer at the head of its next step
     (lbm_step runs the pending ones before it returns).
   LBM_OVL_WALL_SPLIT: the finest level's second sub-step updates the
     blocks its first sub-step's walls do not touch before those walls
     finish (two launches).
   Default: LBM_OVL_BRANCHES | LBM_OVL_LEVELS | LBM_OVL_TRANSFERS;
   lbm_autotune also tries masks with the other two and keeps the fastest.
   Unknown bits give LBM_EINVAL.  Changing the mask recaptures the graphs. */
enum {
  LBM_OVL_BRANCHES = 1,
  LBM_OVL_LEVELS = 2,
  LBM_OVL_TRANSFERS = 4,
  LBM_OVL_DEFER = 8,
  LBM_OVL_WALL_SPLIT = 16,
  LBM_OVL_ALL = 31
};
int lbm_set_overlap_features(lbm_domain* d, int mask);
int lbm_get_overlap_features(const lbm_domain* d, int* mask);
/* What that check found: *faces = 1 if the level-0 faces may run as a
   branch; bit l of *walls set if the walls of level l may.  Either pointer
   may be NULL.  Needs lbm_set_geometry; no device work. */
int lbm_get_overlap(const lbm_domain* d, int* faces, int* walls);

/* Every `every` coarse steps lbm_step checks for NaN/Inf and densities
   outside [0.5, 2] (synchronising); 0 disables (default). */
int lbm_set_watchdog(lbm_domain* d, int every);

/* 1: replay one captured CUDA graph per coarse step (default); 0: launch
   the kernels directly. */
int lbm_use_graphs(lbm_domain* d, int on);

/* Kernel timing with CUDA events on the domain's stream (adds no
   synchronisation inside lbm_step; graphs are bypassed while on).
   lbm_get_timing returns, per kernel class k (0 collide-stream even steps,
   1 collide-stream odd steps, 2 faces, 3 bounce-back + force, 4 interface,
   5 unused), the summed milliseconds, the number of launches and the cell
   updates / links / entries processed since the last call.  Synchronises. */
int lbm_set_timing(lbm_domain* d, int on);
int lbm_get_timing(lbm_domain* d, double ms[6], long long launches[6], long long units[6]);

/* Cell updates per coarse step (sum over levels of fluid cells * 2^l) and
   the number of kernels launched per coarse step. */
int lbm_work_per_step(const lbm_domain* d, long long* cell_updates, int* kernels);

/* Write / read the full state (populations, parities, step and force
   history) to / from a file; the domain must be built identically.
   lbm_load checks the file's header and size before it copies anything: a
   file that does not match the domain gives LBM_EINVAL and leaves the
   domain's state unchanged. */
int lbm_save(lbm_domain* d, const char* path);
int lbm_load(lbm_domain* d, const char* path);

void lbm_destroy(lbm_domain* d);
const char* lbm_status_string(int status);
const char* lbm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
