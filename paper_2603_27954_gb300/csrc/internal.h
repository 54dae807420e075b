// Internal declarations of liblbm (host side and kernel launch wrappers).
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <vector_types.h>  // int2

#include "../../include/lbm.h"

namespace lbm {

constexpr int kQ = 27;
inline int cx(int i) { return i % 3 - 1; }
inline int cy(int i) { return (i / 3) % 3 - 1; }
inline int cz(int i) { return i / 9 - 1; }
inline int opposite(int i) { return 26 - i; }
inline int dir_index(int x, int y, int z) { return (x + 1) + 3 * (y + 1) + 9 * (z + 1); }

// ---------------------------------------------------------------- geometry
struct Prim {
  int kind;  // 0 cylinder, 1 half-space, 2 box
  double p[8];
};

struct Tree {
  std::vector<double> seg;  // rows of 8: x0 y0 z0 x1 y1 z1 D gen
  int count() const { return (int)(seg.size() / 8); }
};

// Eq. (1): rewrite the axiom n times, then interpret the string with a turtle.
int build_lsystem(const lbm_tree_desc& t, Tree* out);
void tree_bounds(const Tree& t, double lo[3], double hi[3]);
double tree_height(const Tree& t);
void tree_centroid(const Tree& t, double c[3]);
void tree_affine(Tree* t, double scale, const double shift[3]);
double frontal_area(const Tree& t, double pitch);
// rows of 9: log10 Re_d, generation, D/H, cos(alpha), I_u, shielding depth, L, D, sin^3(alpha)
void branch_table(const Tree& t, double u, double nu, double height, double i_u, std::vector<double>* out);

bool prim_contains(const Prim& p, const double x[3]);
double prim_entry(const Prim& p, const double x[3], const double d[3]);  // t >= 0 or +inf
void prim_bounds(const Prim& p, double lo[3], double hi[3]);

// ---------------------------------------------------------------- device tables
// Offsets are element offsets (floats) into a level's population array.
// random-Fourier-mode inflow: per mode k (3), a (3), psi, pad
constexpr int kModeCols = 8;
constexpr int kMaxModes = 1024;
uint64_t splitmix(uint64_t seed, uint64_t k);
void rfm_modes(uint64_t seed, int n, double i_u, double u, double l_int, std::vector<double>* out);

// Reference state of the FP16 storage: stored values are (f_i - w_i - r_i) s
// with r_i = f_i^eq(1, U e_x) - w_i, the inflow equilibrium's deviation, so
// that the free stream stores values near zero (the 11-bit significand then
// resolves the flow's departures from it, not from rest).  Its raw moments
// are j_x = U and Pi_xx = U^2 (all others zero); out[3 z + cx + 1] holds
// r_i s for the population with z zero components among (c_y, c_z) and
// x component cx.
struct RefShift {
  float u, u2;
  float out[9];
};

struct FrictionSample {  // wall-shear quadrature point of the finest level
  int slot[2];           // storage blocks of the two sampled fluid cells (slot[1] < 0: one cell)
  int cell[2];           // their indices inside the blocks
  float n[3];            // outward wall normal
  float area;            // quadrature weight (finest cells^2)
  float dist[2];         // normal distances of the cell centres from the wall point
  int seg;               // primitive (branch) the point lies on
  int pad;
};

struct FaceEntry {   // domain faces of level 0 (Sec. 2.3)
  long long dst;
  long long src;     // -1: inflow equilibrium of direction dir
  int dir;
  int pad;
};
struct WallEntry {   // one cut link (Bouzidi linear bounce-back + momentum exchange)
  long long dst, a, b, c;  // a: f*_i(x_f); b: f*_i(x_f - c_i) or -1; c: f*_ibar(x_f)
  float q;
  int dir;
  int seg;                 // branch of the link (links are ordered by branch)
  int pad;
};
struct ExplodeEntry {    // fine inflow before the second fine step
  long long dst;         // fine ghost slot
  long long src[2];      // coarse post-collision slot per coarse parity
};
struct SaveEntry {       // fine post-collision value of the first fine step kept for later
  long long src;
};
struct InflowEntry {     // fine inflow for the next first fine step
  long long dst;         // fine own slot
  long long csrc[2];     // coarse post-collision slot per coarse parity
  int sv;                // saved value the destination holds before this write (its save index), or -1
  int pad;
};
struct CoalesceEntry {   // coarse cell next to the fine region, one direction
  long long dst[2];      // coarse slot per coarse parity (also its coarse source)
  long long fsrc[8];     // >= 0 fine slot; < 0: saved value -(v+1)
  int nfine;
  int ncoarse;
};

// The same tables with 32-bit element offsets, uploaded instead of the
// 64-bit ones when every array they address holds fewer than 2^31 elements
// (40-55 % fewer table bytes per step for the boundary and interface kernels).
struct FaceEntryN {
  int dst, src, dir;
};
struct WallEntryN {
  int dst, a, b, c;
  float q;
  int dir;
};
struct ExplodeEntryN {
  int dst;
  int src[2];
};
struct SaveEntryN {
  int src;
};
struct InflowEntryN {
  int dst;
  int csrc[2];
  int sv;
};
struct CoalesceEntryN {
  int dst[2];
  int fsrc[8];
  short nfine, ncoarse;
};

// FP64 ledger of one refinement interface (coarse level l, fine level l + 1).
// Per coarse step three flows are summed, each as mass and momentum (x, y,
// z), in volume units of a fine cell: In, the coarse values the explode and
// inflow transfers hand to the fine level; OutF, the fine values the coalesce
// transfer takes from it; RecvC, what the coarse slots receive (8 x the
// stored coalesce result minus its n_coarse x old-value part).  Device sums
// are exact 64-bit fixed point (quantum 2^-40 of a population deviation), in
// kLedgerCopies copies to spread atomic traffic; the coalesce launch's last
// CTA folds them into FP64 `last` and `total` and clears them.
constexpr int kLedgerCopies = 32;
constexpr int kLedgerVals = 12;  // In (m, jx, jy, jz), OutF (...), RecvC (...)
struct LedgerDev {
  long long acc[kLedgerCopies][kLedgerVals];
  unsigned done, pad;
  double last[kLedgerVals];
  double total[kLedgerVals];
  double steps;
};
// host-computed parts of the fold: the constant part (w_i + r_i) of every
// entry's full population, per flow, and the fine cell's volume
struct LedgerConst {
  double c[kLedgerVals];
  double vol;
};

// ---------------------------------------------------------------- mesh
enum CellType : uint8_t { FLUID = 0, SOLID = 1, COVERED = 2, OUTSIDE = 3 };
enum BlockState : int8_t { ABSENT = 0, ACTIVE = 1, GHOST = 2 };

struct Link {
  int x, y, z, dir;
  double q;
  int seg;  // primitive (branch) whose surface the link crosses first
};

struct Level {
  int l = 0, B = 16;
  int rlo[3] = {0, 0, 0}, rhi[3] = {0, 0, 0};  // real region, level-l cells
  int org[3] = {0, 0, 0}, nb[3] = {0, 0, 0};    // block grid origin (cells) and extent (blocks)
  bool wrap[3] = {false, false, false};          // periodic axes (level 0)
  int dom[3] = {0, 0, 0};                        // level extent along periodic axes
  std::vector<int> slot;                         // block grid -> storage index, -1 absent
  std::vector<int> grid_of;                      // storage index -> block grid index
  int n_active = 0, n_storage = 0;
  std::vector<uint8_t> type;                     // n_storage * B^3
  std::vector<int> nbr;                          // n_active * 27
  std::vector<int> maskoff;                      // n_active: -1 all fluid, else mask block index
  std::vector<uint8_t> masks;                    // collide flags, B^3 per masked block
  long long n_fluid = 0;
  double nu = 0, omega1 = 1;
  int esize = 4;        // bytes per stored population: 8 (FP64), 4 (FP32) or 2 (FP16)
  float scale = 1.0f;   // stored value = (f - w - r) * scale (r = 0 in FP32)
  std::vector<Link> links;
  std::vector<double> link_q;  // FP64 wall fractions in table order (FP64 storage form)
  std::vector<WallEntry> wall[2];
  std::vector<int> seg_begin;                    // n_seg + 1 offsets into the ordered links
  std::vector<FaceEntry> face[2];
  std::vector<int> face_pos;  // per face entry: pulled-from cell (x, y, z, 0), periodic axes wrapped
  // turbulent inflow: the distinct cells face entries pull the inflow
  // equilibrium from (x, y, z, 0 each), and per face entry the index of its
  // cell (-1 for an entry that copies a fluid value)
  std::vector<int> turb_cells, turb_idx;
  // interface with the next finer level (this level = coarse)
  std::vector<ExplodeEntry> expl;
  std::vector<SaveEntry> save;
  // the save table as the device gets it: entries whose slot an inflow entry
  // saves itself (before overwriting it) carry src = -1
  std::vector<SaveEntry> save_dev;
  std::vector<InflowEntry> infl;
  std::vector<CoalesceEntry> coal;
  double wall_rest[3] = {0, 0, 0};  // sum over the cut links of c_i 2 w_i
  // the walls may run beside the next interface transfer of the coarser level
  // (no slot one writes is read or written by the other; checked on the host)
  bool ovl_walls = false;
  // per parity p of a collide: the active blocks it may update while the
  // walls of the step before still run (no slot they touch is touched by
  // those walls), n_windep[p] of them, followed by the others
  std::vector<int> wblocks[2];
  int n_windep[2] = {0, 0};
  size_t off_wblocks[2] = {0, 0};
  // 32-bit forms (filled when narrow_ok) and the form on the device
  bool narrow_ok = false, narrow = false;
  std::vector<WallEntryN> wall_n[2];
  std::vector<FaceEntryN> face_n[2];
  std::vector<ExplodeEntryN> expl_n;
  std::vector<SaveEntryN> save_n;
  std::vector<InflowEntryN> infl_n;
  std::vector<CoalesceEntryN> coal_n;
  // device offsets (bytes from the bound base)
  size_t off_f = 0, off_nbr = 0, off_maskoff = 0, off_masks = 0;
  size_t off_wall[2] = {0, 0}, off_face[2] = {0, 0};
  size_t off_expl = 0, off_save = 0, off_infl = 0, off_coal = 0, off_saved = 0, off_q64 = 0;
  size_t off_ledger = 0;  // LedgerDev of the interface with the next finer level
  LedgerConst ledger_const{};

  long long cells_per_block() const { return (long long)B * B * B; }
  size_t f_elems() const { return (size_t)n_storage * kQ * cells_per_block(); }
  bool in_real(int x, int y, int z) const {
    return x >= rlo[0] && x < rhi[0] && y >= rlo[1] && y < rhi[1] && z >= rlo[2] && z < rhi[2];
  }
  // storage index and local cell of a level-l cell (periodic wrap applied); -1 if no storage
  int locate(int x, int y, int z, int* local) const;
  CellType cell_type(int x, int y, int z) const;
  long long addr(int x, int y, int z, int dir) const;  // element offset or -1
};

struct Mesh {
  // the level-0 faces may run beside everything up to the end of the coarse
  // step (no slot they touch is touched by the level-0 walls or interface)
  bool ovl_faces = false;
  bool turbulent = false;  // level-0 inflow from random Fourier modes (one tick launch per coarse step)
  bool friction = false;   // wall-shear sums at the end of every coarse step (two launches)
  int L = 1, B = 16;
  int n0[3] = {0, 0, 0};
  int bc[3] = {0, 0, 0};
  std::vector<Level> lv;
  int boxes[6][6] = {};
  std::string error;
};

// Wall-shear quadrature points of the finest level, grouped by primitive.
int build_friction_samples(const Mesh& m, const std::vector<Prim>& prims, std::vector<FrictionSample>* out,
                           std::vector<int>* seg_begin);
// Build block structure, cell types (solid from primitives), links and all tables.
int build_mesh(const lbm_domain_desc& d, const int boxes[6][6], const std::vector<Prim>& prims, Mesh* m);
// Refinement boxes from the tree (finest: bounding box grown by margin; coarser: footprint + 1 block).
void refinement_boxes(const Tree& t, int levels, int block, double margin, int boxes[6][6]);

// ---------------------------------------------------------------- kernels (kernels.cu)
struct CollideArgs {
  void* f;            // level populations: float, or __half when half != 0
  long long f_elems;  // elements in the level's array
  const int* nbr;
  const int* maskoff;
  const uint8_t* masks;
  int n_active;
  float omega1, omega2;
  int galilean;
  double* err;        // set to 1 when a bounded device wait gives up
  int half;           // FP16 storage of scaled deviations
  int f64;            // FP64 storage (the double-precision form; rates below)
  double omega1d, omega2d;
  float scale, inv_scale;
  int wide;           // 64-bit element offsets even when f_elems < 2^31
  int odd_variant;    // LBM_ODD_COLUMNS | LBM_ODD_STAGED | LBM_ODD_DIRECT
  int even_variant;   // LBM_EVEN_DIRECT | LBM_EVEN_TMA | LBM_EVEN_PAIRS
  int zshift_even;    // log2 of the CTAs per active block (each walks B >> zshift slabs)
  int zshift_odd;     //   of the even and of the odd step (one-CTA-per-block kernels)
  RefShift ref;       // FP16 storage reference (unused for FP32)
  const int* blocks;  // launch over these active blocks (n_active of them); nullptr: all, in order
};
int prepare_kernels();
int launch_collide(const CollideArgs& a, int B, int odd, void* stream);
// r_i per population (unscaled), the FP16 storage reference; zero for FP32
struct Ref27 {
  float v[27];
};
struct TurbArgs {      // turbulent inflow; n_modes == 0: uniform inflow equilibrium
  const int* idx;       // per face entry: index of the cell it pulls from, -1: the entry copies a value
  const int* cells;     // per pulled-from cell: level-0 (x, y, z, 0)
  float* vel;           // per pulled-from cell: the step's inflow velocity (ux, uy, uz, 0)
  int n_cells;
  const float* modes;   // n_modes x kModeCols
  int n_modes;
  float u;              // mean inflow speed along x
  float scale;          // storage scale of the level
  const long long* tick;  // coarse steps done
  int shift;            // store relative to the inflow equilibrium (FP16 reference)
};
// Table arguments `e` point to the 64-bit entries, or to the 32-bit ones (the
// ...N types) when `narrow` is set.
int launch_faces(void* f, int esize, const void* e, int narrow, int n, const double feq[27], const TurbArgs& turb,
                 void* stream);
// one launch over a work list of (index into lv, block) pairs; grid <= 0: one CTA per item
// zshift: each item is walked by 2^zshift CTAs (or grid strides) of B >> zshift slabs
int launch_collide_batch(const CollideArgs* lv, const int2* items, int n_items, int B, int odd, int odd_variant,
                         int even_variant, int half, int wide, int grid, int zshift, void* stream);
int launch_tick(long long* tick, void* stream);
// per-sample viscous traction times area, tangential part: out[3 k .. 3 k + 2]
int launch_friction(const void* f, int esize, float inv_scale, const Ref27& ref, int B, const int* nbr, int odd,
                    float omega1, const FrictionSample* e, int n, double* out, void* stream);
// Bouzidi update and momentum exchange of one link table; with `accum` set,
// the force of this step (gauge-form link sums plus rest[3], the exact sum of
// c_i 2 w_i over the links) goes to accum[0..2] and is added to accum[3..6]
// by the launch's last CTA (`done`: a zeroed counter it leaves zeroed).
// q64: the links' wall fractions in FP64 (FP64 storage form), or NULL to use
// the FP32 q of the table entries
int launch_walls(void* f, int esize, const double* q64, float inv_scale, const Ref27& ref, const void* e, int narrow,
                 int n, double* partials, double* link_force, unsigned* done, double* accum, const double rest[3],
                 void* stream);
int launch_segments(const double* link_force, const int* seg_begin, int n_seg, double* seg_accum, void* stream);
int walls_partial_count(int n);
// `esize`: bytes per stored population (2 binary16, 4 FP32, 8 FP64); saved
// values are FP32, or FP64 for the FP64 form.  `ledger` (or NULL) is the
// interface's ledger; c3_log2 = log2 of the cells per block (the direction of
// an entry is the population plane of its destination slot); inv_sc / inv_sf
// undo the storage scale of the coarse / fine level.
// the explode, save and inflow entries of an interface in one launch
int launch_explode(void* fine, const void* coarse, int esize, float ratio, const void* e, int narrow, int ne,
                   const void* s, int ns, const void* ie, int ni, void* saved, int parity, LedgerDev* ledger,
                   int c3_log2, float inv_sf, void* stream);
int launch_coalesce(void* coarse, const void* fine, int esize, float ratio, const void* e, int narrow, int n,
                    const void* saved, int parity, LedgerDev* ledger, const LedgerConst& lc, int c3_log2,
                    float inv_sc, float inv_sf, void* stream);
// fill the 32-bit tables of every level whose addressed arrays allow them
void narrow_tables(Mesh* m);
int launch_fill(void* f, int esize, long long n_blocks, int B, const double dev[27], void* stream);
int launch_mass(const void* f, int esize, float inv_scale, const Ref27& ref, const int* nbr, const int* maskoff,
                const uint8_t* masks, int n_active, int B, int parity, double* partials, void* stream);
int mass_partial_count(int n_active);
int noalloc_max_blocks();
int noalloc_scratch(double** out);
int launch_mass_noalloc(const void* f, int esize, float inv_scale, const Ref27& ref, const int* nbr,
                        const int* maskoff, const uint8_t* masks, int n_active, int B, int parity, double* scratch,
                        void* stream);
const char* cuda_error_string();

// surrogate network kernels (mlp.cu); W / B operands of the GEMMs are BF16 or FP32
const char* mlp_error_string();

}  // namespace lbm
