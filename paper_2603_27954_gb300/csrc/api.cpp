// C-ABI of liblbm (include/lbm.h): domain set-up, device memory binding,
// the recursively sub-cycled step driver, drag and diagnostics.  Every
// exported function is a function-try-block: a C++ exception from inside the
// library (a failed host allocation above all) becomes a status and a
// message instead of crossing the C boundary.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "half_host.h"
#include "internal.h"

using namespace lbm;

namespace {
thread_local std::string g_error;

int fail(int code, const std::string& msg) {
  g_error = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char* what) {
  g_error = std::string(what) + ": " + cudaGetErrorString(e);
  return LBM_ECUDA;
}
// No C++ exception leaves the C-ABI: the one in flight (called from a catch
// handler) becomes a status and a message.
int exception_status() {
  try {
    throw;
  } catch (const std::bad_alloc&) {
    return fail(LBM_ENOMEM, "host memory allocation failed");
  } catch (const std::length_error&) {
    return fail(LBM_ENOMEM, "host allocation too large");
  } catch (const std::exception& e) {
    return fail(LBM_ESTATE, std::string("internal error: ") + e.what());
  } catch (...) {
    return fail(LBM_ESTATE, "internal error");
  }
}
#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

double rest_weight(int i) {
  auto w1 = [](int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; };
  return w1(cx(i)) * w1(cy(i)) * w1(cz(i));
}

// equilibrium: rho times the product of 1-D three-point distributions with
// mean u_a and variance 1/3
double equilibrium(int i, double rho, const double u[3]) {
  auto phi = [](int c, double v) { return c == 0 ? 2.0 / 3.0 - v * v : 0.5 * (1.0 / 3.0 + v * v + c * v); };
  return rho * phi(cx(i), u[0]) * phi(cy(i), u[1]) * phi(cz(i), u[2]);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// automatic z split of a collide launch over `blocks` active blocks (log2 of
// the CTAs per block), from GB300 sweeps with 16^3 blocks: FP32 steps and the
// FP16 odd step run fastest with 8 CTAs per block on every workload; the FP16
// even step gains from a split only while the grid is short (the fewest CTAs
// per block that give at least 32 CTAs per SM); 8^3 blocks are not split
int auto_zshift(const lbm_domain_desc& s, long long blocks, int sms, int odd) {
  if (s.block != 16) return 0;
  if (s.precision == LBM_FP32 || odd) return 3;
  int k = 0;
  while (k < 3 && (blocks << k) < 32LL * sms) ++k;
  return k;
}
// log2 of a requested z split (CTAs per block, a power of two up to B); 0
// (automatic) maps to -2, anything else invalid to -1
int zshift_req(int split, int B) {
  if (split == 0) return -2;
  for (int k = 0; (1 << k) <= B; ++k)
    if (split == (1 << k)) return k;
  return -1;
}

enum { KC_COLLIDE = 0, KC_COLLIDE_ODD = 1, KC_FACES = 2, KC_WALLS = 3, KC_IFACE = 4, KC_N = 6 };
}  // namespace

struct lbm_domain {
  lbm_domain_desc d{};
  cudaStream_t stream = nullptr;
  Tree tree;
  bool have_tree = false;
  std::vector<Prim> prims;
  Mesh mesh;
  bool built = false;
  double H = 0, A_x = 0, nu_f = 0;
  // device
  char* base = nullptr;
  size_t need = 0;
  size_t off_partials = 0, off_accum = 0, off_mpart = 0, off_wdone = 0;
  // parallel branches of the step: [0] the level-0 faces, [1] the walls
  bool overlap = true;
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t ev_fork[2] = {nullptr, nullptr}, ev_join[2] = {nullptr, nullptr};
  bool pend[2] = {false, false};
  // per level with a finer level: its collide and boundary kernels run beside
  // the finer level's first sub-step (they touch different arrays)
  std::vector<cudaStream_t> lside;
  std::vector<cudaEvent_t> lfork, ljoin;
  size_t off_linkf = 0, off_segb = 0, off_segacc = 0;  // per-branch forces (finest level)
  int n_seg = 0;
  bool branch_forces = false;
  bool ledger = true;         // FP64 interface ledger (lbm_set_interface_ledger)
  bool wide_offsets = false;  // force the 64-bit-offset collide kernels
  int odd_variant = LBM_ODD_COLUMNS, even_variant = LBM_EVEN_DIRECT;
  int z_split_even = 0, z_split_odd = 0;  // collide CTAs per active block; 0: automatic
  int sms = 0;                             // SM count of the device (queried at the first launch)
  // storage reference r_i (deviation of the inflow equilibrium for FP16, zero for FP32)
  double ref[27] = {};
  Ref27 ref27{};
  // wall-shear quadrature (friction force, C_F)
  std::vector<FrictionSample> fsamp;
  std::vector<int> fseg_begin;
  size_t off_fsamp = 0, off_fforce = 0, off_fsegb = 0, off_facc = 0, off_fmean = 0;
  bool friction_mean = false;
  // host tables page-locked in place at the first binding (faster, steadier uploads)
  std::vector<void*> pinned;
  // turbulent inflow (random Fourier modes), on when d.i_u > 0
  int n_modes = 256;
  double l_int = 0;  // integral length in level-0 cells; 0: the tree height
  size_t off_modes = 0, off_turbidx = 0, off_turbcells = 0, off_turbvel = 0, off_tick = 0;
  int max_wall_parts = 0;
  float feq_in[27];     // inflow equilibrium minus the rest weights, FP32
  double feq_in_d[27];  // the same in FP64 (FP64 storage form)
  int parity0 = 0;
  long long steps = 0;
  bool use_graphs = true;
  // graph[v][p]: one coarse step of parity p; v = 0 starts from a complete
  // state, v = 1 first runs the coalesce transfers the previous step left
  // pending (their parities in coal_in[p]); either leaves coal_out[p]
  cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  // runs of kRun[r] coarse steps (parity p first) in one graph, where no
  // transfer is left pending between steps: fewer graph launches and
  // boundaries between them
  cudaGraphExec_t graphr[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  std::vector<int> coal_in[2], coal_out[2];
  // per level: parity of the level's last step whose coalesce transfer is
  // still to run (-1: none); lbm_step runs them before it returns
  std::vector<int> pend_coal;
  int wall_branch_level = -1;  // level whose walls branch 1 carries
  // reorderings on while overlap is on (deferred coalesce and the collide
  // split around the walls join measured slower on the tree workloads;
  // lbm_autotune tries them)
  int ovl_feat = LBM_OVL_BRANCHES | LBM_OVL_LEVELS | LBM_OVL_TRANSFERS;
  int watchdog = 0;
  int last_status = LBM_OK;
  // timing
  bool timing = false;
  struct Rec {
    cudaEvent_t a, b;
    int cls;
    long long units;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
  double ms[KC_N] = {};
  long long launches[KC_N] = {}, units[KC_N] = {};

  template <class T>
  T* dev(size_t off) const { return reinterpret_cast<T*>(base + off); }
};

namespace {

void unpin_tables(lbm_domain* d) {
  for (void* p : d->pinned) cudaHostUnregister(p);
  d->pinned.clear();
}

// page-lock the larger host tables so that lbm_bind_memory uploads them by
// DMA from pinned memory; a table that cannot be registered stays pageable
void pin_tables(lbm_domain* d) {
  if (!d->pinned.empty()) return;
  auto pin = [&](void* p, size_t bytes) {
    if (bytes < (1u << 16)) return;
    if (cudaHostRegister(p, bytes, cudaHostRegisterDefault) == cudaSuccess) d->pinned.push_back(p);
    else cudaGetLastError();
  };
  for (Level& v : d->mesh.lv) {
    pin(v.nbr.data(), v.nbr.size() * sizeof(int));
    pin(v.maskoff.data(), v.maskoff.size() * sizeof(int));
    pin(v.masks.data(), v.masks.size());
    if (v.narrow_ok && !d->wide_offsets) {
      for (int p = 0; p < 2; ++p) {
        pin(v.wall_n[p].data(), v.wall_n[p].size() * sizeof(WallEntryN));
        pin(v.face_n[p].data(), v.face_n[p].size() * sizeof(FaceEntryN));
      }
      pin(v.expl_n.data(), v.expl_n.size() * sizeof(ExplodeEntryN));
      pin(v.save_n.data(), v.save_n.size() * sizeof(SaveEntryN));
      pin(v.infl_n.data(), v.infl_n.size() * sizeof(InflowEntryN));
      pin(v.coal_n.data(), v.coal_n.size() * sizeof(CoalesceEntryN));
      continue;
    }
    for (int p = 0; p < 2; ++p) {
      pin(v.wall[p].data(), v.wall[p].size() * sizeof(WallEntry));
      pin(v.face[p].data(), v.face[p].size() * sizeof(FaceEntry));
    }
    pin(v.expl.data(), v.expl.size() * sizeof(ExplodeEntry));
    pin(v.save_dev.data(), v.save_dev.size() * sizeof(SaveEntry));
    pin(v.infl.data(), v.infl.size() * sizeof(InflowEntry));
    pin(v.coal.data(), v.coal.size() * sizeof(CoalesceEntry));
  }
  pin(d->fsamp.data(), d->fsamp.size() * sizeof(FrictionSample));
}

void free_graphs(lbm_domain* d) {
  for (auto& gv : d->graph)
    for (auto& g : gv)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
  for (auto& gv : d->graphr)
    for (auto& g : gv)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
}

cudaEvent_t take_event(lbm_domain* d) {
  if (d->pool_used == d->pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    d->pool.push_back(e);
  }
  return d->pool[d->pool_used++];
}

struct Timed {
  lbm_domain* d;
  int cls;
  long long units;
  cudaEvent_t a = nullptr;
  Timed(lbm_domain* dd, int c, long long u) : d(dd), cls(c), units(u) {
    if (d->timing) {
      a = take_event(d);
      cudaEventRecord(a, d->stream);
    }
  }
  ~Timed() {
    if (d->timing) {
      cudaEvent_t b = take_event(d);
      cudaEventRecord(b, d->stream);
      d->recs.push_back({a, b, cls, units});
    }
  }
};

// the storage reference in the collision's form: j_x and Pi_xx of r, and r_i s
// per (zero components among c_y, c_z; c_x) class
RefShift ref_shift(const lbm_domain* dm, const Level& v) {
  RefShift r{};
  if (dm->d.precision != LBM_FP16_DEV) return r;
  const double U = dm->d.u_in;
  r.u = (float)U;
  r.u2 = (float)(U * U);
  const double wyz[3] = {1.0 / 36.0, 1.0 / 9.0, 4.0 / 9.0};
  const double rx[3] = {0.5 * (U * U - U), -U * U, 0.5 * (U * U + U)};
  for (int z = 0; z < 3; ++z)
    for (int c = 0; c < 3; ++c) r.out[3 * z + c] = (float)(wyz[z] * rx[c] * v.scale);
  return r;
}

int device_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 152;
  return n > 0 ? n : 152;
}

int level_zshift(lbm_domain* dm, const Level& v, int odd) {
  const int req = odd ? dm->z_split_odd : dm->z_split_even;
  if (req) return zshift_req(req, dm->d.block);
  if (!dm->sms) dm->sms = device_sms();
  return auto_zshift(dm->d, v.n_active, dm->sms, odd);
}

CollideArgs collide_args(lbm_domain* dm, int l) {
  Level& v = dm->mesh.lv[l];
  return CollideArgs{dm->base + v.off_f, (long long)v.f_elems(), dm->dev<int>(v.off_nbr),
                     dm->dev<int>(v.off_maskoff), dm->dev<uint8_t>(v.off_masks), v.n_active, (float)v.omega1,
                     (float)dm->d.omega2, dm->d.galilean, dm->dev<double>(dm->off_accum) + 7, v.esize == 2,
                     v.esize == 8, v.omega1, dm->d.omega2, v.scale,
                     1.0f / v.scale, dm->wide_offsets ? 1 : 0, dm->odd_variant, dm->even_variant,
                     level_zshift(dm, v, 0), level_zshift(dm, v, 1), ref_shift(dm, v)};
}

// Branches of the step on side streams: fork from the domain's stream, run,
// and join back before the next collide (walls) or at the end of the coarse
// step (faces, walls).  Inside a graph capture they become parallel branches.
int side_streams(lbm_domain* d) {
  if (d->side[0]) return LBM_OK;
  for (int k = 0; k < 2; ++k) {
    CK(cudaStreamCreateWithFlags(&d->side[k], cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&d->ev_fork[k], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&d->ev_join[k], cudaEventDisableTiming));
  }
  return LBM_OK;
}
int join_branch(lbm_domain* d, int k) {
  if (!d->pend[k]) return LBM_OK;
  d->pend[k] = false;
  CK(cudaStreamWaitEvent(d->stream, d->ev_join[k], 0));
  return LBM_OK;
}
// the stream branch k's kernels go to (forked from `parent`, by default the
// domain's stream)
int fork_branch(lbm_domain* d, int k, cudaStream_t* s, cudaStream_t parent = nullptr) {
  int rc = side_streams(d);
  if (!rc) rc = join_branch(d, k);
  if (rc) return rc;
  CK(cudaEventRecord(d->ev_fork[k], parent ? parent : d->stream));
  CK(cudaStreamWaitEvent(d->side[k], d->ev_fork[k], 0));
  *s = d->side[k];
  return LBM_OK;
}
int close_branch(lbm_domain* d, int k) {
  CK(cudaEventRecord(d->ev_join[k], d->side[k]));
  d->pend[k] = true;
  return LBM_OK;
}
// level l's own work on its side stream, beside the finer levels' first
// sub-step; joined before the interface transfer that needs both
int fork_level(lbm_domain* d, int l, cudaStream_t* s) {
  if ((int)d->lside.size() < d->mesh.L) {
    const size_t n0 = d->lside.size();
    d->lside.resize(d->mesh.L, nullptr);
    d->lfork.resize(d->mesh.L, nullptr);
    d->ljoin.resize(d->mesh.L, nullptr);
    for (size_t k = n0; k < d->lside.size(); ++k) {
      CK(cudaStreamCreateWithFlags(&d->lside[k], cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&d->lfork[k], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&d->ljoin[k], cudaEventDisableTiming));
    }
  }
  CK(cudaEventRecord(d->lfork[l], d->stream));
  CK(cudaStreamWaitEvent(d->lside[l], d->lfork[l], 0));
  *s = d->lside[l];
  return LBM_OK;
}
int join_level(lbm_domain* d, int l) {
  CK(cudaEventRecord(d->ljoin[l], d->lside[l]));
  CK(cudaStreamWaitEvent(d->stream, d->ljoin[l], 0));
  return LBM_OK;
}

void destroy_side_streams(lbm_domain* d) {
  for (size_t k = 0; k < d->lside.size(); ++k) {
    if (d->lside[k]) {
      cudaStreamSynchronize(d->lside[k]);
      cudaStreamDestroy(d->lside[k]);
    }
    if (d->lfork[k]) cudaEventDestroy(d->lfork[k]);
    if (d->ljoin[k]) cudaEventDestroy(d->ljoin[k]);
  }
  d->lside.clear();
  d->lfork.clear();
  d->ljoin.clear();
  for (int k = 0; k < 2; ++k) {
    if (d->side[k]) {
      cudaStreamSynchronize(d->side[k]);
      cudaStreamDestroy(d->side[k]);
    }
    if (d->ev_fork[k]) cudaEventDestroy(d->ev_fork[k]);
    if (d->ev_join[k]) cudaEventDestroy(d->ev_join[k]);
    d->side[k] = nullptr;
    d->ev_fork[k] = d->ev_join[k] = nullptr;
  }
}

// whether a reordering of the step is on
bool ovl(const lbm_domain* d, int feature) { return d->overlap && !d->timing && (d->ovl_feat & feature); }

// level l after its collide-stream sweep: faces (level 0), bounce-back and
// momentum exchange, per-branch and total force reductions (finest level).
// With `branches` the faces and the walls run on side streams where the host
// check found them independent of what follows (results are identical).
int post_collide(lbm_domain* dm, int l, int parity, cudaStream_t s, bool branches) {
  Mesh& m = dm->mesh;
  Level& v = m.lv[l];
  void* f = dm->base + v.off_f;
  const int esize = v.esize;
  int rc;
  // the faces may branch off the level's side stream too (the host check
  // covers everything up to the end of the coarse step); the walls only off
  // the domain's stream
  const bool face_branch = branches && ovl(dm, LBM_OVL_BRANCHES) && m.ovl_faces;
  branches = branches && ovl(dm, LBM_OVL_BRANCHES) && s == dm->stream;
  if (l == 0 && !v.face[parity].empty()) {
    cudaStream_t fs = s;
    if (face_branch && (rc = fork_branch(dm, 0, &fs, s))) return rc;
    Timed t(dm, KC_FACES, (long long)v.face[parity].size());
    double feq[27];
    for (int i = 0; i < 27; ++i)
      feq[i] = esize == 8 ? dm->feq_in_d[i] : (double)(float)((dm->feq_in[i] - dm->ref[i]) * v.scale);
    TurbArgs tb{nullptr, nullptr, nullptr, 0, nullptr, 0, (float)dm->d.u_in, v.scale, nullptr,
                dm->d.precision == LBM_FP16_DEV};
    if (dm->d.i_u > 0) {
      tb.idx = dm->dev<int>(dm->off_turbidx);
      tb.cells = dm->dev<int>(dm->off_turbcells);
      tb.vel = dm->dev<float>(dm->off_turbvel);
      tb.n_cells = (int)(v.turb_cells.size() / 4);
      tb.modes = dm->dev<float>(dm->off_modes);
      tb.n_modes = dm->n_modes;
      tb.tick = dm->dev<long long>(dm->off_tick);
    }
    if ((rc = launch_faces(f, esize, dm->base + v.off_face[parity], v.narrow, (int)v.face[parity].size(), feq, tb,
                           fs)))
      return rc;
    if (fs != s && (rc = close_branch(dm, 0))) return rc;
  }
  if (!v.wall[parity].empty()) {
    Timed t(dm, KC_WALLS, (long long)v.wall[parity].size());
    const cudaStream_t s_main = s;
    if (branches && v.ovl_walls) {
      if ((rc = fork_branch(dm, 1, &s))) return rc;
      dm->wall_branch_level = l;
    }
    int n = (int)v.wall[parity].size();
    const bool per_branch = dm->branch_forces && l == m.L - 1;
    // the finest level's walls reduce the force of the step in the same launch
    const bool finest = l == m.L - 1;
    if ((rc = launch_walls(f, esize, esize == 8 ? dm->dev<double>(v.off_q64) : nullptr, 1.0f / v.scale, dm->ref27,
                           dm->base + v.off_wall[parity], v.narrow, n,
                           dm->dev<double>(dm->off_partials), per_branch ? dm->dev<double>(dm->off_linkf) : nullptr,
                           dm->dev<unsigned>(dm->off_wdone), finest ? dm->dev<double>(dm->off_accum) : nullptr,
                           v.wall_rest, s)))
      return rc;
    if (per_branch && (rc = launch_segments(dm->dev<double>(dm->off_linkf), dm->dev<int>(dm->off_segb), dm->n_seg,
                                            dm->dev<double>(dm->off_segacc), s)))
      return rc;
    if (s != s_main && (rc = close_branch(dm, 1))) return rc;
  }
  return LBM_OK;
}

int c3_log2(int B) { return B == 16 ? 12 : 9; }
LedgerDev* ledger_of(lbm_domain* dm, const Level& v) {
  return dm->ledger ? dm->dev<LedgerDev>(v.off_ledger) : nullptr;
}

// The transfers from the coarse level to the finer one, in up to two
// launches per coarse step: `explode` (coarse post-collision values into the
// fine ghost slots the finer level's second sub-step pulls from: they only
// need the coarse collide, and the fine level's first sub-step touches its
// active cells' own slots only, so they may run beside it) and
// `save_inflow` (the fine values of the first sub-step that leave the box,
// for the coalesce transfer, and the fine inflow for the next first
// sub-step: both touch slots the second sub-step neither reads nor writes,
// so they may run beside it; they must finish before the coalesce
// transfer, which reads the saved values and overwrites coarse slots the
// inflow reads).
int iface_transfer(lbm_domain* dm, int l, int parity, cudaStream_t s, bool explode, bool save_inflow) {
  Level& v = dm->mesh.lv[l];
  Level& F = dm->mesh.lv[l + 1];
  const int ne = explode ? (int)v.expl.size() : 0;
  const int ns = save_inflow ? (int)v.save.size() : 0, ni = save_inflow ? (int)v.infl.size() : 0;
  Timed t(dm, KC_IFACE, (long long)ne + ni);
  return launch_explode(dm->base + F.off_f, dm->base + v.off_f, v.esize, F.scale / v.scale,
                        dm->base + v.off_expl, v.narrow, ne, dm->base + v.off_save, ns, dm->base + v.off_infl, ni,
                        dm->base + v.off_saved, parity, ledger_of(dm, v), c3_log2(v.B), 1.0f / F.scale, s);
}

// after the fine level's second sub-step: coarse cells next to the fine
// region from their children
int iface_coalesce(lbm_domain* dm, int l, int parity, cudaStream_t s) {
  Level& v = dm->mesh.lv[l];
  Level& F = dm->mesh.lv[l + 1];
  Timed t(dm, KC_IFACE, (long long)v.coal.size());
  return launch_coalesce(dm->base + v.off_f, dm->base + F.off_f, v.esize, F.scale / v.scale, dm->base + v.off_coal,
                         v.narrow, (int)v.coal.size(), dm->base + v.off_saved, parity, ledger_of(dm, v),
                         v.ledger_const, c3_log2(v.B), 1.0f / v.scale, 1.0f / F.scale, s);
}

// friction of the finest level at the current step boundary, added to acc
int friction_into(lbm_domain* dm, int odd, double* acc, cudaStream_t s) {
  const Level& v = dm->mesh.lv.back();
  if (dm->fsamp.empty()) return LBM_OK;
  int rc = launch_friction(dm->base + v.off_f, v.esize, 1.0f / v.scale, dm->ref27, v.B, dm->dev<int>(v.off_nbr), odd,
                           (float)v.omega1, dm->dev<FrictionSample>(dm->off_fsamp), (int)dm->fsamp.size(),
                           dm->dev<double>(dm->off_fforce), s);
  if (rc) return rc;
  return launch_segments(dm->dev<double>(dm->off_fforce), dm->dev<int>(dm->off_fsegb), (int)dm->prims.size(), acc, s);
}

// after the last kernel of a coarse step of parity p
int end_coarse_step(lbm_domain* dm, int parity, cudaStream_t s) {
  int rc;
  if ((rc = join_branch(dm, 0)) || (rc = join_branch(dm, 1))) return rc;
  if (dm->d.i_u > 0 && (rc = launch_tick(dm->dev<long long>(dm->off_tick), s))) return rc;
  if (dm->friction_mean) {
    // the finest level's incoming values: parity 0 on refined domains, else the next level-0 parity
    const int odd = dm->mesh.L == 1 ? (parity ^ 1) : 0;
    if ((rc = friction_into(dm, odd, dm->dev<double>(dm->off_fmean), s))) return rc;
  }
  return LBM_OK;
}

// one step of level l (recursively the two steps of every finer level)
// whether level l's collide of this parity runs in two launches around the
// join of the walls its previous step left running on branch 1: first the
// blocks those walls do not touch, then the rest
bool wall_split(const lbm_domain* dm, const Level& v, int l, int parity) {
  return ovl(dm, LBM_OVL_WALL_SPLIT) && dm->pend[1] && dm->wall_branch_level == l && v.n_windep[parity] > 0 &&
         v.n_windep[parity] < v.n_active && dm->odd_variant != LBM_ODD_STAGED;
}

int advance(lbm_domain* dm, int l, int parity) {
  Mesh& m = dm->mesh;
  Level& v = m.lv[l];
  int rc;
  const bool wsplit = wall_split(dm, v, l, parity);
  // walls before the next collide of any level (of the blocks they touch)
  if (!wsplit && (rc = join_branch(dm, 1))) return rc;
  // a level with a finer level runs its collide and boundary kernels beside
  // the finer levels' first sub-step (disjoint arrays), joined before explode;
  // not when it has cut links (the wall kernels of all levels share their
  // force partials)
  const bool split = l + 1 < m.L && ovl(dm, LBM_OVL_LEVELS) && v.wall[0].empty();
  cudaStream_t cs = dm->stream;
  if (split && (rc = fork_level(dm, l, &cs))) return rc;
  if ((int)dm->pend_coal.size() != m.L) dm->pend_coal.assign(m.L, -1);
  if (dm->pend_coal[l] >= 0) {
    // the coalesce transfer of this level's previous step: it reads the finer
    // level's ghost and saved values, which nothing touches before the
    // explode below, and writes this level's slots, which the collide reads
    if ((rc = iface_coalesce(dm, l, dm->pend_coal[l], cs))) return rc;
    dm->pend_coal[l] = -1;
  }
  if (wsplit) {
    // the blocks the walls do not touch on this stream (a level with walls
    // is never split off: cs is the domain's stream); the others on the
    // walls' branch after the walls and after everything this stream did so
    // far (the coarser level's explode among it).  The next fork or the end
    // of the coarse step joins the branch.
    CK(cudaEventRecord(dm->ev_fork[1], dm->stream));
    CK(cudaStreamWaitEvent(dm->side[1], dm->ev_fork[1], 0));
    CollideArgs a = collide_args(dm, l);
    a.blocks = dm->dev<int>(v.off_wblocks[parity]);
    a.n_active = v.n_windep[parity];
    if ((rc = launch_collide(a, v.B, parity, cs))) return rc;
    a.blocks += v.n_windep[parity];
    a.n_active = v.n_active - v.n_windep[parity];
    if ((rc = launch_collide(a, v.B, parity, dm->side[1]))) return rc;
    if ((rc = close_branch(dm, 1))) return rc;
  } else {
    Timed t(dm, parity ? KC_COLLIDE_ODD : KC_COLLIDE, v.n_fluid);
    if ((rc = launch_collide(collide_args(dm, l), v.B, parity, cs))) return rc;
  }
  if ((rc = post_collide(dm, l, parity, cs, true))) return rc;
  if (l + 1 < m.L) {
    // the transfers with the finer level run beside its sub-steps when the
    // finer level's walls touch none of their slots (host check); else in
    // the serial order
    const Level& F = m.lv[l + 1];
    const bool walls_clear = F.wall[0].empty() || F.ovl_walls;
    const bool beside = ovl(dm, LBM_OVL_TRANSFERS) && walls_clear;
    // explode right after this level's collide, on its side stream beside
    // the finer level's first sub-step when the level is split off
    const bool expl_side = split && beside;
    if (expl_side && (rc = iface_transfer(dm, l, parity, cs, true, false))) return rc;
    if ((rc = advance(dm, l + 1, 0))) return rc;
    if (split && (rc = join_level(dm, l))) return rc;
    // save and inflow entries on the level's side stream beside the finer
    // level's second sub-step, joined before the coalesce transfer
    const bool branch = beside && (v.save.size() || v.infl.size());
    if (!expl_side || !branch) {
      if ((rc = iface_transfer(dm, l, parity, dm->stream, !expl_side, !branch))) return rc;
    }
    if (branch) {
      cudaStream_t is;
      if ((rc = fork_level(dm, l, &is)) || (rc = iface_transfer(dm, l, parity, is, false, true))) return rc;
    }
    if ((rc = advance(dm, l + 1, 1))) return rc;
    if (branch && (rc = join_level(dm, l))) return rc;
    // the coalesce transfer waits for the head of this level's next step,
    // beside the finer level's first sub-step (which touches neither the
    // fine ghost and saved values it reads nor this level)
    if (ovl(dm, LBM_OVL_DEFER) && walls_clear) dm->pend_coal[l] = parity;
    else if ((rc = iface_coalesce(dm, l, parity, dm->stream))) return rc;
  }
  if (l == 0) return end_coarse_step(dm, parity, dm->stream);
  return LBM_OK;
}

// the pending coalesce transfers, finest first (each reads only its finer
// level's ghost and saved values, which no other pending transfer writes)
int flush_coalesce(lbm_domain* dm) {
  for (int l = (int)dm->pend_coal.size() - 1; l >= 0; --l) {
    if (dm->pend_coal[l] < 0) continue;
    int rc = iface_coalesce(dm, l, dm->pend_coal[l], dm->stream);
    if (rc) return rc;
    dm->pend_coal[l] = -1;
  }
  return LBM_OK;
}
bool any_pending(const lbm_domain* dm) {
  for (int p : dm->pend_coal)
    if (p >= 0) return true;
  return false;
}

int kernels_per_step(const lbm_domain* d, int l) {
  const Mesh& m = d->mesh;
  const Level& v = m.lv[l];
  int k = 1;
  // the finest level's second sub-step in two launches around the join of
  // the first sub-step's walls
  const bool on = d->overlap;
  if (l + 2 == m.L) {
    const Level& F = m.lv[l + 1];
    if (on && (d->ovl_feat & LBM_OVL_WALL_SPLIT) && (d->ovl_feat & LBM_OVL_BRANCHES) && F.ovl_walls &&
        F.n_windep[1] > 0 && F.n_windep[1] < F.n_active && d->odd_variant != LBM_ODD_STAGED)
      k += 1;
  }
  if (l == 0 && !v.face[0].empty()) k += 1;
  if (l == 0 && m.turbulent) k += 2;
  if (l == 0 && m.friction) k += 2;
  if (!v.wall[0].empty()) k += 1;
  // explode, save + inflow (launches of their own when the transfers run
  // beside the finer level's sub-steps, else one), coalesce
  if (l + 1 < m.L) {
    const Level& F = m.lv[l + 1];
    const bool beside = on && (d->ovl_feat & LBM_OVL_TRANSFERS) && (F.wall[0].empty() || F.ovl_walls);
    const bool any = v.expl.size() || v.save.size() || v.infl.size();
    k += 2 * kernels_per_step(d, l + 1) + (v.coal.empty() ? 0 : 1) +
         (beside ? (v.expl.empty() ? 0 : 1) + (v.save.size() || v.infl.size() ? 1 : 0) : (any ? 1 : 0));
  }
  return k;
}

int build(lbm_domain* d) {
  // viscosity from Re_H = U H / nu on the finest level (Sec. 2.3)
  if (d->d.re_h > 0) {
    if (!(d->H > 0)) return fail(LBM_EINVAL, "Re_H needs a tree with a height");
    d->nu_f = d->d.u_in * d->H / d->d.re_h;
  } else {
    d->nu_f = d->d.nu_finest;
  }
  if (!(d->nu_f > 0)) return fail(LBM_EINVAL, "viscosity must be positive");
  int boxes[6][6];
  std::memcpy(boxes, d->d.boxes, sizeof boxes);
  bool given = false;
  for (int l = 1; l < d->d.levels; ++l)
    for (int q = 0; q < 6; ++q) given |= boxes[l][q] != 0;
  if (d->d.levels > 1 && !given) {
    if (!d->have_tree || d->tree.count() == 0) return fail(LBM_EINVAL, "refinement needs boxes or a tree");
    refinement_boxes(d->tree, d->d.levels, d->d.block, d->d.refine_margin, boxes);
  }
  unpin_tables(d);
  d->mesh = Mesh();
  int rc = build_mesh(d->d, boxes, d->prims, &d->mesh);
  if (rc) return fail(rc, d->mesh.error);
  const int L = d->d.levels;
  for (int l = 0; l < L; ++l) {
    Level& v = d->mesh.lv[l];
    v.nu = d->nu_f * std::ldexp(1.0, -(L - 1 - l));
    v.omega1 = 1.0 / (3.0 * v.nu + 0.5);
    // FP16: deviations are at most ~0.1, so 2^13 keeps them far from both the
    // FP16 overflow (65504) and its subnormal range (below 6.1e-5 / 2^13)
    v.esize = d->d.precision == LBM_FP16_DEV ? 2 : (d->d.precision == LBM_FP64 ? 8 : 4);
    v.scale = d->d.precision == LBM_FP16_DEV ? 8192.0f : 1.0f;
  }
  narrow_tables(&d->mesh);
  // exact total of c_i 2 w_i over each level's cut links (zero for a body
  // whose links close a surface), the rest-weight part of the momentum
  // exchange that the wall kernel leaves out of its FP32 link sums
  for (Level& v : d->mesh.lv) {
    for (int a = 0; a < 3; ++a) v.wall_rest[a] = 0.0;
    for (const Link& k : v.links) {
      const double w2 = 2.0 * rest_weight(k.dir);
      v.wall_rest[0] += cx(k.dir) * w2;
      v.wall_rest[1] += cy(k.dir) * w2;
      v.wall_rest[2] += cz(k.dir) * w2;
    }
  }
  // device layout (table space for the 64-bit form, which the 32-bit one fits)
  size_t off = 0;
  auto put = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  d->max_wall_parts = 1;
  size_t max_blocks = 1;
  for (int l = 0; l < L; ++l) {
    Level& v = d->mesh.lv[l];
    v.off_f = put(v.f_elems() * (size_t)v.esize);
    v.off_nbr = put(v.nbr.size() * sizeof(int));
    v.off_maskoff = put(v.maskoff.size() * sizeof(int));
    v.off_masks = put(v.masks.size());
    for (int p = 0; p < 2; ++p) v.off_wblocks[p] = put(v.wblocks[p].size() * sizeof(int));
    for (int p = 0; p < 2; ++p) {
      v.off_wall[p] = put(v.wall[p].size() * sizeof(WallEntry));
      v.off_face[p] = put(v.face[p].size() * sizeof(FaceEntry));
    }
    v.off_expl = put(v.expl.size() * sizeof(ExplodeEntry));
    v.off_save = put(v.save.size() * sizeof(SaveEntry));
    v.off_infl = put(v.infl.size() * sizeof(InflowEntry));
    v.off_coal = put(v.coal.size() * sizeof(CoalesceEntry));
    v.off_saved = put(v.save.size() * (v.esize == 8 ? sizeof(double) : sizeof(float)));
    v.link_q.clear();
    if (v.esize == 8)
      for (const Link& k : v.links) v.link_q.push_back(k.q);
    v.off_q64 = put(v.link_q.size() * sizeof(double));
    v.off_ledger = put(l + 1 < L ? sizeof(LedgerDev) : 0);
    d->max_wall_parts = std::max(d->max_wall_parts, walls_partial_count((int)v.wall[0].size()));
    max_blocks = std::max(max_blocks, (size_t)v.n_active);
  }
  {
    const Level& fl = d->mesh.lv[L - 1];
    d->n_seg = (int)d->prims.size();
    d->off_linkf = put(fl.links.size() * 3 * sizeof(double));
    d->off_segb = put((size_t)(d->n_seg + 1) * sizeof(int));
    d->off_segacc = put((size_t)d->n_seg * 4 * sizeof(double));
  }
  d->off_partials = put((size_t)d->max_wall_parts * 3 * sizeof(double));
  d->off_accum = put(8 * sizeof(double));
  d->off_tick = put(sizeof(long long));
  build_friction_samples(d->mesh, d->prims, &d->fsamp, &d->fseg_begin);
  d->off_fsamp = put(d->fsamp.size() * sizeof(FrictionSample));
  d->off_fforce = put(d->fsamp.size() * 3 * sizeof(double));
  d->off_fsegb = put(d->fseg_begin.size() * sizeof(int));
  d->off_facc = put(std::max<size_t>(1, d->prims.size()) * 4 * sizeof(double));
  d->off_fmean = put(std::max<size_t>(1, d->prims.size()) * 4 * sizeof(double));
  d->mesh.turbulent = d->d.i_u > 0;
  d->mesh.friction = d->friction_mean;
  if (d->d.i_u > 0) {
    d->off_modes = put((size_t)kMaxModes * kModeCols * sizeof(float));
    const Level& l0 = d->mesh.lv[0];
    d->off_turbidx = put(l0.turb_idx.size() * sizeof(int));
    d->off_turbcells = put(l0.turb_cells.size() * sizeof(int));
    d->off_turbvel = put(l0.turb_cells.size() * sizeof(float));
  }
  d->off_mpart = put(max_blocks * 5 * sizeof(double));
  d->off_wdone = put(sizeof(unsigned));
  d->need = off;
  double u[3] = {d->d.u_in, 0, 0};
  for (int i = 0; i < 27; ++i) {
    d->feq_in_d[i] = equilibrium(i, 1.0, u) - rest_weight(i);
    d->feq_in[i] = (float)d->feq_in_d[i];
  }
  // FP16 storage keeps (f - w - r) s with r the inflow equilibrium's deviation:
  // the free stream is then stored as values near zero
  for (int i = 0; i < 27; ++i) {
    d->ref[i] = d->d.precision == LBM_FP16_DEV ? equilibrium(i, 1.0, u) - rest_weight(i) : 0.0;
    d->ref27.v[i] = (float)d->ref[i];
  }
  // the constant part (w_i + r_i) of the full populations the interface
  // flows carry, per flow, and the fine cell volume (level-0 cell = 1)
  for (int l = 0; l + 1 < L; ++l) {
    Level& v = d->mesh.lv[l];
    LedgerConst& lc = v.ledger_const;
    lc = LedgerConst{};
    lc.vol = std::ldexp(1.0, -3 * (l + 1));
    const long long c3 = v.cells_per_block();
    auto add = [&](int flow, int dir, double weight) {
      const double wr = (rest_weight(dir) + d->ref[dir]) * weight;
      lc.c[4 * flow] += wr;
      lc.c[4 * flow + 1] += cx(dir) * wr;
      lc.c[4 * flow + 2] += cy(dir) * wr;
      lc.c[4 * flow + 3] += cz(dir) * wr;
    };
    for (const ExplodeEntry& e : v.expl) add(0, 26 - (int)((e.dst / c3) % 27), 1.0);
    for (const InflowEntry& e : v.infl) add(0, (int)((e.dst / c3) % 27), 1.0);
    for (const CoalesceEntry& e : v.coal) {
      const int dir = 26 - (int)((e.dst[0] / c3) % 27);
      add(1, dir, e.nfine);
      add(2, dir, e.nfine);
    }
  }
  d->built = true;
  return LBM_OK;
}

double integral_length(const lbm_domain* d) {
  return d->l_int > 0 ? d->l_int : d->H * std::ldexp(1.0, -(d->d.levels - 1));
}

void make_modes(const lbm_domain* d, std::vector<double>* modes) {
  rfm_modes(d->d.seed, d->n_modes, d->d.i_u, d->d.u_in, integral_length(d), modes);
}

int upload_modes(lbm_domain* d) {
  std::vector<double> m;
  make_modes(d, &m);
  std::vector<float> mf(m.begin(), m.end());
  if (!mf.empty())
    CK(cudaMemcpyAsync(d->base + d->off_modes, mf.data(), mf.size() * sizeof(float), cudaMemcpyHostToDevice,
                       d->stream));
  CK(cudaStreamSynchronize(d->stream));
  return LBM_OK;
}

// the device copy of the coarse-step count (turbulent inflow time)
int set_tick(lbm_domain* d) {
  CK(cudaMemcpyAsync(d->base + d->off_tick, &d->steps, sizeof(long long), cudaMemcpyHostToDevice, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  return LBM_OK;
}

// boundary and interface tables of every level, 32-bit where the level allows
// it and 64-bit offsets are not forced (the device space fits the 64-bit form)
int upload_tables(lbm_domain* d) {
  auto cp = [&](size_t off, const void* src, size_t bytes) -> cudaError_t {
    if (!bytes) return cudaSuccess;
    return cudaMemcpyAsync(d->base + off, src, bytes, cudaMemcpyHostToDevice, d->stream);
  };
  for (Level& v : d->mesh.lv) {
    v.narrow = v.narrow_ok && !d->wide_offsets;
    if (v.narrow) {
      for (int p = 0; p < 2; ++p) {
        CK(cp(v.off_wall[p], v.wall_n[p].data(), v.wall_n[p].size() * sizeof(WallEntryN)));
        CK(cp(v.off_face[p], v.face_n[p].data(), v.face_n[p].size() * sizeof(FaceEntryN)));
      }
      CK(cp(v.off_expl, v.expl_n.data(), v.expl_n.size() * sizeof(ExplodeEntryN)));
      CK(cp(v.off_save, v.save_n.data(), v.save_n.size() * sizeof(SaveEntryN)));
      CK(cp(v.off_infl, v.infl_n.data(), v.infl_n.size() * sizeof(InflowEntryN)));
      CK(cp(v.off_coal, v.coal_n.data(), v.coal_n.size() * sizeof(CoalesceEntryN)));
      continue;
    }
    for (int p = 0; p < 2; ++p) {
      CK(cp(v.off_wall[p], v.wall[p].data(), v.wall[p].size() * sizeof(WallEntry)));
      CK(cp(v.off_face[p], v.face[p].data(), v.face[p].size() * sizeof(FaceEntry)));
    }
    CK(cp(v.off_expl, v.expl.data(), v.expl.size() * sizeof(ExplodeEntry)));
    CK(cp(v.off_save, v.save_dev.data(), v.save_dev.size() * sizeof(SaveEntry)));
    CK(cp(v.off_infl, v.infl.data(), v.infl.size() * sizeof(InflowEntry)));
    CK(cp(v.off_coal, v.coal.data(), v.coal.size() * sizeof(CoalesceEntry)));
  }
  return LBM_OK;
}

// host-to-device bytes of one binding: the tables upload() copies (in the
// form the device uses), the turbulence modes and the step counter; the
// populations are initialised on the device and not copied
size_t upload_bytes(const lbm_domain* d) {
  size_t b = 0;
  for (const Level& v : d->mesh.lv) {
    b += v.nbr.size() * sizeof(int) + v.maskoff.size() * sizeof(int) + v.masks.size() +
         v.link_q.size() * sizeof(double) + (v.wblocks[0].size() + v.wblocks[1].size()) * sizeof(int);
    if (v.narrow_ok && !d->wide_offsets) {
      for (int p = 0; p < 2; ++p) b += v.wall_n[p].size() * sizeof(WallEntryN) + v.face_n[p].size() * sizeof(FaceEntryN);
      b += v.expl_n.size() * sizeof(ExplodeEntryN) + v.save_n.size() * sizeof(SaveEntryN) +
           v.infl_n.size() * sizeof(InflowEntryN) + v.coal_n.size() * sizeof(CoalesceEntryN);
    } else {
      for (int p = 0; p < 2; ++p) b += v.wall[p].size() * sizeof(WallEntry) + v.face[p].size() * sizeof(FaceEntry);
      b += v.expl.size() * sizeof(ExplodeEntry) + v.save.size() * sizeof(SaveEntry) +
           v.infl.size() * sizeof(InflowEntry) + v.coal.size() * sizeof(CoalesceEntry);
    }
  }
  if (d->n_seg) b += d->mesh.lv.back().seg_begin.size() * sizeof(int);
  b += d->fsamp.size() * sizeof(FrictionSample) + d->fseg_begin.size() * sizeof(int);
  if (d->d.i_u > 0)
    b += (d->mesh.lv[0].turb_idx.size() + d->mesh.lv[0].turb_cells.size()) * sizeof(int) +
         (size_t)d->n_modes * kModeCols * sizeof(float);
  return b + sizeof(long long);
}

int upload(lbm_domain* d) {
  auto cp = [&](size_t off, const void* src, size_t bytes) -> cudaError_t {
    if (!bytes) return cudaSuccess;
    return cudaMemcpyAsync(d->base + off, src, bytes, cudaMemcpyHostToDevice, d->stream);
  };
  for (Level& v : d->mesh.lv) {
    CK(cp(v.off_q64, v.link_q.data(), v.link_q.size() * sizeof(double)));
    CK(cp(v.off_nbr, v.nbr.data(), v.nbr.size() * sizeof(int)));
    CK(cp(v.off_maskoff, v.maskoff.data(), v.maskoff.size() * sizeof(int)));
    CK(cp(v.off_masks, v.masks.data(), v.masks.size()));
    for (int p = 0; p < 2; ++p) CK(cp(v.off_wblocks[p], v.wblocks[p].data(), v.wblocks[p].size() * sizeof(int)));
  }
  int rc = upload_tables(d);
  if (rc) return rc;
  const Level& fl = d->mesh.lv.back();
  if (d->n_seg) CK(cp(d->off_segb, fl.seg_begin.data(), fl.seg_begin.size() * sizeof(int)));
  CK(cp(d->off_fsamp, d->fsamp.data(), d->fsamp.size() * sizeof(FrictionSample)));
  CK(cp(d->off_fsegb, d->fseg_begin.data(), d->fseg_begin.size() * sizeof(int)));
  if (d->d.i_u > 0) {
    const Level& l0 = d->mesh.lv[0];
    CK(cp(d->off_turbidx, l0.turb_idx.data(), l0.turb_idx.size() * sizeof(int)));
    CK(cp(d->off_turbcells, l0.turb_cells.data(), l0.turb_cells.size() * sizeof(int)));
    int rc = upload_modes(d);
    if (rc) return rc;
  }
  return LBM_OK;
}

int reset_force(lbm_domain* d) {
  CK(cudaMemsetAsync(d->base + d->off_accum, 0, 8 * sizeof(double), d->stream));
  CK(cudaMemsetAsync(d->base + d->off_wdone, 0, sizeof(unsigned), d->stream));
  CK(cudaMemsetAsync(d->base + d->off_fmean, 0, std::max<size_t>(1, d->prims.size()) * 4 * sizeof(double), d->stream));
  if (d->n_seg) CK(cudaMemsetAsync(d->base + d->off_segacc, 0, (size_t)d->n_seg * 4 * sizeof(double), d->stream));
  for (int l = 0; l + 1 < d->mesh.L; ++l)
    CK(cudaMemsetAsync(d->base + d->mesh.lv[l].off_ledger, 0, sizeof(LedgerDev), d->stream));
  return LBM_OK;
}

int fill_uniform(lbm_domain* d, double rho, const double u[3]) {
  for (Level& v : d->mesh.lv) {
    double dev[27];
    for (int i = 0; i < 27; ++i) dev[i] = (equilibrium(i, rho, u) - rest_weight(i) - d->ref[i]) * v.scale;
    int rc = launch_fill(d->base + v.off_f, v.esize, v.n_storage, v.B, dev, d->stream);
    if (rc) return fail(rc, cuda_error_string());
  }
  d->parity0 = 0;
  return reset_force(d);
}

int level_parity(const lbm_domain* d, int l) { return l == 0 ? d->parity0 : 0; }

// slot holding the incoming f_i of a cell at the current coarse-step boundary
long long incoming_slot(const Level& v, int parity, int x, int y, int z, int i) {
  if (!parity) return v.addr(x, y, z, i);
  return v.addr(x - cx(i), y - cy(i), z - cz(i), opposite(i));
}

// capture one coarse step of parity p starting from the pending transfers
// `pre`; the host-side pending state is restored afterwards
int capture_one(lbm_domain* d, int p, const std::vector<int>& pre, cudaGraphExec_t* out, std::vector<int>* post) {
  const std::vector<int> keep = d->pend_coal;
  d->pend_coal = pre;
  cudaGraph_t g;
  CK(cudaStreamBeginCapture(d->stream, cudaStreamCaptureModeThreadLocal));
  int rc = advance(d, 0, p);
  cudaError_t e = cudaStreamEndCapture(d->stream, &g);
  *post = d->pend_coal;
  d->pend_coal = keep;
  if (rc) return fail(rc, cuda_error_string());
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  return LBM_OK;
}

// coarse steps per run graph (even counts: a run ends at the parity it
// started with)
constexpr int kRun[2] = {8, 2};

// `steps` coarse steps from a complete state, leaving none pending
int capture_run(lbm_domain* d, int p, int steps, cudaGraphExec_t* out) {
  const std::vector<int> keep = d->pend_coal;
  d->pend_coal.assign(d->mesh.L, -1);
  cudaGraph_t g;
  CK(cudaStreamBeginCapture(d->stream, cudaStreamCaptureModeThreadLocal));
  int rc = LBM_OK;
  for (int k = 0; k < steps && !rc; ++k) rc = advance(d, 0, (p + k) & 1);
  cudaError_t e = cudaStreamEndCapture(d->stream, &g);
  d->pend_coal = keep;
  if (rc) return fail(rc, cuda_error_string());
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  return LBM_OK;
}

int capture_graphs(lbm_domain* d) {
  if (!d->use_graphs || d->stream == nullptr || d->timing) return LBM_OK;
  const std::vector<int> none(d->mesh.L, -1);
  int rc;
  for (int p = 0; p < 2; ++p)
    if (!d->graph[0][p] && (rc = capture_one(d, p, none, &d->graph[0][p], &d->coal_out[p]))) return rc;
  if (d->coal_out[0] == none && d->coal_out[1] == none)
    for (int r = 0; r < 2; ++r)
      for (int p = 0; p < 2; ++p)
        if (!d->graphr[r][p] && (rc = capture_run(d, p, kRun[r], &d->graphr[r][p]))) return rc;
  // the chained form of parity p follows a step of parity 1 - p
  for (int p = 0; p < 2; ++p) {
    d->coal_in[p] = d->coal_out[1 - p];
    if (d->coal_in[p] == none || d->graph[1][p]) continue;
    std::vector<int> post;
    if ((rc = capture_one(d, p, d->coal_in[p], &d->graph[1][p], &post))) return rc;
  }
  return LBM_OK;
}

int mass_device(lbm_domain* d, double* mass, double mom[3], double* bad, int only = -1) {
  double m = 0, p[3] = {0, 0, 0}, b = 0;
  std::vector<double> part;
  for (int l = 0; l < d->mesh.L; ++l) {
    if (only >= 0 && l != only) continue;
    Level& v = d->mesh.lv[l];
    if (!v.n_active) continue;
    int rc = launch_mass(d->base + v.off_f, v.esize, 1.0f / v.scale, d->ref27, d->dev<int>(v.off_nbr),
                         d->dev<int>(v.off_maskoff), d->dev<uint8_t>(v.off_masks), v.n_active, v.B,
                         level_parity(d, l), d->dev<double>(d->off_mpart), d->stream);
    if (rc) return fail(rc, cuda_error_string());
    part.resize((size_t)v.n_active * 5);
    CK(cudaMemcpyAsync(part.data(), d->base + d->off_mpart, part.size() * sizeof(double), cudaMemcpyDeviceToHost,
                       d->stream));
    CK(cudaStreamSynchronize(d->stream));
    double w = std::ldexp(1.0, -3 * l), ml = 0, pl[3] = {0, 0, 0}, bl = 0;
    for (int s = 0; s < v.n_active; ++s) {
      // subtract the cells that are not fluid: k_mass skips them already
      ml += part[5 * s];
      pl[0] += part[5 * s + 1];
      pl[1] += part[5 * s + 2];
      pl[2] += part[5 * s + 3];
      bl += part[5 * s + 4];
    }
    m += w * ml;
    for (int a = 0; a < 3; ++a) p[a] += w * pl[a];
    b += bl;
  }
  if (mass) *mass = m;
  if (mom)
    for (int a = 0; a < 3; ++a) mom[a] = p[a];
  if (bad) *bad = b;
  return LBM_OK;
}

bool valid_level(const lbm_domain* d, int level) { return d && d->built && level >= 0 && level < d->mesh.L; }

long long box_cells(const Level& v) {
  return (long long)(v.rhi[0] - v.rlo[0]) * (v.rhi[1] - v.rlo[1]) * (v.rhi[2] - v.rlo[2]);
}

int download_level(lbm_domain* d, const Level& v, std::vector<uint8_t>& host) {
  host.resize(v.f_elems() * (size_t)v.esize);
  CK(cudaMemcpyAsync(host.data(), d->base + v.off_f, host.size(), cudaMemcpyDeviceToHost, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  return LBM_OK;
}

// stored element k decoded and unscaled: f - w - r of the population it holds
// (r the storage reference, zero for FP32)
double stored_dev(const Level& v, const std::vector<uint8_t>& host, long long k) {
  if (v.esize == 8) {
    double x;
    std::memcpy(&x, host.data() + 8 * k, 8);
    return x;
  }
  if (v.esize == 2) {
    uint16_t h;
    std::memcpy(&h, host.data() + 2 * k, 2);
    return (double)half_bits_to_float(h) / v.scale;
  }
  float x;
  std::memcpy(&x, host.data() + 4 * k, 4);
  return x;
}

void store_dev(const Level& v, std::vector<uint8_t>& host, long long k, double dev) {
  if (v.esize == 8) {
    std::memcpy(host.data() + 8 * k, &dev, 8);
    return;
  }
  if (v.esize == 2) {
    const uint16_t h = float_to_half_bits((float)(dev * v.scale));
    std::memcpy(host.data() + 2 * k, &h, 2);
  } else {
    const float x = (float)dev;
    std::memcpy(host.data() + 4 * k, &x, 4);
  }
}

}  // namespace

extern "C" {

const char* lbm_last_error(void) { return g_error.c_str(); }

const char* lbm_status_string(int s) {
  switch (s) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "out of memory";
    case LBM_ECUDA: return "CUDA error";
    case LBM_EUNSTABLE: return "unstable: non-finite or out-of-range density";
    case LBM_ESTATE: return "call out of order";
    case LBM_ETIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

int lbm_create_domain(const lbm_domain_desc* desc, void* cuda_stream, lbm_domain** out) try {
  if (!desc || !out) return fail(LBM_EINVAL, "null argument");
  *out = nullptr;
  const lbm_domain_desc& s = *desc;
  if (s.nx < 1 || s.ny < 1 || s.nz < 1 || s.levels < 1 || s.levels > 6 || (s.block != 8 && s.block != 16))
    return fail(LBM_EINVAL, "domain size, levels (1..6) or block (8|16) out of range");
  if ((long long)s.nx * s.ny * s.nz > (1LL << 34)) return fail(LBM_EINVAL, "domain too large");
  if (s.bc[0] != LBM_BC_PERIODIC && s.bc[0] != LBM_BC_INOUT) return fail(LBM_EINVAL, "x faces: periodic or in/out");
  for (int a = 1; a < 3; ++a)
    if (s.bc[a] != LBM_BC_PERIODIC && s.bc[a] != LBM_BC_SLIP && s.bc[a] != LBM_BC_INFLOW)
      return fail(LBM_EINVAL, "y/z faces: periodic, slip or inflow");
  if (!(std::fabs(s.u_in) < 0.3)) return fail(LBM_EINVAL, "inflow speed must be below 0.3");
  if (!(s.i_u >= 0.0 && s.i_u <= 0.5)) return fail(LBM_EINVAL, "inflow turbulence intensity must lie in [0, 0.5]");
  if (s.i_u > 0 && s.bc[0] != LBM_BC_INOUT) return fail(LBM_EINVAL, "turbulent inflow needs the in/out x faces");
  if (s.precision != LBM_FP64 && s.precision != LBM_FP32 && s.precision != LBM_FP16_DEV)
    return fail(LBM_EINVAL, "precision must be LBM_FP64, LBM_FP32 or LBM_FP16_DEV");
  if (s.precision == LBM_FP64 && s.i_u > 0)
    return fail(LBM_EINVAL, "turbulent inflow needs FP32 or FP16 storage");
  if (!(s.omega2 > 0 && s.omega2 < 2)) return fail(LBM_EINVAL, "omega2 must lie in (0, 2)");
  auto* d = new (std::nothrow) lbm_domain();
  if (!d) return fail(LBM_ENOMEM, "host allocation");
  d->d = s;
  d->stream = (cudaStream_t)cuda_stream;
  if (s.precision == LBM_FP16_DEV) {
    d->even_variant = LBM_EVEN_PAIRS;
    d->odd_variant = LBM_ODD_PAIRS;
  }
  *out = d;
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_set_geometry_prims(lbm_domain* d, const int* kind, const double* params, int n) try {
  if (!d || n < 0 || (n > 0 && (!kind || !params))) return fail(LBM_EINVAL, "bad primitives");
  if (d->base) return fail(LBM_ESTATE, "geometry is fixed once memory is bound");
  d->prims.clear();
  for (int k = 0; k < n; ++k) {
    if (kind[k] < 0 || kind[k] > 2) return fail(LBM_EINVAL, "primitive kind must be 0, 1 or 2");
    Prim p{kind[k], {}};
    std::memcpy(p.p, params + 8 * k, 8 * sizeof(double));
    d->prims.push_back(p);
  }
  if (!d->have_tree) d->H = 0;
  return build(d);
} catch (...) {
  return exception_status();
}

int lbm_set_geometry_segments(lbm_domain* d, const double* seg, int n) try {
  if (!d || n < 0 || (n > 0 && !seg)) return fail(LBM_EINVAL, "bad segments");
  if (d->base) return fail(LBM_ESTATE, "geometry is fixed once memory is bound");
  d->tree.seg.assign(seg, seg + 8 * (size_t)n);
  d->have_tree = true;
  d->prims.clear();
  for (int k = 0; k < n; ++k) {
    if (!(seg[8 * k + 6] > 0)) return fail(LBM_EINVAL, "segment diameter must be positive");
    Prim p{0, {}};
    std::memcpy(p.p, seg + 8 * k, 8 * sizeof(double));
    d->prims.push_back(p);
  }
  d->H = n ? tree_height(d->tree) : 0.0;
  d->A_x = n ? frontal_area(d->tree, 0.125) : 0.0;
  return build(d);
} catch (...) {
  return exception_status();
}

int lbm_set_geometry(lbm_domain* d, const lbm_tree_desc* t) try {
  if (!d || !t) return fail(LBM_EINVAL, "null argument");
  if (!(t->trunk_cells > 0)) return fail(LBM_EINVAL, "trunk_cells must be positive");
  Tree tr;
  int rc = build_lsystem(*t, &tr);
  if (rc) return fail(rc, "bad L-system parameters");
  if (tr.count() > 0) {
    const int fin = 1 << (d->d.levels - 1);
    double shift0[3] = {0, 0, 0};
    tree_affine(&tr, t->trunk_cells / t->s0, shift0);
    double c[3];
    tree_centroid(tr, c);
    double target[3] = {d->d.nx * fin / 4.0, d->d.ny * fin / 2.0, d->d.nz * fin / 2.0};
    double sh[3] = {target[0] - c[0], target[1] - c[1], target[2] - c[2]};
    tree_affine(&tr, 1.0, sh);
  }
  return lbm_set_geometry_segments(d, tr.seg.data(), tr.count());
} catch (...) {
  return exception_status();
}

int lbm_memory_requirements(const lbm_domain* d, size_t* bytes) try {
  if (!d || !bytes) return fail(LBM_EINVAL, "null argument");
  if (!d->built) return fail(LBM_ESTATE, "set the geometry first");
  *bytes = d->need;
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_memory_breakdown(const lbm_domain* d, size_t* populations, size_t* uploaded) try {
  if (!d) return fail(LBM_EINVAL, "null argument");
  if (!d->built) return fail(LBM_ESTATE, "set the geometry first");
  if (populations) {
    size_t p = 0;
    for (const Level& v : d->mesh.lv) p += v.f_elems() * (size_t)v.esize;
    *populations = p;
  }
  if (uploaded) *uploaded = upload_bytes(d);
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_bind_memory(lbm_domain* d, void* ptr, size_t bytes) try {
  if (!d || !ptr) return fail(LBM_EINVAL, "null argument");
  if (!d->built) return fail(LBM_ESTATE, "set the geometry first");
  if (bytes < d->need) return fail(LBM_ENOMEM, "bound buffer smaller than lbm_memory_requirements");
  if ((uintptr_t)ptr & 255) return fail(LBM_EINVAL, "bound buffer must be 256-byte aligned");
  free_graphs(d);
  d->base = (char*)ptr;
  pin_tables(d);
  int rc = prepare_kernels();
  if (rc) return fail(rc, cuda_error_string());
  rc = upload(d);
  if (rc) return rc;
  double u[3] = {d->d.u_in, 0, 0};
  if ((rc = fill_uniform(d, 1.0, u))) return rc;
  d->steps = 0;
  return set_tick(d);
} catch (...) {
  return exception_status();
}

int lbm_init_uniform(lbm_domain* d, double rho, const double u[3]) try {
  if (!d || !u) return fail(LBM_EINVAL, "null argument");
  if (!d->base) return fail(LBM_ESTATE, "bind memory first");
  int rc = fill_uniform(d, rho, u);
  if (rc) return rc;
  d->steps = 0;
  return set_tick(d);
} catch (...) {
  return exception_status();
}

int lbm_init_field(lbm_domain* d, int level, const double* rho, const double* u, size_t n) try {
  if (!d || !rho || !u) return fail(LBM_EINVAL, "null argument");
  if (!d->base) return fail(LBM_ESTATE, "bind memory first");
  if (!valid_level(d, level)) return fail(LBM_EINVAL, "bad level");
  Level& v = d->mesh.lv[level];
  if ((long long)n != box_cells(v)) return fail(LBM_EINVAL, "cell count does not match the level's box");
  std::vector<uint8_t> host;
  int rc = download_level(d, v, host);
  if (rc) return rc;
  const int par = level_parity(d, level);
  size_t k = 0;
  for (int z = v.rlo[2]; z < v.rhi[2]; ++z)
    for (int y = v.rlo[1]; y < v.rhi[1]; ++y)
      for (int x = v.rlo[0]; x < v.rhi[0]; ++x, ++k) {
        if (v.cell_type(x, y, z) != FLUID) continue;
        for (int i = 0; i < kQ; ++i)
          store_dev(v, host, incoming_slot(v, par, x, y, z, i),
                    equilibrium(i, rho[k], u + 3 * k) - rest_weight(i) - d->ref[i]);
      }
  CK(cudaMemcpyAsync(d->base + v.off_f, host.data(), host.size(), cudaMemcpyHostToDevice, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_step(lbm_domain* d, int n) try {
  if (!d || n < 0) return fail(LBM_EINVAL, "bad argument");
  if (!d->base) return fail(LBM_ESTATE, "bind memory first");
  int rc = capture_graphs(d);
  if (rc) return rc;
  for (int k = 0; k < n; ++k) {
    const int p = d->parity0;
    bool ran = false;
    for (int r = 0; r < 2 && !ran; ++r)
      if (d->graphr[r][p] && !d->timing && k + kRun[r] <= n && d->watchdog <= 0 && !any_pending(d)) {
        CK(cudaGraphLaunch(d->graphr[r][p], d->stream));
        d->steps += kRun[r];
        k += kRun[r] - 1;  // an even run: the parity is back to p
        ran = true;
      }
    if (ran) continue;
    if (d->graph[0][p] && !d->timing) {
      // a step that follows one in this call starts with the transfers that
      // one left pending (the chained graph), else from a complete state
      const bool chain = any_pending(d);
      if (chain && (d->pend_coal != d->coal_in[p] || !d->graph[1][p]) && (rc = flush_coalesce(d)))
        return fail(rc, cuda_error_string());
      CK(cudaGraphLaunch(d->graph[any_pending(d) ? 1 : 0][p], d->stream));
      d->pend_coal = d->coal_out[p];
    } else {
      if ((rc = advance(d, 0, p))) return fail(rc, cuda_error_string());
    }
    d->parity0 ^= 1;
    d->steps++;
    if (d->watchdog > 0 && d->steps % d->watchdog == 0) {
      double bad = 0;
      if ((rc = flush_coalesce(d))) return fail(rc, cuda_error_string());
      if ((rc = mass_device(d, nullptr, nullptr, &bad))) return rc;
      d->last_status = bad > 0 ? LBM_EUNSTABLE : LBM_OK;
      if (bad > 0) return fail(LBM_EUNSTABLE, "watchdog: non-finite or out-of-range density");
    }
  }
  if ((rc = flush_coalesce(d))) return fail(rc, cuda_error_string());
  return d->last_status;
} catch (...) {
  return exception_status();
}

int lbm_drag_enqueue(lbm_domain* d, double host_acc[8]) try {
  if (!d || !host_acc) return fail(LBM_EINVAL, "null argument");
  if (!d->base) return fail(LBM_ESTATE, "bind memory first");
  CK(cudaMemcpyAsync(host_acc, d->base + d->off_accum, 8 * sizeof(double), cudaMemcpyDeviceToHost, d->stream));
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_drag_decode(const lbm_domain* d, const double acc[8], double last[3], double mean[3], double* c_d) try {
  if (!d || !acc) return fail(LBM_EINVAL, "null argument");
  if (acc[7] != 0.0) return fail(LBM_ETIMEOUT, "a bounded device wait gave up (collide staging)");
  if (last)
    for (int a = 0; a < 3; ++a) last[a] = acc[a];
  if (mean)
    for (int a = 0; a < 3; ++a) mean[a] = acc[6] > 0 ? acc[3 + a] / acc[6] : 0.0;
  if (c_d) {
    double u = d->d.u_in;
    *c_d = (d->A_x > 0 && u != 0) ? acc[0] / (0.5 * u * u * d->A_x) : std::numeric_limits<double>::quiet_NaN();
  }
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_drag(lbm_domain* d, double last[3], double mean[3], double* c_d) try {
  if (!d) return fail(LBM_EINVAL, "null argument");
  if (!d->base) return fail(LBM_ESTATE, "bind memory first");
  double acc[8];
  CK(cudaMemcpyAsync(acc, d->base + d->off_accum, sizeof acc, cudaMemcpyDeviceToHost, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  return lbm_drag_decode(d, acc, last, mean, c_d);
} catch (...) {
  return exception_status();
}

int lbm_reset_force(lbm_domain* d) try {
  if (!d) return fail(LBM_EINVAL, "null argument");
  if (!d->base) return fail(LBM_ESTATE, "bind memory first");
  return reset_force(d);
} catch (...) {
  return exception_status();
}

int lbm_get_populations(lbm_domain* d, int level, double* f, size_t n) try {
  if (!d || !f) return fail(LBM_EINVAL, "null argument");
  if (!d->base) return fail(LBM_ESTATE, "bind memory first");
  if (!valid_level(d, level)) return fail(LBM_EINVAL, "bad level");
  Level& v = d->mesh.lv[level];
  if ((long long)n != box_cells(v)) return fail(LBM_EINVAL, "cell count does not match the level's box");
  std::vector<uint8_t> host;
  int rc = download_level(d, v, host);
  if (rc) return rc;
  const int par = level_parity(d, level);
  size_t k = 0;
  for (int z = v.rlo[2]; z < v.rhi[2]; ++z)
    for (int y = v.rlo[1]; y < v.rhi[1]; ++y)
      for (int x = v.rlo[0]; x < v.rhi[0]; ++x, ++k) {
        bool fl = v.cell_type(x, y, z) == FLUID;
        for (int i = 0; i < kQ; ++i)
          f[27 * k + i] = fl ? rest_weight(i) + d->ref[i] + stored_dev(v, host, incoming_slot(v, par, x, y, z, i))
                             : std::numeric_limits<double>::quiet_NaN();
      }
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_get_populations_window(lbm_domain* d, int level, const int lo[3], const int hi[3], double* f,
                               size_t n) try {
  if (!d || !f || !lo || !hi) return fail(LBM_EINVAL, "null argument");
  if (!d->base) return fail(LBM_ESTATE, "bind memory first");
  if (!valid_level(d, level)) return fail(LBM_EINVAL, "bad level");
  const Level& v = d->mesh.lv[level];
  long long cells = 1;
  for (int a = 0; a < 3; ++a) {
    if (lo[a] < 0 || lo[a] >= hi[a] || hi[a] > v.rhi[a] - v.rlo[a])
      return fail(LBM_EINVAL, "window empty or outside the level's box");
    cells *= hi[a] - lo[a];
  }
  if ((long long)n != cells) return fail(LBM_EINVAL, "cell count does not match the window");
  const int par = level_parity(d, level);
  // the stored element each (cell, direction) reads, -1 for cells that are not fluid
  std::vector<long long> slot((size_t)cells * kQ, -1), uniq;
  uniq.reserve(slot.size());
  size_t k = 0;
  for (int z = lo[2]; z < hi[2]; ++z)
    for (int y = lo[1]; y < hi[1]; ++y)
      for (int x = lo[0]; x < hi[0]; ++x, ++k) {
        const int gx = v.rlo[0] + x, gy = v.rlo[1] + y, gz = v.rlo[2] + z;
        if (v.cell_type(gx, gy, gz) != FLUID) continue;
        for (int i = 0; i < kQ; ++i) {
          const long long e = incoming_slot(v, par, gx, gy, gz, i);
          if (e < 0 || e >= (long long)v.f_elems()) return fail(LBM_ESTATE, "fluid cell without storage");
          slot[kQ * k + i] = e;
          uniq.push_back(e);
        }
      }
  std::sort(uniq.begin(), uniq.end());
  uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
  // one copy per run of consecutive elements
  std::vector<uint8_t> host(uniq.size() * (size_t)v.esize);
  for (size_t a = 0; a < uniq.size();) {
    size_t b = a + 1;
    while (b < uniq.size() && uniq[b] == uniq[b - 1] + 1) ++b;
    CK(cudaMemcpyAsync(host.data() + a * v.esize, d->base + v.off_f + (size_t)uniq[a] * v.esize,
                       (b - a) * (size_t)v.esize, cudaMemcpyDeviceToHost, d->stream));
    a = b;
  }
  CK(cudaStreamSynchronize(d->stream));
  for (size_t c = 0; c < (size_t)cells; ++c)
    for (int i = 0; i < kQ; ++i) {
      const long long e = slot[kQ * c + i];
      if (e < 0) {
        f[kQ * c + i] = std::numeric_limits<double>::quiet_NaN();
        continue;
      }
      const long long pos = std::lower_bound(uniq.begin(), uniq.end(), e) - uniq.begin();
      f[kQ * c + i] = rest_weight(i) + d->ref[i] + stored_dev(v, host, pos);
    }
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_get_velocity(lbm_domain* d, int level, double* rho, double* u, size_t n) try {
  if (!d || !rho || !u) return fail(LBM_EINVAL, "null argument");
  if (!valid_level(d, level)) return fail(LBM_EINVAL, "bad level");
  std::vector<double> f(n * 27);
  int rc = lbm_get_populations(d, level, f.data(), n);
  if (rc) return rc;
  for (size_t k = 0; k < n; ++k) {
    double r = 0, j[3] = {0, 0, 0};
    for (int i = 0; i < kQ; ++i) {
      double v = f[27 * k + i];
      r += v;
      j[0] += cx(i) * v;
      j[1] += cy(i) * v;
      j[2] += cz(i) * v;
    }
    rho[k] = r;
    for (int a = 0; a < 3; ++a) u[3 * k + a] = j[a] / r;
  }
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_mass(lbm_domain* d, double* mass, double mom[3]) try {
  if (!d) return fail(LBM_EINVAL, "null argument");
  if (!d->base) return fail(LBM_ESTATE, "bind memory first");
  return mass_device(d, mass, mom, nullptr);
} catch (...) {
  return exception_status();
}

int lbm_mass_noalloc(lbm_domain* d, double* mass, double mom[3]) try {
  if (!d) return fail(LBM_EINVAL, "null argument");
  if (!d->base) return fail(LBM_ESTATE, "bind memory first");
  for (const Level& v : d->mesh.lv)
    if (v.n_active > noalloc_max_blocks())
      return fail(LBM_EINVAL, "a level has more active blocks than lbm_mass_noalloc supports (" +
                                  std::to_string(noalloc_max_blocks()) + ")");
  double* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc) return fail(rc, cuda_error_string());
  double m = 0, p[3] = {0, 0, 0};
  for (int l = 0; l < d->mesh.L; ++l) {
    Level& v = d->mesh.lv[l];
    if (!v.n_active) continue;
    rc = launch_mass_noalloc(d->base + v.off_f, v.esize, 1.0f / v.scale, d->ref27, d->dev<int>(v.off_nbr),
                             d->dev<int>(v.off_maskoff), d->dev<uint8_t>(v.off_masks), v.n_active, v.B,
                             level_parity(d, l), scratch, d->stream);
    if (rc) return fail(rc, cuda_error_string());
    double tot[5];
    CK(cudaMemcpyAsync(tot, scratch + (size_t)noalloc_max_blocks() * 5, sizeof tot, cudaMemcpyDeviceToHost,
                       d->stream));
    CK(cudaStreamSynchronize(d->stream));
    const double w = std::ldexp(1.0, -3 * l);
    m += w * tot[0];
    for (int a = 0; a < 3; ++a) p[a] += w * tot[1 + a];
  }
  if (mass) *mass = m;
  if (mom)
    for (int a = 0; a < 3; ++a) mom[a] = p[a];
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_level_mass(lbm_domain* d, int level, double* mass, double mom[3]) try {
  if (!d) return fail(LBM_EINVAL, "null argument");
  if (!d->base) return fail(LBM_ESTATE, "bind memory first");
  if (!valid_level(d, level)) return fail(LBM_EINVAL, "bad level");
  return mass_device(d, mass, mom, nullptr, level);
} catch (...) {
  return exception_status();
}

int lbm_set_interface_ledger(lbm_domain* d, int on) try {
  if (!d) return fail(LBM_EINVAL, "null argument");
  if (d->ledger != (on != 0)) {
    free_graphs(d);
    d->ledger = on != 0;
    if (d->base)
      for (int l = 0; l + 1 < d->mesh.L; ++l)
        CK(cudaMemsetAsync(d->base + d->mesh.lv[l].off_ledger, 0, sizeof(LedgerDev), d->stream));
  }
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_interface_ledger(lbm_domain* d, int level, double last[12], double total[12], long long* steps) try {
  if (!d) return fail(LBM_EINVAL, "null argument");
  if (!d->base) return fail(LBM_ESTATE, "bind memory first");
  if (!valid_level(d, level) || level + 1 >= d->mesh.L) return fail(LBM_EINVAL, "no interface below this level");
  LedgerDev h;
  CK(cudaMemcpyAsync(&h, d->base + d->mesh.lv[level].off_ledger, sizeof h, cudaMemcpyDeviceToHost, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  for (int k = 0; k < kLedgerVals; ++k) {
    if (last) last[k] = h.last[k];
    if (total) total[k] = h.total[k];
  }
  if (steps) *steps = (long long)h.steps;
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_level_info(const lbm_domain* d, int level, int lo[3], int hi[3], long long* n_fluid, long long* n_links,
                   long long* n_active_blocks) try {
  if (!valid_level(d, level)) return fail(LBM_EINVAL, "bad level or geometry not set");
  const Level& v = d->mesh.lv[level];
  for (int a = 0; a < 3; ++a) {
    if (lo) lo[a] = v.rlo[a];
    if (hi) hi[a] = v.rhi[a];
  }
  if (n_fluid) *n_fluid = v.n_fluid;
  if (n_links) *n_links = (long long)v.links.size();
  if (n_active_blocks) *n_active_blocks = v.n_active;
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_geometry_info(const lbm_domain* d, double* height, double* area, int* nseg, double* nu_f) try {
  if (!d || !d->built) return fail(LBM_ESTATE, "geometry not set");
  if (height) *height = d->H;
  if (area) *area = d->A_x;
  if (nseg) *nseg = d->have_tree ? d->tree.count() : 0;
  if (nu_f) *nu_f = d->nu_f;
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_get_cell_types(const lbm_domain* d, int level, unsigned char* out, size_t n) try {
  if (!out || !valid_level(d, level)) return fail(LBM_EINVAL, "bad argument");
  const Level& v = d->mesh.lv[level];
  if ((long long)n != box_cells(v)) return fail(LBM_EINVAL, "cell count does not match the level's box");
  // blocks without storage hold no fluid cell: inside the next finer level's
  // box they are covered by it, elsewhere (the finest level) solid
  const Level* fine = level + 1 < d->mesh.L ? &d->mesh.lv[level + 1] : nullptr;
  auto under_fine = [&](int x, int y, int z) {
    if (!fine) return false;
    const int c[3] = {x, y, z};
    for (int a = 0; a < 3; ++a)
      if (2 * c[a] < fine->rlo[a] || 2 * c[a] + 1 >= fine->rhi[a]) return false;
    return true;
  };
  size_t k = 0;
  for (int z = v.rlo[2]; z < v.rhi[2]; ++z)
    for (int y = v.rlo[1]; y < v.rhi[1]; ++y)
      for (int x = v.rlo[0]; x < v.rhi[0]; ++x, ++k) {
        CellType t = v.cell_type(x, y, z);
        if (t == OUTSIDE) t = under_fine(x, y, z) ? COVERED : SOLID;
        out[k] = (unsigned char)t;
      }
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_get_links(const lbm_domain* d, int level, long long* cell, int* dir, double* q, size_t n,
                  long long* count) try {
  if (!valid_level(d, level)) return fail(LBM_EINVAL, "bad level or geometry not set");
  const Level& v = d->mesh.lv[level];
  if (count) *count = (long long)v.links.size();
  if (!cell || !dir || !q) return LBM_OK;
  const long long nx = v.rhi[0] - v.rlo[0], ny = v.rhi[1] - v.rlo[1];
  for (size_t k = 0; k < v.links.size() && k < n; ++k) {
    const Link& L = v.links[k];
    cell[k] = (L.x - v.rlo[0]) + nx * ((L.y - v.rlo[1]) + ny * (L.z - v.rlo[2]));
    dir[k] = L.dir;
    q[k] = L.q;
  }
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_get_link_branches(const lbm_domain* d, int level, int* branch, size_t n, long long* count) try {
  if (!valid_level(d, level)) return fail(LBM_EINVAL, "bad level or geometry not set");
  const Level& v = d->mesh.lv[level];
  if (count) *count = (long long)v.links.size();
  if (branch)
    for (size_t k = 0; k < v.links.size() && k < n; ++k) branch[k] = v.links[k].seg;
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_get_segments(const lbm_domain* d, double* seg, int n, int* count) try {
  if (!d) return fail(LBM_EINVAL, "null argument");
  int c = d->have_tree ? d->tree.count() : 0;
  if (count) *count = c;
  if (seg)
    for (int k = 0; k < c && k < n; ++k) std::memcpy(seg + 8 * k, &d->tree.seg[8 * k], 8 * sizeof(double));
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_set_branch_forces(lbm_domain* d, int on) try {
  if (!d) return fail(LBM_EINVAL, "null argument");
  if (d->branch_forces != (on != 0)) free_graphs(d);
  d->branch_forces = on != 0;
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_get_branch_forces(lbm_domain* d, double* mean, int n, long long* steps) try {
  if (!d) return fail(LBM_EINVAL, "null argument");
  if (!d->base) return fail(LBM_ESTATE, "bind memory first");
  if (n < d->n_seg) return fail(LBM_EINVAL, "capacity below the number of branches");
  std::vector<double> acc((size_t)d->n_seg * 4);
  if (d->n_seg) {
    CK(cudaMemcpyAsync(acc.data(), d->base + d->off_segacc, acc.size() * sizeof(double), cudaMemcpyDeviceToHost,
                       d->stream));
    CK(cudaStreamSynchronize(d->stream));
  }
  long long cnt = d->n_seg ? (long long)acc[3] : 0;
  for (int k = 0; k < d->n_seg; ++k)
    for (int a = 0; a < 3; ++a) mean[3 * k + a] = acc[4 * k + 3] > 0 ? acc[4 * k + a] / acc[4 * k + 3] : 0.0;
  if (steps) *steps = cnt;
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_branch_table(const lbm_domain* d, double* rows, int n, int* count) try {
  if (!d || !d->built) return fail(LBM_ESTATE, "geometry not set");
  if (!d->have_tree) return fail(LBM_ESTATE, "no tree: set the geometry from a tree or segments");
  std::vector<double> tab;
  branch_table(d->tree, d->d.u_in, d->nu_f, d->H, d->d.i_u, &tab);
  const int c = d->tree.count();
  if (count) *count = c;
  if (rows) {
    if (n < c) return fail(LBM_EINVAL, "capacity below the number of branches");
    std::memcpy(rows, tab.data(), tab.size() * sizeof(double));
  }
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_branch_coefficients(lbm_domain* d, double* c_drag, double* c_fric, int n, double* cd, double* cf) try {
  if (!d) return fail(LBM_EINVAL, "null argument");
  if (!d->base) return fail(LBM_ESTATE, "bind memory first");
  if (!d->have_tree) return fail(LBM_ESTATE, "no tree: set the geometry from a tree or segments");
  const int nb = d->tree.count();
  if ((c_drag || c_fric) && n < nb) return fail(LBM_EINVAL, "capacity below the number of branches");
  const double u = d->d.u_in, q = 0.5 * u * u;
  if (!(q > 0)) return fail(LBM_ESTATE, "no inflow speed to normalise by");
  std::vector<double> fb((size_t)std::max(1, nb) * 3), fr((size_t)std::max(1, nb) * 3);
  long long steps = 0;
  int rc = lbm_get_branch_forces(d, fb.data(), nb, &steps);
  if (rc) return rc;
  double fmean[3] = {0, 0, 0};
  long long fsteps = 0;
  if (d->friction_mean && (rc = lbm_get_friction_mean(d, fmean, fr.data(), nb, &fsteps))) return rc;
  double mean[3];
  if ((rc = lbm_drag(d, nullptr, mean, nullptr))) return rc;
  // Eq. (2): F_d,k = c_k (rho U^2 / 2) L_k D_k, rho = 1; segment rows hold L and D
  for (int k = 0; k < nb; ++k) {
    const double* sg = &d->tree.seg[8 * (size_t)k];
    const double len = std::sqrt((sg[3] - sg[0]) * (sg[3] - sg[0]) + (sg[4] - sg[1]) * (sg[4] - sg[1]) +
                                 (sg[5] - sg[2]) * (sg[5] - sg[2]));
    const double ld = q * len * sg[6];
    if (c_drag) c_drag[k] = steps > 0 ? fb[3 * (size_t)k] / ld : 0.0;
    if (c_fric) c_fric[k] = fsteps > 0 ? fr[3 * (size_t)k] / ld : 0.0;
  }
  // Eqs. (7), (8) over the same window: C_D = F_x / (rho U^2 A_x / 2), and C_F likewise
  if (cd) *cd = d->A_x > 0 ? mean[0] / (q * d->A_x) : std::numeric_limits<double>::quiet_NaN();
  if (cf) *cf = d->A_x > 0 && fsteps > 0 ? fmean[0] / (q * d->A_x) : std::numeric_limits<double>::quiet_NaN();
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_branch_drag_estimate(const double* rows, int n, const double* c_sect, double area, double* cd_est,
                             double* c_out) try {
  if (!rows || !cd_est || n < 0 || !(area > 0)) return fail(LBM_EINVAL, "bad argument");
  double sum = 0;
  for (int k = 0; k < n; ++k) {
    const double* r = rows + LBM_BRANCH_COLS * (size_t)k;
    const double c = c_sect ? c_sect[k] : (1.0 + 10.0 * std::pow(10.0, -2.0 / 3.0 * r[0])) * r[8];
    if (c_out) c_out[k] = c;
    sum += c * r[6] * r[7];
  }
  *cd_est = sum / area;
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_set_inflow_turbulence(lbm_domain* d, int n_modes, double integral_length) try {
  if (!d || n_modes < 1 || n_modes > kMaxModes || integral_length < 0) return fail(LBM_EINVAL, "bad argument");
  if (!(d->d.i_u > 0)) return fail(LBM_ESTATE, "the domain has uniform inflow (i_u = 0)");
  d->n_modes = n_modes;
  d->l_int = integral_length;
  if (d->base) {
    free_graphs(d);
    return upload_modes(d);
  }
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_inflow_modes(const lbm_domain* d, double* modes, int n, int* count) try {
  if (!d) return fail(LBM_EINVAL, "null argument");
  if (!d->built) return fail(LBM_ESTATE, "set the geometry first");
  const int c = d->d.i_u > 0 ? d->n_modes : 0;
  if (count) *count = c;
  if (modes && c) {
    if (n < c) return fail(LBM_EINVAL, "capacity below the number of modes");
    std::vector<double> m;
    make_modes(d, &m);
    for (int k = 0; k < c; ++k)
      for (int j = 0; j < 7; ++j) modes[7 * k + j] = m[(size_t)k * kModeCols + j];
  }
  return LBM_OK;
} catch (...) {
  return exception_status();
}

// sums the per-branch accumulators into total and (optionally) per-branch rows
void friction_rows(const lbm_domain* d, const std::vector<double>& acc, double total[3], double* rows, bool mean,
                   long long* steps) {
  for (int a = 0; a < 3; ++a) total[a] = 0;
  long long cnt = 0;
  for (size_t k = 0; k < d->prims.size(); ++k) {
    const double w = mean ? (acc[4 * k + 3] > 0 ? 1.0 / acc[4 * k + 3] : 0.0) : 1.0;
    cnt = std::max(cnt, (long long)acc[4 * k + 3]);
    for (int a = 0; a < 3; ++a) {
      const double v = acc[4 * k + a] * w;
      total[a] += v;
      if (rows) rows[3 * k + a] = v;
    }
  }
  if (steps) *steps = cnt;
}

int lbm_friction(lbm_domain* d, double force[3], double* per_branch, int n, double* c_f) try {
  if (!d || !force) return fail(LBM_EINVAL, "null argument");
  if (!d->base) return fail(LBM_ESTATE, "bind memory first");
  if (per_branch && n < (int)d->prims.size()) return fail(LBM_EINVAL, "capacity below the number of branches");
  const size_t nb = std::max<size_t>(1, d->prims.size()) * 4;
  CK(cudaMemsetAsync(d->base + d->off_facc, 0, nb * sizeof(double), d->stream));
  int rc = friction_into(d, level_parity(d, d->mesh.L - 1), d->dev<double>(d->off_facc), d->stream);
  if (rc) return fail(rc, cuda_error_string());
  std::vector<double> acc(nb);
  CK(cudaMemcpyAsync(acc.data(), d->base + d->off_facc, nb * sizeof(double), cudaMemcpyDeviceToHost, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  friction_rows(d, acc, force, per_branch, false, nullptr);
  if (c_f) {
    const double u = d->d.u_in;
    *c_f = (d->A_x > 0 && u != 0) ? force[0] / (0.5 * u * u * d->A_x) : std::numeric_limits<double>::quiet_NaN();
  }
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_set_friction_mean(lbm_domain* d, int on) try {
  if (!d) return fail(LBM_EINVAL, "null argument");
  if (d->friction_mean != (on != 0)) free_graphs(d);
  d->friction_mean = on != 0;
  d->mesh.friction = d->friction_mean;
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_get_friction_mean(lbm_domain* d, double mean[3], double* per_branch, int n, long long* steps) try {
  if (!d || !mean) return fail(LBM_EINVAL, "null argument");
  if (!d->base) return fail(LBM_ESTATE, "bind memory first");
  if (per_branch && n < (int)d->prims.size()) return fail(LBM_EINVAL, "capacity below the number of branches");
  const size_t nb = std::max<size_t>(1, d->prims.size()) * 4;
  std::vector<double> acc(nb);
  CK(cudaMemcpyAsync(acc.data(), d->base + d->off_fmean, nb * sizeof(double), cudaMemcpyDeviceToHost, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  friction_rows(d, acc, mean, per_branch, true, steps);
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_friction_samples(const lbm_domain* d, double* rows, int n, int* count) try {
  if (!d || !d->built) return fail(LBM_ESTATE, "set the geometry first");
  const int c = (int)d->fsamp.size();
  if (count) *count = c;
  if (rows) {
    if (n < c) return fail(LBM_EINVAL, "capacity below the number of samples");
    const Level& v = d->mesh.lv.back();
    const int B = v.B;
    auto cell_xyz = [&](int slot, int cell, double* r) {
      const int gi = v.grid_of[slot];
      r[0] = v.org[0] + (gi % v.nb[0]) * B + cell % B;
      r[1] = v.org[1] + ((gi / v.nb[0]) % v.nb[1]) * B + (cell / B) % B;
      r[2] = v.org[2] + (gi / (v.nb[0] * v.nb[1])) * B + cell / (B * B);
    };
    for (int k = 0; k < c; ++k) {
      const FrictionSample& q = d->fsamp[k];
      double* r = rows + 13 * (size_t)k;
      cell_xyz(q.slot[0], q.cell[0], r);
      if (q.slot[1] >= 0) cell_xyz(q.slot[1], q.cell[1], r + 3);
      else r[3] = r[4] = r[5] = -1e9;
      for (int a = 0; a < 3; ++a) r[6 + a] = q.n[a];
      r[9] = q.area;
      r[10] = q.dist[0];
      r[11] = q.slot[1] >= 0 ? q.dist[1] : 0.0;
      r[12] = q.seg;
    }
  }
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_set_overlap(lbm_domain* d, int on) try {
  if (!d) return fail(LBM_EINVAL, "null argument");
  if (d->overlap != (on != 0)) free_graphs(d);
  d->overlap = on != 0;
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_set_overlap_features(lbm_domain* d, int mask) try {
  if (!d || (mask & ~LBM_OVL_ALL)) return fail(LBM_EINVAL, "bad argument");
  if (d->ovl_feat != mask) free_graphs(d);
  d->ovl_feat = mask;
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_get_overlap_features(const lbm_domain* d, int* mask) try {
  if (!d || !mask) return fail(LBM_EINVAL, "null argument");
  *mask = d->ovl_feat;
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_get_overlap(const lbm_domain* d, int* faces, int* walls) try {
  if (!d) return fail(LBM_EINVAL, "null argument");
  if (!d->built) return fail(LBM_ESTATE, "set the geometry first");
  if (faces) *faces = d->mesh.ovl_faces ? 1 : 0;
  if (walls) {
    *walls = 0;
    for (int l = 0; l < d->mesh.L; ++l)
      if (d->mesh.lv[l].ovl_walls) *walls |= 1 << l;
  }
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_set_wide_offsets(lbm_domain* d, int on) try {
  if (!d) return fail(LBM_EINVAL, "null argument");
  const bool change = d->wide_offsets != (on != 0);
  if (change) free_graphs(d);
  d->wide_offsets = on != 0;
  // the tables follow (their device space holds the 64-bit form either way)
  if (change && d->base) return upload_tables(d);
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_set_watchdog(lbm_domain* d, int every) try {
  if (!d || every < 0) return fail(LBM_EINVAL, "bad argument");
  d->watchdog = every;
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_use_graphs(lbm_domain* d, int on) try {
  if (!d) return fail(LBM_EINVAL, "null argument");
  d->use_graphs = on != 0;
  if (!on) free_graphs(d);
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_set_timing(lbm_domain* d, int on) try {
  if (!d) return fail(LBM_EINVAL, "null argument");
  d->timing = on != 0;
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_get_timing(lbm_domain* d, double ms[6], long long launches[6], long long units[6]) try {
  if (!d) return fail(LBM_EINVAL, "null argument");
  if (d->base) CK(cudaStreamSynchronize(d->stream));
  for (auto& r : d->recs) {
    float t = 0;
    CK(cudaEventElapsedTime(&t, r.a, r.b));
    d->ms[r.cls] += t;
    d->launches[r.cls] += 1;
    d->units[r.cls] += r.units;
  }
  d->recs.clear();
  d->pool_used = 0;
  for (int k = 0; k < KC_N; ++k) {
    if (ms) ms[k] = d->ms[k];
    if (launches) launches[k] = d->launches[k];
    if (units) units[k] = d->units[k];
    d->ms[k] = 0;
    d->launches[k] = 0;
    d->units[k] = 0;
  }
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_work_per_step(const lbm_domain* d, long long* cell_updates, int* kernels) try {
  if (!d || !d->built) return fail(LBM_ESTATE, "geometry not set");
  long long cu = 0;
  for (int l = 0; l < d->mesh.L; ++l) cu += d->mesh.lv[l].n_fluid << l;
  if (cell_updates) *cell_updates = cu;
  if (kernels) *kernels = kernels_per_step(d, 0);
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_save(lbm_domain* d, const char* path) try {
  if (!d || !path) return fail(LBM_EINVAL, "null argument");
  if (!d->base) return fail(LBM_ESTATE, "bind memory first");
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return fail(LBM_EINVAL, "cannot open file");
  const char magic[8] = {'L', 'B', 'M', 'S', 'T', 'A', 'T', '1'};
  long long hdr[4] = {(long long)d->need, d->parity0, d->steps, d->mesh.L};
  std::fwrite(magic, 1, 8, fp);
  std::fwrite(hdr, sizeof hdr, 1, fp);
  std::vector<uint8_t> host;
  for (const Level& v : d->mesh.lv) {
    int rc = download_level(d, v, host);
    if (rc) {
      std::fclose(fp);
      return rc;
    }
    std::fwrite(host.data(), 1, host.size(), fp);
  }
  double acc[8];
  cudaError_t e = cudaMemcpyAsync(acc, d->base + d->off_accum, sizeof acc, cudaMemcpyDeviceToHost, d->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
  if (e != cudaSuccess) {
    std::fclose(fp);
    return cuda_fail(e, "cudaMemcpyAsync");
  }
  std::fwrite(acc, sizeof acc, 1, fp);
  bool ok = std::fclose(fp) == 0;
  return ok ? LBM_OK : fail(LBM_EINVAL, "write failed");
} catch (...) {
  return exception_status();
}

int lbm_load(lbm_domain* d, const char* path) try {
  if (!d || !path) return fail(LBM_EINVAL, "null argument");
  if (!d->base) return fail(LBM_ESTATE, "bind memory first");
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return fail(LBM_EINVAL, "cannot open file");
  char magic[8];
  long long hdr[4];
  bool ok = std::fread(magic, 1, 8, fp) == 8 && std::memcmp(magic, "LBMSTAT1", 8) == 0 &&
            std::fread(hdr, sizeof hdr, 1, fp) == 1 && hdr[0] == (long long)d->need && hdr[3] == d->mesh.L &&
            (hdr[1] == 0 || hdr[1] == 1) && hdr[2] >= 0;
  if (!ok) {
    std::fclose(fp);
    return fail(LBM_EINVAL, "state file does not match this domain");
  }
  // the whole file is checked for the size lbm_save writes before anything
  // is copied, so that a truncated file leaves the domain's state unchanged
  long long want = 8 + (long long)sizeof hdr + 8 * (long long)sizeof(double);
  for (const Level& v : d->mesh.lv) want += (long long)(v.f_elems() * (size_t)v.esize);
  const long long here = (long long)ftello(fp);
  if (fseeko(fp, 0, SEEK_END) != 0 || (long long)ftello(fp) != want || fseeko(fp, (off_t)here, SEEK_SET) != 0) {
    std::fclose(fp);
    return fail(LBM_EINVAL, "state file has the wrong size for this domain");
  }
  std::vector<uint8_t> host;
  for (const Level& v : d->mesh.lv) {
    host.resize(v.f_elems() * (size_t)v.esize);
    if (std::fread(host.data(), 1, host.size(), fp) != host.size()) {
      std::fclose(fp);
      return fail(LBM_EINVAL, "truncated state file");
    }
    cudaError_t e = cudaMemcpyAsync(d->base + v.off_f, host.data(), host.size(), cudaMemcpyHostToDevice, d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    if (e != cudaSuccess) {
      std::fclose(fp);
      return cuda_fail(e, "cudaMemcpyAsync");
    }
  }
  double acc[8];
  if (std::fread(acc, sizeof acc, 1, fp) != 1) {
    std::fclose(fp);
    return fail(LBM_EINVAL, "truncated state file");
  }
  std::fclose(fp);
  CK(cudaMemcpyAsync(d->base + d->off_accum, acc, sizeof acc, cudaMemcpyHostToDevice, d->stream));
  CK(cudaStreamSynchronize(d->stream));
  free_graphs(d);
  d->parity0 = (int)hdr[1];
  d->steps = hdr[2];
  return set_tick(d);
} catch (...) {
  return exception_status();
}

void lbm_destroy(lbm_domain* d) try {
  if (!d) return;
  free_graphs(d);
  destroy_side_streams(d);
  unpin_tables(d);
  for (auto e : d->pool) cudaEventDestroy(e);
  delete d;
} catch (...) {
  exception_status();
}


// ---------------------------------------------------------------- schedules and autotuning

namespace {

bool variant_ok(const lbm_domain* d, int odd, int even) {
  if (odd < LBM_ODD_COLUMNS || odd > LBM_ODD_PAIRS_8 || even < LBM_EVEN_DIRECT || even > LBM_EVEN_PAIRS) return false;
  if ((odd == LBM_ODD_PAIRS_7 || odd == LBM_ODD_PAIRS_8) && d->d.block != 16) return false;
  // the FP64 form has one kernel per parity (direct addressing)
  if (d->d.precision == LBM_FP64) return (odd == LBM_ODD_COLUMNS || odd == LBM_ODD_DIRECT) && even == LBM_EVEN_DIRECT;
  const bool staged_ok = d->d.precision == LBM_FP32 && d->d.block == 16;
  if (odd == LBM_ODD_STAGED && !staged_ok) return false;
  if (even == LBM_EVEN_TMA && !staged_ok) return false;
  return true;
}

// CUDA-event time of `steps` coarse steps after one untimed step
int time_steps(lbm_domain* d, int steps, double* ms) {
  int rc = lbm_step(d, 1);
  if (rc) return rc;
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  CK(cudaEventRecord(a, d->stream));
  rc = lbm_step(d, steps);
  CK(cudaEventRecord(b, d->stream));
  CK(cudaEventSynchronize(b));
  float t = 0;
  cudaEventElapsedTime(&t, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms = t / std::max(1, steps);
  return rc;
}

}  // namespace

int lbm_set_schedule(lbm_domain* d, const lbm_schedule* s) try {
  if (!d || !s) return fail(LBM_EINVAL, "null argument");
  if (!variant_ok(d, s->odd_variant, s->even_variant)) return fail(LBM_EINVAL, "variant not available here");
  if (zshift_req(s->z_split_even, d->d.block) == -1 || zshift_req(s->z_split_odd, d->d.block) == -1)
    return fail(LBM_EINVAL, "z splits must be 0 or a power of two up to the block size");
  if (d->odd_variant != s->odd_variant || d->even_variant != s->even_variant || d->z_split_even != s->z_split_even ||
      d->z_split_odd != s->z_split_odd)
    free_graphs(d);
  d->odd_variant = s->odd_variant;
  d->even_variant = s->even_variant;
  d->z_split_even = s->z_split_even;
  d->z_split_odd = s->z_split_odd;
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_get_schedule(const lbm_domain* d, lbm_schedule* s) try {
  if (!d || !s) return fail(LBM_EINVAL, "null argument");
  s->ctas_per_sm = 0;
  s->odd_variant = d->odd_variant;
  s->even_variant = d->even_variant;
  s->z_split_even = d->z_split_even;
  s->z_split_odd = d->z_split_odd;
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_autotune(lbm_domain* d, int steps, lbm_schedule* best, double* ms_per_step) try {
  if (!d || steps < 1) return fail(LBM_EINVAL, "bad argument");
  if (!d->base) return fail(LBM_ESTATE, "bind memory first");
  lbm_schedule b;
  int rc = lbm_get_schedule(d, &b);
  if (rc) return rc;
  double bms = std::numeric_limits<double>::infinity();
  auto try_one = [&](const lbm_schedule& c) -> int {
    int r = lbm_set_schedule(d, &c);
    double ms;
    if (!r) r = time_steps(d, steps, &ms);
    if (!r && ms < bms) {
      bms = ms;
      b = c;
    }
    return r;
  };
  // coordinate search: the kernel variants at the current z splits, then the
  // even step's split, then the odd step's
  const lbm_schedule start = b;
  for (int odd = LBM_ODD_COLUMNS; odd <= LBM_ODD_PAIRS_8; ++odd)
    for (int even = LBM_EVEN_DIRECT; even <= LBM_EVEN_PAIRS; ++even) {
      if (!variant_ok(d, odd, even)) continue;
      lbm_schedule c = start;
      c.odd_variant = odd;
      c.even_variant = even;
      if ((rc = try_one(c))) return rc;
    }
  for (int z = 0; z <= d->d.block; z = z ? 2 * z : 1) {
    lbm_schedule c = b;
    c.z_split_even = z;
    if ((rc = try_one(c))) return rc;
  }
  for (int z = 0; z <= d->d.block; z = z ? 2 * z : 1) {
    lbm_schedule c = b;
    c.z_split_odd = z;
    if ((rc = try_one(c))) return rc;
  }
  rc = lbm_set_schedule(d, &b);
  if (rc) return rc;
  // then the reorderings of the step under that schedule: a few candidate
  // masks, each timed twice over at least 16 steps (their differences are a
  // few per cent)
  if (d->overlap && d->use_graphs) {
    const int kMasks[] = {LBM_OVL_BRANCHES | LBM_OVL_LEVELS | LBM_OVL_TRANSFERS, LBM_OVL_BRANCHES | LBM_OVL_LEVELS,
                          LBM_OVL_ALL & ~LBM_OVL_WALL_SPLIT, LBM_OVL_ALL & ~LBM_OVL_DEFER, LBM_OVL_ALL,
                          LBM_OVL_BRANCHES};
    const int n = std::max(steps, 16);
    double mbest = std::numeric_limits<double>::infinity();
    int mask = d->ovl_feat;
    for (int rep = 0; rep < 2; ++rep)
      for (int k = 0; k < 6; ++k) {
        const int m = kMasks[rep ? 5 - k : k];
        double ms;
        if ((rc = lbm_set_overlap_features(d, m)) || (rc = time_steps(d, n, &ms))) return rc;
        if (ms < mbest) {
          mbest = ms;
          mask = m;
        }
      }
    if ((rc = lbm_set_overlap_features(d, mask))) return rc;
    bms = std::min(bms, mbest);
  }
  if (best) *best = b;
  if (ms_per_step) *ms_per_step = bms;
  return LBM_OK;
} catch (...) {
  return exception_status();
}

}  // extern "C"

// ---------------------------------------------------------------- batches

struct lbm_batch {
  std::vector<lbm_domain*> doms;
  cudaStream_t stream = nullptr;
  int B = 16, half = 0, wide = 0, L = 1, sms = 1;
  std::vector<CollideArgs> descs;          // per (domain, level)
  std::vector<std::vector<int2>> items;    // per depth: (descriptor, block) of every domain with that level
  char* base = nullptr;
  size_t need = 0, off_descs = 0;
  std::vector<size_t> off_items;
  lbm_schedule sched{0, LBM_ODD_COLUMNS, LBM_EVEN_DIRECT, 0, 0};
  bool use_graphs = true;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  // per-domain work of a phase runs on one side stream per domain, joined
  // before the next collide launch (parallel branches in the captured graph)
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> done;
  cudaEvent_t fork = nullptr;
};

namespace {

// run fn(d, stream) for every domain that qualifies, each on its own side
// stream forked from and joined back into the batch stream
template <class F>
int fan_out(lbm_batch* b, F&& fn) {
  CK(cudaEventRecord(b->fork, b->stream));
  for (size_t k = 0; k < b->doms.size(); ++k) {
    CK(cudaStreamWaitEvent(b->side[k], b->fork, 0));
    int rc = fn(b->doms[k], b->side[k]);
    if (rc) return fail(rc, cuda_error_string());
    CK(cudaEventRecord(b->done[k], b->side[k]));
  }
  for (size_t k = 0; k < b->doms.size(); ++k) CK(cudaStreamWaitEvent(b->stream, b->done[k], 0));
  return LBM_OK;
}

void free_batch_graphs(lbm_batch* b) {
  for (auto& g : b->graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

// device descriptors follow the domains' schedules and offsets
void build_descs(lbm_batch* b) {
  b->descs.clear();
  for (lbm_domain* d : b->doms) {
    d->odd_variant = b->sched.odd_variant;
    for (int l = 0; l < d->mesh.L; ++l) b->descs.push_back(collide_args(d, l));
  }
}

// z split of the batch's collide launch at depth l: the schedule's, or the
// automatic rule over all the depth's blocks
int batch_zshift(lbm_batch* b, int l, int parity) {
  const int req = parity ? b->sched.z_split_odd : b->sched.z_split_even;
  if (req) return zshift_req(req, b->B);
  return auto_zshift(b->doms[0]->d, (long long)b->items[l].size(), b->sms, parity);
}

int batch_advance(lbm_batch* b, int l, int parity) {
  const int grid = b->sched.ctas_per_sm > 0 ? b->sched.ctas_per_sm * b->sms : 0;
  int rc = launch_collide_batch(reinterpret_cast<const CollideArgs*>(b->base + b->off_descs),
                                reinterpret_cast<const int2*>(b->base + b->off_items[l]), (int)b->items[l].size(), b->B,
                                parity, b->sched.odd_variant, b->sched.even_variant, b->half, b->wide, grid,
                                batch_zshift(b, l, parity), b->stream);
  if (rc) return fail(rc, cuda_error_string());
  if ((rc = fan_out(b, [&](lbm_domain* d, cudaStream_t s) {
         return l < d->mesh.L ? post_collide(d, l, parity, s, false) : LBM_OK;
       })))
    return rc;
  if (l + 1 < b->L) {
    if ((rc = batch_advance(b, l + 1, 0))) return rc;
    if ((rc = fan_out(b, [&](lbm_domain* d, cudaStream_t s) {
           return l + 1 < d->mesh.L ? iface_transfer(d, l, parity, s, true, true) : LBM_OK;
         })))
      return rc;
    if ((rc = batch_advance(b, l + 1, 1))) return rc;
    if ((rc = fan_out(b, [&](lbm_domain* d, cudaStream_t s) {
           int r = l + 1 < d->mesh.L ? iface_coalesce(d, l, parity, s) : LBM_OK;
           if (!r && l == 0) r = end_coarse_step(d, parity, s);
           return r;
         })))
      return rc;
  } else if (l == 0) {
    if ((rc = fan_out(b, [&](lbm_domain* d, cudaStream_t s) { return end_coarse_step(d, parity, s); }))) return rc;
  }
  return LBM_OK;
}

int upload_descs(lbm_batch* b) {
  build_descs(b);
  CK(cudaMemcpyAsync(b->base + b->off_descs, b->descs.data(), b->descs.size() * sizeof(CollideArgs),
                     cudaMemcpyHostToDevice, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  return LBM_OK;
}

int capture_batch(lbm_batch* b) {
  if (!b->use_graphs || b->stream == nullptr) return LBM_OK;
  for (int p = 0; p < 2; ++p) {
    if (b->graph[p]) continue;
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int rc = batch_advance(b, 0, p);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->graph[p], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  }
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_batch_create(lbm_domain* const* domains, int n, void* cuda_stream, lbm_batch** out) try {
  if (!domains || n < 1 || !out) return fail(LBM_EINVAL, "bad argument");
  *out = nullptr;
  auto* b = new (std::nothrow) lbm_batch();
  if (!b) return fail(LBM_ENOMEM, "host allocation");
  b->stream = (cudaStream_t)cuda_stream;
  for (int k = 0; k < n; ++k) {
    lbm_domain* d = domains[k];
    std::string why;
    if (!d || !d->base) why = "every domain must have bound memory";
    else if (d->d.block != domains[0]->d.block) why = "all domains must share the block size";
    else if (d->d.precision != domains[0]->d.precision) why = "all domains must share the storage precision";
    else if (d->d.precision == LBM_FP64) why = "batches take FP32 or FP16 storage";
    else if (d->parity0 != domains[0]->parity0) why = "all domains must be at the same step parity";
    else if (d->timing) why = "per-class timing must be off";
    for (int j = 0; j < k && why.empty(); ++j)
      if (domains[j] == d) why = "a domain appears twice";
    if (!why.empty()) {
      delete b;
      return fail(LBM_EINVAL, why);
    }
    b->doms.push_back(d);
    b->L = std::max(b->L, d->mesh.L);
    for (const Level& v : d->mesh.lv)
      if (v.f_elems() >= (1LL << 31) || d->wide_offsets) b->wide = 1;
  }
  b->B = domains[0]->d.block;
  b->half = domains[0]->d.precision == LBM_FP16_DEV;
  bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; k < n && ok; ++k) {
    cudaStream_t st;
    cudaEvent_t ev;
    ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) b->side.push_back(st);
    ok = ok && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
    if (ok) b->done.push_back(ev);
  }
  if (!ok) {
    lbm_batch_destroy(b);
    return fail(LBM_ECUDA, "stream or event creation failed");
  }
  int dev = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) b->sms = 1;
  b->items.assign(b->L, {});
  int desc = 0;
  for (lbm_domain* d : b->doms)
    for (int l = 0; l < d->mesh.L; ++l, ++desc)
      for (int s2 = 0; s2 < d->mesh.lv[l].n_active; ++s2) b->items[l].push_back(int2{desc, s2});
  size_t off = 0;
  auto put = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  b->off_descs = put((size_t)desc * sizeof(CollideArgs));
  for (int l = 0; l < b->L; ++l) b->off_items.push_back(put(b->items[l].size() * sizeof(int2)));
  b->need = off;
  *out = b;
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_batch_memory_requirements(const lbm_batch* b, size_t* bytes) try {
  if (!b || !bytes) return fail(LBM_EINVAL, "null argument");
  *bytes = b->need;
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_batch_bind_memory(lbm_batch* b, void* ptr, size_t bytes) try {
  if (!b || !ptr) return fail(LBM_EINVAL, "null argument");
  if (bytes < b->need) return fail(LBM_ENOMEM, "bound buffer smaller than lbm_batch_memory_requirements");
  if ((uintptr_t)ptr & 255) return fail(LBM_EINVAL, "bound buffer must be 256-byte aligned");
  free_batch_graphs(b);
  b->base = (char*)ptr;
  for (int l = 0; l < b->L; ++l)
    if (!b->items[l].empty())
      CK(cudaMemcpyAsync(b->base + b->off_items[l], b->items[l].data(), b->items[l].size() * sizeof(int2),
                         cudaMemcpyHostToDevice, b->stream));
  return upload_descs(b);
} catch (...) {
  return exception_status();
}

int lbm_batch_set_schedule(lbm_batch* b, const lbm_schedule* s) try {
  if (!b || !s) return fail(LBM_EINVAL, "null argument");
  if (s->ctas_per_sm < 0 || s->ctas_per_sm > 64 ||
      (s->odd_variant != LBM_ODD_COLUMNS && s->odd_variant != LBM_ODD_DIRECT && s->odd_variant != LBM_ODD_PAIRS) ||
      (s->even_variant != LBM_EVEN_DIRECT && s->even_variant != LBM_EVEN_PAIRS))
    return fail(LBM_EINVAL,
                "batches take column-pointer, direct or paired odd steps, direct or paired even steps and 0..64 CTAs "
                "per SM");
  if (zshift_req(s->z_split_even, b->B) == -1 || zshift_req(s->z_split_odd, b->B) == -1)
    return fail(LBM_EINVAL, "z splits must be 0 or a power of two up to the block size");
  b->sched = *s;
  free_batch_graphs(b);
  for (lbm_domain* d : b->doms) free_graphs(d);
  if (b->base) return upload_descs(b);
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_batch_get_schedule(const lbm_batch* b, lbm_schedule* s) try {
  if (!b || !s) return fail(LBM_EINVAL, "null argument");
  *s = b->sched;
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_batch_step(lbm_batch* b, int n) try {
  if (!b || n < 0) return fail(LBM_EINVAL, "bad argument");
  if (!b->base) return fail(LBM_ESTATE, "bind memory first");
  const int p0 = b->doms[0]->parity0;
  for (lbm_domain* d : b->doms)
    if (d->parity0 != p0 || !d->base) return fail(LBM_ESTATE, "domains left lockstep or lost their memory");
  int rc = capture_batch(b);
  if (rc) return rc;
  for (int k = 0; k < n; ++k) {
    const int p = b->doms[0]->parity0;
    if (b->graph[p]) {
      CK(cudaGraphLaunch(b->graph[p], b->stream));
    } else if ((rc = batch_advance(b, 0, p))) {
      return rc;
    }
    for (lbm_domain* d : b->doms) {
      d->parity0 ^= 1;
      d->steps++;
    }
  }
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_batch_use_graphs(lbm_batch* b, int on) try {
  if (!b) return fail(LBM_EINVAL, "null argument");
  b->use_graphs = on != 0;
  if (!on) free_batch_graphs(b);
  return LBM_OK;
} catch (...) {
  return exception_status();
}

int lbm_batch_autotune(lbm_batch* b, int steps, lbm_schedule* best, double* ms_per_step) try {
  if (!b || steps < 1) return fail(LBM_EINVAL, "bad argument");
  if (!b->base) return fail(LBM_ESTATE, "bind memory first");
  static const int kCtas[] = {0, 1, 2, 3, 4, 6, 8};
  lbm_schedule bs = b->sched;
  double bms = std::numeric_limits<double>::infinity();
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int rc = LBM_OK;
  auto try_one = [&](const lbm_schedule& s) -> int {
    int r = lbm_batch_set_schedule(b, &s);
    if (!r) r = lbm_batch_step(b, 1);
    if (r) return r;
    cudaEventRecord(e0, b->stream);
    if ((r = lbm_batch_step(b, steps))) return r;
    cudaEventRecord(e1, b->stream);
    cudaEventSynchronize(e1);
    float t = 0;
    cudaEventElapsedTime(&t, e0, e1);
    if (t / steps < bms) {
      bms = t / steps;
      bs = s;
    }
    return LBM_OK;
  };
  // coordinate search: odd variant and persistent grid at the current z
  // splits, then the even step's split, then the odd step's
  const lbm_schedule start = b->sched;
  // the collide variants at one CTA per work unit, then the persistent grid
  // for the best of them, then the z splits
  for (int odd : {(int)LBM_ODD_COLUMNS, (int)LBM_ODD_DIRECT, (int)LBM_ODD_PAIRS})
    for (int even : {(int)LBM_EVEN_DIRECT, (int)LBM_EVEN_PAIRS}) {
      lbm_schedule s = start;
      s.ctas_per_sm = 0;
      s.odd_variant = odd;
      s.even_variant = even;
      if (!rc) rc = try_one(s);
    }
  const lbm_schedule variants = bs;
  for (int c : kCtas) {
    if (c == 0) continue;
    lbm_schedule s = variants;
    s.ctas_per_sm = c;
    if (!rc) rc = try_one(s);
  }
  for (int z = 0; z <= b->B && !rc; z = z ? 2 * z : 1) {
    lbm_schedule s = bs;
    s.z_split_even = z;
    rc = try_one(s);
  }
  for (int z = 0; z <= b->B && !rc; z = z ? 2 * z : 1) {
    lbm_schedule s = bs;
    s.z_split_odd = z;
    rc = try_one(s);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if ((rc = lbm_batch_set_schedule(b, &bs))) return rc;
  if (best) *best = bs;
  if (ms_per_step) *ms_per_step = bms;
  return LBM_OK;
} catch (...) {
  return exception_status();
}

void lbm_batch_destroy(lbm_batch* b) try {
  if (!b) return;
  free_batch_graphs(b);
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (cudaStream_t st : b->side) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (cudaEvent_t ev : b->done) cudaEventDestroy(ev);
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
} catch (...) {
  exception_status();
}

}  // extern "C"
