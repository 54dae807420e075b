// GB300 (sm_103a) kernels of the cumulant LBM step.
//
//  k_collide   fused collision + streaming, in-place AA pattern, one CTA per
//              active block, one thread per (x, y) column walking z (Sec. 2.2:
//              the cumulant LBM of Geier et al. 2015).
//  k_faces     domain faces of level 0 (Sec. 2.3: inflow, zero-gradient
//              outflow; slip or inflow lateral faces).
//  k_walls     Bouzidi linear bounce-back on cut links fused with the
//              momentum-exchange force (Sec. 2.2: interpolated bounce-back,
//              Wen et al. 2014; C_D by Eq. 7): float-float warp sums, FP64
//              CTA partials, and the fixed-order FP64 total by the last CTA
//              (deterministic).
//  k_explode (with the inflow entries) / k_coalesce   refinement-interface
//              transfer of Sec. 2.2's octree refinement (volumetric explode and
//              coalesce, with the FP64 interface ledger).
//  k_fill      equilibrium initialisation; k_mass FP64 mass / momentum.
//
// The step is a bandwidth-bound stencil: every population is read once and
// written once per cell update (2 x 27 x 4 bytes in FP32); no tensor cores.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <type_traits>

#include "collide.cuh"
#include "cumulant.cuh"
#include "internal.h"

namespace lbm {
namespace {

struct Feq27 {
  float v[27];
};
struct Vals27 {  // values of the FP64 form, and fill values of every form
  double v[27];
};

template <typename S, typename E, typename FQ>
__global__ void k_faces(S* __restrict__ f, const E* __restrict__ e, int n, FQ feq) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const E x = e[t];
  if (x.src < 0) Store<S>::st(f, x.dst, feq.v[x.dir]);
  else f[x.dst] = f[x.src];
}

// deviation f_i^eq(rho = 1, u) - w_i of the product-form equilibrium: per
// axis 2/3 - u^2 for c = 0 and (1/3 + u^2 + c u) / 2 for c = +-1
__device__ __forceinline__ float eq_axis(int c, float u) {
  return c == 0 ? 2.0f / 3.0f - u * u : 0.5f * (1.0f / 3.0f + u * u + c * u);
}
__device__ __forceinline__ float eq_dev(int i, float ux, float uy, float uz) {
  const int a = dcx(i), b = dcy(i), c = dcz(i);
  const float w = (a ? 1.0f / 6.0f : 2.0f / 3.0f) * (b ? 1.0f / 6.0f : 2.0f / 3.0f) * (c ? 1.0f / 6.0f : 2.0f / 3.0f);
  return eq_axis(a, ux) * eq_axis(b, uy) * eq_axis(c, uz) - w;
}

// turbulent inflow velocity U e_x + sum_n a_n cos(k_n . (p - U t e_x) + psi_n)
// at the centre p of every cell the faces pull the inflow equilibrium from,
// t = coarse steps done (frozen field carried at U); once per cell and step
__global__ void __launch_bounds__(128) k_turb_velocity(TurbArgs tb) {
  extern __shared__ float sm[];  // the mode table
  for (int k = threadIdx.x; k < tb.n_modes * kModeCols; k += blockDim.x) sm[k] = tb.modes[k];
  __syncthreads();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tb.n_cells) return;
  const float px = tb.cells[4 * t] + 0.5f - tb.u * (float)(*tb.tick);
  const float py = tb.cells[4 * t + 1] + 0.5f, pz = tb.cells[4 * t + 2] + 0.5f;
  float ux = tb.u, uy = 0.0f, uz = 0.0f;
  for (int m = 0; m < tb.n_modes; ++m) {
    const float* r = sm + m * kModeCols;
    const float c = cosf(fmaf(r[0], px, fmaf(r[1], py, fmaf(r[2], pz, r[6]))));
    ux = fmaf(r[3], c, ux);
    uy = fmaf(r[4], c, uy);
    uz = fmaf(r[5], c, uz);
  }
  reinterpret_cast<float4*>(tb.vel)[t] = make_float4(ux, uy, uz, 0.0f);
}

// faces with a turbulent inflow: entries that pull the inflow equilibrium get
// it at their pulled-from cell's velocity of the step (k_turb_velocity)
template <typename S, typename E>
__global__ void __launch_bounds__(256) k_faces_turb(S* __restrict__ f, const E* __restrict__ e, int n,
                                                     TurbArgs tb) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const E x = e[t];
  if (x.src >= 0) {
    f[x.dst] = f[x.src];
    return;
  }
  const float4 v = reinterpret_cast<const float4*>(tb.vel)[tb.idx[t]];
  const float r = tb.shift ? eq_dev(x.dir, tb.u, 0.0f, 0.0f) : 0.0f;
  Store<S>::st(f, x.dst, (eq_dev(x.dir, v.x, v.y, v.z) - r) * tb.scale);
}

__global__ void k_tick(long long* tick) { *tick += 1; }

// Viscous stress of one cell from its pre-collision populations (incoming
// values at the step boundary: own slots on even parity, (x - c_i, ibar) on
// odd parity):
//   Pi^neq = sum_i c c (f_i - f_i^eq) = sum_i c c d_i - (sum_i d_i) I / 3 - j j / rho,
//   sigma' = -(1 - omega1 / 2) dev(Pi^neq)
template <int B, typename S>
__device__ void cell_stress(const S* __restrict__ f, const int* __restrict__ nbr, int slot, int cell, int odd,
                            float om1, float inv_scale, const Ref27& ref, double sg[3][3]) {
  constexpr int C3 = B * B * B;
  const int lx = cell % B, ly = (cell / B) % B, lz = cell / (B * B);
  double sum = 0, j[3] = {0, 0, 0}, P[6] = {0, 0, 0, 0, 0, 0};  // xx yy zz xy xz yz
  for (int i = 0; i < 27; ++i) {
    long long a;
    if (!odd) {
      a = ((long long)slot * 27 + i) * C3 + cell;
    } else {
      const int nx = lx - dcx(i), ny = ly - dcy(i), nz = lz - dcz(i);
      const int bd = block_digit<B>(nx) + 3 * block_digit<B>(ny) + 9 * block_digit<B>(nz);
      const int nc = ((nz & (B - 1)) * B + (ny & (B - 1))) * B + (nx & (B - 1));
      a = ((long long)nbr[(size_t)slot * 27 + bd] * 27 + (26 - i)) * C3 + nc;
    }
    const double d = (double)Store<S>::ld(f, a) * inv_scale + (double)ref.v[i];
    const int cx_ = dcx(i), cy_ = dcy(i), cz_ = dcz(i);
    sum += d;
    j[0] += cx_ * d;
    j[1] += cy_ * d;
    j[2] += cz_ * d;
    P[0] += cx_ * cx_ * d;
    P[1] += cy_ * cy_ * d;
    P[2] += cz_ * cz_ * d;
    P[3] += cx_ * cy_ * d;
    P[4] += cx_ * cz_ * d;
    P[5] += cy_ * cz_ * d;
  }
  const double rho = 1.0 + sum;
  double Q[3][3];
  Q[0][0] = P[0] - sum / 3.0 - j[0] * j[0] / rho;
  Q[1][1] = P[1] - sum / 3.0 - j[1] * j[1] / rho;
  Q[2][2] = P[2] - sum / 3.0 - j[2] * j[2] / rho;
  Q[0][1] = Q[1][0] = P[3] - j[0] * j[1] / rho;
  Q[0][2] = Q[2][0] = P[4] - j[0] * j[2] / rho;
  Q[1][2] = Q[2][1] = P[5] - j[1] * j[2] / rho;
  const double tr = (Q[0][0] + Q[1][1] + Q[2][2]) / 3.0;
  const double c = -(1.0 - 0.5 * (double)om1);
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < 3; ++q) sg[r][q] = c * (Q[r][q] - (r == q ? tr : 0.0));
}

// Friction force of one quadrature point: the stress extrapolated linearly to
// the wall from its two cells (or that of its one cell), tangential traction
// (sigma' n minus its normal part) times the area.  out[3 k .. 3 k + 2].
template <int B, typename S>
__global__ void __launch_bounds__(128) k_friction(const S* __restrict__ f, const FrictionSample* __restrict__ e, int n,
                                                   const int* __restrict__ nbr, int odd, float om1, float inv_scale,
                                                   Ref27 ref, double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const FrictionSample sm = e[t];
  double sa[3][3], sw[3][3];
  cell_stress<B, S>(f, nbr, sm.slot[0], sm.cell[0], odd, om1, inv_scale, ref, sa);
  if (sm.slot[1] >= 0) {
    double sb[3][3];
    cell_stress<B, S>(f, nbr, sm.slot[1], sm.cell[1], odd, om1, inv_scale, ref, sb);
    const double w = (double)sm.dist[0] / ((double)sm.dist[1] - (double)sm.dist[0]);
    for (int r = 0; r < 3; ++r)
      for (int q = 0; q < 3; ++q) sw[r][q] = sa[r][q] + (sa[r][q] - sb[r][q]) * w;
  } else {
    for (int r = 0; r < 3; ++r)
      for (int q = 0; q < 3; ++q) sw[r][q] = sa[r][q];
  }
  const double nv[3] = {sm.n[0], sm.n[1], sm.n[2]};
  double tv[3];
  for (int k = 0; k < 3; ++k) tv[k] = sw[k][0] * nv[0] + sw[k][1] * nv[1] + sw[k][2] * nv[2];
  const double tn = tv[0] * nv[0] + tv[1] * nv[1] + tv[2] * nv[2];
  for (int k = 0; k < 3; ++k) out[3 * (size_t)t + k] = (tv[k] - tn * nv[k]) * (double)sm.area;
}

constexpr int kWallThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// block-wide FP64 sum of three values in a fixed order; result valid in thread 0
template <int NT>
__device__ void block_sum3(double& a, double& b, double& c) {
  __shared__ double s[3][NT / 32];
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_sum(c);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    s[0][w] = a;
    s[1][w] = b;
    s[2][w] = c;
  }
  __syncthreads();
  if (w == 0) {
    a = lane < NT / 32 ? s[0][lane] : 0.0;
    b = lane < NT / 32 ? s[1][lane] : 0.0;
    c = lane < NT / 32 ? s[2][lane] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
  }
}

// float-float value (hi + lo, |lo| <= ulp(hi) / 2) and its exact-error sum
// (Knuth's TwoSum, then Dekker's fast renormalisation): ~2^-44 relative,
// enough for FP64 bookkeeping of the momentum exchange without FP64 math in
// every lane (GB300's FP64 rate is a small fraction of its FP32 rate)
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  const float t = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float h = __fadd_rn(s, t);
  return FF{h, __fsub_rn(t, __fsub_rn(h, s))};
}
__device__ __forceinline__ FF ff_warp_sum(FF v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = ff_add(v, FF{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)});
  return v;
}

// One launch per cut-link table: Bouzidi update, the momentum exchange of
// every link in gauge form g = c_i (f*_i + f_ibar - 2 w_i) (FP32 per link,
// float-float warp sums, FP64 per CTA), and - with `accum` set - the last CTA
// to finish sums the CTA partials in a fixed order into accum[0..6] (the
// 2 w_i terms enter as their exact host-side total `rest`).  `done` counts
// finished CTAs and is reset by the last one.
template <typename S, typename E>
__global__ void __launch_bounds__(kWallThreads) k_walls(S* __restrict__ f, const E* __restrict__ e, int n,
                                                        const double* __restrict__ q64, float inv_scale, Ref27 ref,
                                                        double* __restrict__ partials,
                                                        double* __restrict__ link_force, unsigned* __restrict__ done,
                                                        double* __restrict__ accum, double3 rest) {
  using V = typename Store<S>::V;  // FP32, or FP64 for the double-precision form
  const int t = blockIdx.x * kWallThreads + threadIdx.x;
  V gx = 0, gy = 0, gz = 0;
  if (t < n) {
    const E w = e[t];
    const V fa = Store<S>::ld(f, w.a);  // f*_i(x_f), toward the wall (stored deviation)
    const V q = q64 ? (V)q64[t] : (V)w.q;  // the FP64 form keeps q in FP64
    V out;
    V wi_ref = 1.0f;  // interpolation weight on direction-i populations
    if (w.b < 0) {
      out = fa;  // second fluid node missing: simple bounce-back
    } else if (q < 0.5f) {
      out = 2.0f * q * fa + (1.0f - 2.0f * q) * Store<S>::ld(f, w.b);
    } else {
      const V fc = Store<S>::ld(f, w.c);
      wi_ref = 1.0f / (2.0f * q);
      out = fa * wi_ref + (2.0f * q - 1.0f) / (2.0f * q) * fc;
    }
    // the interpolation weights add up to 1, so relative to the storage
    // reference the result for population ibar carries (r_i - r_ibar) times
    // the weight on the direction-i terms (all of it unless q >= 1/2, where
    // f*_ibar(x_f) takes the rest)
    const int i = w.dir;
    if constexpr (Store<S>::scaled) out += wi_ref * (ref.v[i] - ref.v[26 - i]) / inv_scale;
    Store<S>::st(f, w.dst, out);
    // gauge-form momentum exchange of the link, resting wall: full
    // populations minus the rest weights, (f*_i - w_i) + (f_ibar - w_ibar)
    V sum = fa + out;
    if constexpr (Store<S>::scaled) sum = fmaf(sum, inv_scale, ref.v[i] + ref.v[26 - i]);
    gx = dcx(i) ? (dcx(i) > 0 ? sum : -sum) : (V)0;
    gy = dcy(i) ? (dcy(i) > 0 ? sum : -sum) : (V)0;
    gz = dcz(i) ? (dcz(i) > 0 ? sum : -sum) : (V)0;
    // per-link force for the branch sums: a branch's links do not close a
    // surface, so the reference pressure must not enter
    if (link_force) {
      link_force[3 * (size_t)t] = gx;
      link_force[3 * (size_t)t + 1] = gy;
      link_force[3 * (size_t)t + 2] = gz;
    }
  }
  // warp sums: float-float in FP32 (about 2^-44 relative), plain FP64 for the
  // double-precision form
  double wx, wy, wz;
  if constexpr (sizeof(V) == 4) {
    const FF sx = ff_warp_sum(FF{gx, 0.0f}), sy = ff_warp_sum(FF{gy, 0.0f}), sz = ff_warp_sum(FF{gz, 0.0f});
    wx = (double)sx.hi + (double)sx.lo;
    wy = (double)sy.hi + (double)sy.lo;
    wz = (double)sz.hi + (double)sz.lo;
  } else {
    wx = warp_sum(gx);
    wy = warp_sum(gy);
    wz = warp_sum(gz);
  }
  __shared__ double ws[3][kWallThreads / 32];
  __shared__ bool last;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    ws[0][wid] = wx;
    ws[1][wid] = wy;
    ws[2][wid] = wz;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int k = 0; k < kWallThreads / 32; ++k) {
      a += ws[0][k];
      b += ws[1][k];
      c += ws[2][k];
    }
    partials[3 * blockIdx.x + 0] = a;
    partials[3 * blockIdx.x + 1] = b;
    partials[3 * blockIdx.x + 2] = c;
    last = false;
    if (accum) {
      __threadfence();  // partials visible before the count
      last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
  }
  __syncthreads();
  if (!last) return;
  // last CTA: fixed-order FP64 sum of all CTA partials (the same for any
  // completion order)
  __threadfence();
  double a = 0.0, b = 0.0, c = 0.0;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += kWallThreads) {
    a += __ldcg(&partials[3 * k]);
    b += __ldcg(&partials[3 * k + 1]);
    c += __ldcg(&partials[3 * k + 2]);
  }
  block_sum3<kWallThreads>(a, b, c);
  if (threadIdx.x == 0) {
    a += rest.x;
    b += rest.y;
    c += rest.z;
    accum[0] = a;
    accum[1] = b;
    accum[2] = c;
    accum[3] += a;
    accum[4] += b;
    accum[5] += c;
    accum[6] += 1.0;
    *done = 0u;
  }
}

// per-branch force of one finest step: one CTA per branch sums its links
// (contiguous, fixed order) and adds them to the branch's running sums
// seg_accum[4 k .. 4 k + 2]; seg_accum[4 k + 3] counts the steps
__global__ void __launch_bounds__(256) k_segments(const double* __restrict__ link_force,
                                                  const int* __restrict__ seg_begin, double* __restrict__ seg_accum) {
  const int k = blockIdx.x;
  double a = 0, b = 0, c = 0;
  for (int j = seg_begin[k] + threadIdx.x; j < seg_begin[k + 1]; j += 256) {
    a += link_force[3 * (size_t)j];
    b += link_force[3 * (size_t)j + 1];
    c += link_force[3 * (size_t)j + 2];
  }
  block_sum3<256>(a, b, c);
  if (threadIdx.x == 0) {
    seg_accum[4 * k] += a;
    seg_accum[4 * k + 1] += b;
    seg_accum[4 * k + 2] += c;
    seg_accum[4 * k + 3] += 1.0;
  }
}

// ---------------------------------------------------------------- interface ledger

// a population deviation in the ledger's fixed point (quantum 2^-40): exact for
// binary16 values (11 significant bits times 2^-13), rounded at 2^-41 for
// FP32 values below 2^-17 and for FP64 values
__device__ __forceinline__ long long fx40(float v) { return __float2ll_rn(v * 0x1p40f); }
__device__ __forceinline__ long long fx40(double v) { return __double2ll_rn(v * 0x1p40); }

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Adds NF flows of every thread's entry (q[f]: fixed-point population values
// of direction dir, dir < 0 for a thread without an entry) to the ledger's
// values [4 first, 4 first + 4 NF): mass and the three momentum components.
// Warps whose entries share one direction (the tables are ordered by
// destination slot, so most do) sum one value per flow, the others four;
// lanes 0..4 NF - 1 then add the warp's sums to one of the kLedgerCopies
// copies (chosen by warp), so no CTA-wide barrier is needed.  Every lane of
// the warp must call it.
template <int NF>
__device__ __forceinline__ void ledger_add(LedgerDev* __restrict__ L, int first, const long long (&q)[NF], int dir) {
  const int lane = threadIdx.x & 31;
  const int d0 = __reduce_max_sync(0xffffffffu, dir);
  const bool uni = __all_sync(0xffffffffu, dir < 0 || dir == d0);
  long long mine = 0;  // lane 4 f + c holds component c of flow f
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    if (uni) {
      const long long m = warp_sum_ll(q[f]);  // valid in lane 0
      const long long mb = __shfl_sync(0xffffffffu, m, 0);
      const int c = lane - 4 * f;
      if (c >= 0 && c < 4 && d0 >= 0) mine = c == 0 ? mb : (c == 1 ? dcx(d0) : (c == 2 ? dcy(d0) : dcz(d0))) * mb;
    } else {
      const int cxx = dir < 0 ? 0 : dcx(dir), cyy = dir < 0 ? 0 : dcy(dir), czz = dir < 0 ? 0 : dcz(dir);
      const long long v[4] = {q[f], cxx * q[f], cyy * q[f], czz * q[f]};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const long long sum = __shfl_sync(0xffffffffu, warp_sum_ll(v[c]), 0);
        if (lane == 4 * f + c) mine = sum;
      }
    }
  }
  if (lane < 4 * NF && mine) {
    const int copy = (int)((blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) % kLedgerCopies);
    atomicAdd(reinterpret_cast<unsigned long long*>(&L->acc[copy][first + lane]), (unsigned long long)mine);
  }
}

// A warp's running ledger sum over consecutive entries of a thread (the
// explode and the inflow entry of the same index) that share one direction:
// entries add to it while the warp's direction stays the same, and it is
// reduced and added to the ledger only when the direction changes and at the
// end.  (Four entries per thread cut the reductions further but slowed the
// transfers' dependent gathers more: interface kernels 78.5 -> 85.7 us per
// coarse step on GB300.)
struct LedgerRun {
  long long acc = 0;
  int dir = -1;  // the run's direction, the same in every lane
};
__device__ __forceinline__ void ledger_flush(LedgerRun& r, LedgerDev* __restrict__ L, int first) {
  if (r.dir >= 0) {
    const long long q[1] = {r.acc};
    ledger_add<1>(L, first, q, r.dir);
  }
  r.acc = 0;
  r.dir = -1;
}
__device__ __forceinline__ void ledger_run_add(LedgerRun& r, LedgerDev* __restrict__ L, int first, long long q,
                                               int dir) {
  const int d0 = __reduce_max_sync(0xffffffffu, dir);
  const bool uni = __all_sync(0xffffffffu, dir < 0 || dir == d0);
  if (uni && (d0 < 0 || r.dir < 0 || d0 == r.dir)) {
    r.acc += q;
    if (d0 >= 0) r.dir = d0;
    return;
  }
  ledger_flush(r, L, first);
  if (uni) {
    r.acc = q;
    r.dir = d0;
  } else {
    const long long qq[1] = {q};
    ledger_add<1>(L, first, qq, dir);
  }
}

// population plane of an element offset (log2 of the cells per block given)
__device__ __forceinline__ int plane_of(long long off, int c3_log2) { return (int)((off >> c3_log2) % 27); }

// a 64-bit integer as float with round-to-odd (truncated, last bit set when
// inexact): rounding that to binary16 gives the correctly rounded binary16 of
// the integer (float keeps more than two bits beyond binary16's eleven)
__device__ __forceinline__ float ll_to_float_odd(long long q) {
  const float z = __ll2float_rz(q);
  if (__float2ll_rz(z) == q) return z;
  return __uint_as_float(__float_as_uint(z) | 1u);
}

// Interface kernels.  ratio = s_fine / s_coarse maps stored coarse values to
// the fine scale (1 for FP32 and FP64); saved values are fine-scaled values of
// the arithmetic type (FP32, FP64 for the double-precision form).
//
// One kernel moves what the coarse step hands to the fine level, from three
// entry tables: the explode entries (coarse post-collision values into the
// fine ghost slots the second sub-step pulls from), the save entries (fine
// values of the first sub-step that leave the box, for the coalesce
// transfer) and the inflow entries (the values the fine cells at the box
// edge pull at the next first sub-step).  Ghost slots live in ghost blocks,
// which the first sub-step (an even step: own slots of active blocks only)
// never touches, so the explode entries may run beside it.  The save sources,
// slots (x, ibar) of active cells with x + c_i outside the box, and the
// inflow destinations, slots (x, i) with x - c_i outside, are neither read
// nor written by the second sub-step (either would need an active cell at
// that outside point), so the save and inflow entries may run beside it.
// Every save source is also an inflow destination (slot (b, ibar) with
// b + c_i outside the box is where b pulls f_ibar at the next first
// sub-step): the inflow entry's thread saves it before writing, and the save
// entry itself is skipped (src = -1), so no thread reads a slot another
// thread of the launch writes.
template <typename S, typename E, typename SE, typename IE>
__global__ void __launch_bounds__(256) k_explode(S* __restrict__ fine, const S* __restrict__ coarse,
                                                 const E* __restrict__ e, int ne, const SE* __restrict__ s, int ns,
                                                 const IE* __restrict__ ie, int ni,
                                                 typename Store<S>::V* __restrict__ saved, int parity, float ratio,
                                                 LedgerDev* __restrict__ ledger, int c3_log2, float inv_sf) {
  using V = typename Store<S>::V;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long q = 0, qi = 0;
  int dir = -1, diri = -1;
  if (t < ne) {
    const E x = e[t];
    const V v = Store<S>::ld(coarse, parity ? x.src[1] : x.src[0]) * ratio;
    Store<S>::st(fine, x.dst, v);
    if (ledger) {
      q = fx40(v * (V)inv_sf);
      dir = 26 - plane_of(x.dst, c3_log2);
    }
  }
  if (t < ns) {
    const auto src = s[t].src;
    if (src >= 0) saved[t] = Store<S>::ld(fine, src);
  }
  if (t < ni) {
    const IE x = ie[t];
    // a destination that also holds a value leaving the box is saved by
    // this thread before it is overwritten
    if (x.sv >= 0) saved[x.sv] = Store<S>::ld(fine, x.dst);
    const V v = Store<S>::ld(coarse, parity ? x.csrc[1] : x.csrc[0]) * ratio;
    Store<S>::st(fine, x.dst, v);
    if (ledger) {
      qi = fx40(v * (V)inv_sf);
      diri = plane_of(x.dst, c3_log2);
    }
  }
  if (ledger) {
    LedgerRun run;
    ledger_run_add(run, ledger, 0, q, dir);
    ledger_run_add(run, ledger, 0, qi, diri);
    ledger_flush(run, ledger, 0);
  }
}

// Coarse cell next to the fine region, one direction: the mean of its 8
// children's values (fine values, or n_coarse times its own coarse value),
// summed exactly and rounded to storage once.  In the reduced forms the sum
// is taken in 64-bit fixed point (deviations x 2^40: exact for binary16
// values, within 2^-41 per value in FP32, far below one FP32 unit of any
// deviation above 1e-5), then rounded once (FP32: the integer to nearest
// float; binary16: via round-to-odd float); the FP64 form sums in FP64.
// With a ledger: the fine values taken (OutF) and what the coarse slot
// receives, 8 x stored - n_coarse x old (RecvC); the launch's last CTA folds
// the coarse step's sums into the FP64 records.
template <typename S, typename E>
__global__ void k_coalesce(S* __restrict__ coarse, const S* __restrict__ fine, const E* __restrict__ e, int n,
                           const typename Store<S>::V* __restrict__ saved, int parity, float ratio,
                           LedgerDev* __restrict__ ledger, LedgerConst lc, int c3_log2, float inv_sc, float inv_sf) {
  using V = typename Store<S>::V;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  long long q[2] = {0, 0};
  int dir = -1;
  if (t < n) {
    const E& x = e[t];
    const long long dst = parity ? x.dst[1] : x.dst[0];
    const V vc = x.ncoarse ? Store<S>::ld(coarse, dst) : (V)0;
    if constexpr (sizeof(V) == 4) {
      long long qf = 0;  // the fine values' deviations, fixed point
      for (int k = 0; k < x.nfine; ++k) {
        const long long s = x.fsrc[k];
        qf += fx40((s >= 0 ? Store<S>::ld(fine, s) : saved[-s - 1]) * inv_sf);
      }
      const long long qc = x.ncoarse ? fx40(vc * inv_sc) : 0;
      const long long qt = qf + x.ncoarse * qc;  // 8 x the new deviation, fixed point
      // the new stored value: qt x 2^-43 deviations x the coarse scale, one rounding
      float stored;
      if constexpr (std::is_same<S, __half>::value) {
        const __half h = __float2half_rn(ll_to_float_odd(qt) * (0x1p-43f / inv_sc));
        coarse[dst] = h;
        stored = __half2float(h);
      } else {
        stored = __ll2float_rn(qt) * 0x1p-43f;
        Store<S>::st(coarse, dst, stored);
      }
      if (ledger) {
        q[0] = qf;
        // 8 x the stored deviation x 2^40 is an integer in both forms (the
        // rounded qt in FP32, a binary16 value x 2^30): exact
        q[1] = __float2ll_rn(stored * (0x1p43f * inv_sc)) - x.ncoarse * qc;
      }
    } else {
      V acc = 0;
      long long qf = 0;
      for (int k = 0; k < x.nfine; ++k) {
        const long long s = x.fsrc[k];
        const V v = s >= 0 ? Store<S>::ld(fine, s) : saved[-s - 1];
        acc += v;
        if (ledger) qf += fx40(v);
      }
      const V stored = (acc / (V)ratio + (V)x.ncoarse * vc) * 0.125;
      Store<S>::st(coarse, dst, stored);
      if (ledger) {
        q[0] = qf;
        q[1] = 8 * fx40(stored) - (long long)x.ncoarse * fx40(vc);
      }
    }
    if (ledger) {
      const int pl = plane_of(dst, c3_log2);
      dir = parity ? pl : 26 - pl;
    }
  }
  if (!ledger) return;
  ledger_add<2>(ledger, 4, q, dir);
  // the last CTA of the launch folds the step's sums (explode, inflow and this
  // launch) into the FP64 records and clears them for the next coarse step
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&ledger->done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < kLedgerVals) {
    const int k = threadIdx.x;
    long long sum = 0;
    for (int c = 0; c < kLedgerCopies; ++c) {
      sum += (long long)__ldcg(reinterpret_cast<const unsigned long long*>(&ledger->acc[c][k]));
      ledger->acc[c][k] = 0;
    }
    const double v = lc.vol * ((double)sum * 0x1p-40 + lc.c[k]);
    ledger->last[k] = v;
    ledger->total[k] += v;
  }
  if (threadIdx.x == 0) {
    ledger->steps += 1.0;
    ledger->done = 0u;
  }
}

// one CTA per (storage block, population plane): the plane's C3 values are
// all equal, written as 16-byte words (dev: the stored value per plane, in
// FP64, rounded to the storage type here)
template <typename S>
__global__ void __launch_bounds__(256) k_fill(S* __restrict__ f, int c3, Vals27 dev) {
  const long long chunk = blockIdx.x;
  const double vd = dev.v[(int)(chunk % 27)];
  uint4 w;
  if (std::is_same<S, float>::value) {
    const unsigned b = __float_as_uint((float)vd);
    w = make_uint4(b, b, b, b);
  } else if (std::is_same<S, __half>::value) {
    const unsigned short h = __half_as_ushort(__float2half_rn((float)vd));
    const unsigned b = (unsigned)h | ((unsigned)h << 16);
    w = make_uint4(b, b, b, b);
  } else {
    const unsigned long long b = (unsigned long long)__double_as_longlong(vd);
    w = make_uint4((unsigned)b, (unsigned)(b >> 32), (unsigned)b, (unsigned)(b >> 32));
  }
  uint4* p = reinterpret_cast<uint4*>(f + chunk * c3);
  const int nw = c3 * (int)sizeof(S) / 16;
  for (int k = threadIdx.x; k < nw; k += blockDim.x) p[k] = w;
}

// FP64 mass and momentum of the incoming populations of one level; per CTA
// partials [mass, jx, jy, jz, bad cells]
template <int B, typename S>
__global__ void __launch_bounds__(B * B) k_mass(const S* __restrict__ f, const int* __restrict__ nbr,
                                                const int* __restrict__ maskoff, const uint8_t* __restrict__ masks,
                                                int parity, float inv_scale, Ref27 ref,
                                                double* __restrict__ partials) {
  constexpr int C3 = B * B * B;
  __shared__ long long s_base[27];
  __shared__ double s_bad[B * B / 32];
  const int blk = blockIdx.x;
  if (threadIdx.x < 27) s_base[threadIdx.x] = (long long)nbr[(size_t)blk * 27 + threadIdx.x] * (27LL * C3);
  __syncthreads();
  const int lx = threadIdx.x % B, ly = threadIdx.x / B;
  const int mo = maskoff[blk];
  const uint8_t* mask = mo >= 0 ? masks + (size_t)mo * C3 : nullptr;
  double m = 0, jx = 0, jy = 0, jz = 0, bad = 0;
  for (int lz = 0; lz < B; ++lz) {
    const int cell = (lz * B + ly) * B + lx;
    if (mask && !mask[cell]) continue;
    double rho = 0, ax = 0, ay = 0, az = 0;
#pragma unroll
    for (int i = 0; i < 27; ++i) {
      typename Store<S>::V v;
      if (!parity) {
        v = Store<S>::ld(f, s_base[13] + i * C3 + cell);
      } else {
        const int nx = lx - dcx(i), ny = ly - dcy(i), nz = lz - dcz(i);
        const int bd = block_digit<B>(nx) + 3 * block_digit<B>(ny) + 9 * block_digit<B>(nz);
        const int nc = ((nz & (B - 1)) * B + (ny & (B - 1))) * B + (nx & (B - 1));
        v = Store<S>::ld(f, s_base[bd] + (26 - i) * C3 + nc);
      }
      double vd = v;
      if (Store<S>::scaled) vd = (double)v * inv_scale + (double)ref.v[i];
      const double w = (dcx(i) ? 1.0 / 6.0 : 2.0 / 3.0) * (dcy(i) ? 1.0 / 6.0 : 2.0 / 3.0) *
                       (dcz(i) ? 1.0 / 6.0 : 2.0 / 3.0);
      rho += w + vd;
      ax += dcx(i) * vd;
      ay += dcy(i) * vd;
      az += dcz(i) * vd;
    }
    if (!(rho >= 0.5 && rho <= 2.0)) bad += 1.0;  // also catches NaN
    m += rho;
    jx += ax;
    jy += ay;
    jz += az;
  }
  block_sum3<B * B>(m, jx, jy);
  double z = warp_sum(jz), b = warp_sum(bad);
  __shared__ double s_z[B * B / 32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    s_z[w] = z;
    s_bad[w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double zz = 0, bb = 0;
    for (int k = 0; k < B * B / 32; ++k) {
      zz += s_z[k];
      bb += s_bad[k];
    }
    double* p = partials + 5 * (size_t)blk;
    p[0] = m;
    p[1] = jx;
    p[2] = jy;
    p[3] = zz;
    p[4] = bb;
  }
}

// Scratch for lbm_mass_noalloc: per-block partial sums [mass, jx, jy, jz,
// bad] of one level, then the 5 totals.  It lives in the library image, so
// that entry point needs no device memory from its caller; host code must
// use the address from cudaGetSymbolAddress, never the symbol itself.
constexpr int kNoAllocMaxBlocks = 32768;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxBlocks * 5 + 8];

// fixed-order FP64 sum of n rows of 5 partials into out[0..4]
__global__ void __launch_bounds__(256) k_sum5(const double* __restrict__ partials, int n, double* __restrict__ out) {
  double a = 0, b = 0, c = 0, d = 0, e = 0;
  for (int k = threadIdx.x; k < n; k += 256) {
    a += partials[5 * k];
    b += partials[5 * k + 1];
    c += partials[5 * k + 2];
    d += partials[5 * k + 3];
    e += partials[5 * k + 4];
  }
  block_sum3<256>(a, b, c);
  __syncthreads();
  double z = 0.0;
  block_sum3<256>(d, e, z);
  if (threadIdx.x == 0) {
    out[0] = a;
    out[1] = b;
    out[2] = c;
    out[3] = d;
    out[4] = e;
  }
}

thread_local char g_err[256] = "";

int check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(g_err, sizeof g_err, "%s: %s", what, cudaGetErrorString(e));
    return LBM_ECUDA;
  }
  return LBM_OK;
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

const char* cuda_error_string() { return g_err; }

// call fn with a typed null pointer of the storage type of `esize` bytes per
// population (2: binary16, 4: FP32, 8: FP64)
template <class F>
void by_storage(int esize, F&& fn) {
  if (esize == 2) fn((__half*)nullptr);
  else if (esize == 8) fn((double*)nullptr);
  else fn((float*)nullptr);
}

template <int B, typename IDX, typename S>
void collide_on(const CollideArgs& a, int odd, cudaStream_t s) {
  constexpr bool f32 = std::is_same<S, float>::value;
  if (odd) {
    if (f32 && a.odd_variant == LBM_ODD_STAGED && B == 16)
      k_collide_odd_staged<IDX><<<a.n_active, 256, kStageBytes, s>>>(a);
    else if (a.odd_variant == LBM_ODD_PAIRS_7 && B == 16)
      k_collide_odd_p2<B, IDX, S, 7><<<a.n_active << a.zshift_odd, B * B / 2, 0, s>>>(a);
    else if (a.odd_variant == LBM_ODD_PAIRS_8 && B == 16)
      k_collide_odd_p2<B, IDX, S, 8><<<a.n_active << a.zshift_odd, B * B / 2, 0, s>>>(a);
    else if (a.odd_variant == LBM_ODD_PAIRS || a.odd_variant == LBM_ODD_PAIRS_7 || a.odd_variant == LBM_ODD_PAIRS_8)
      k_collide_odd_p2<B, IDX, S, 6><<<a.n_active << a.zshift_odd, B * B / 2, 0, s>>>(a);
    else if (a.odd_variant == LBM_ODD_DIRECT) k_collide<B, true, IDX, S><<<a.n_active << a.zshift_odd, B * B, 0, s>>>(a);
    else k_collide_odd_cols<B, IDX, S><<<a.n_active << a.zshift_odd, B * B, 0, s>>>(a);
  } else {
    if (f32 && a.even_variant == LBM_EVEN_TMA && B == 16)
      k_collide_even_tma<IDX><<<a.n_active, 256, kEvenBytes, s>>>(a);
    else if (a.even_variant == LBM_EVEN_PAIRS)
      k_collide_even_p2<B, IDX, S><<<a.n_active << a.zshift_even, B * B / 2, 0, s>>>(a);
    else k_collide<B, false, IDX, S><<<a.n_active << a.zshift_even, B * B, 0, s>>>(a);
  }
}

template <int B, typename IDX>
void collide_f64_on(const CollideArgs& a, int odd, cudaStream_t s) {
  if (odd) k_collide_f64<B, true, IDX><<<a.n_active << a.zshift_odd, B * B, 0, s>>>(a);
  else k_collide_f64<B, false, IDX><<<a.n_active << a.zshift_even, B * B, 0, s>>>(a);
}

template <typename S>
void collide_typed(const CollideArgs& a, int B, int odd, cudaStream_t s) {
  const bool small = !a.wide && a.f_elems < (1LL << 31);
  if (B == 16) {
    if (small) collide_on<16, int, S>(a, odd, s);
    else collide_on<16, long long, S>(a, odd, s);
  } else {
    if (small) collide_on<8, int, S>(a, odd, s);
    else collide_on<8, long long, S>(a, odd, s);
  }
}

void collide_f64(const CollideArgs& a, int B, int odd, cudaStream_t s) {
  const bool small = !a.wide && a.f_elems < (1LL << 31);
  if (B == 16) {
    if (small) collide_f64_on<16, int>(a, odd, s);
    else collide_f64_on<16, long long>(a, odd, s);
  } else {
    if (small) collide_f64_on<8, int>(a, odd, s);
    else collide_f64_on<8, long long>(a, odd, s);
  }
}

template <int B, typename IDX, typename S>
void batch_on(const CollideArgs* lv, const int2* items, int n, int kind, int grid, int zshift, cudaStream_t s) {
  if (kind == 0) k_collide_batch<B, 0, IDX, S><<<grid, B * B, 0, s>>>(lv, items, n, zshift);
  else if (kind == 1) k_collide_batch<B, 1, IDX, S><<<grid, B * B, 0, s>>>(lv, items, n, zshift);
  else if (kind == 2) k_collide_batch<B, 2, IDX, S><<<grid, B * B, 0, s>>>(lv, items, n, zshift);
  else if (kind == 3) k_collide_batch<B, 3, IDX, S><<<grid, B * B / 2, 0, s>>>(lv, items, n, zshift);
  else k_collide_batch<B, 4, IDX, S><<<grid, B * B / 2, 0, s>>>(lv, items, n, zshift);
}

template <typename S>
void batch_typed(const CollideArgs* lv, const int2* items, int n, int B, int wide, int kind, int grid, int zshift,
                 cudaStream_t s) {
  if (B == 16) {
    if (!wide) batch_on<16, int, S>(lv, items, n, kind, grid, zshift, s);
    else batch_on<16, long long, S>(lv, items, n, kind, grid, zshift, s);
  } else {
    if (!wide) batch_on<8, int, S>(lv, items, n, kind, grid, zshift, s);
    else batch_on<8, long long, S>(lv, items, n, kind, grid, zshift, s);
  }
}

int prepare_kernels() {
  cudaError_t e = cudaFuncSetAttribute(k_collide_odd_staged<int>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kStageBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_collide_odd_staged<long long>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kStageBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_collide_even_tma<int>, cudaFuncAttributeMaxDynamicSharedMemorySize, kEvenBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_collide_even_tma<long long>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kEvenBytes);
  if (e != cudaSuccess) {
    snprintf(g_err, sizeof g_err, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    return LBM_ECUDA;
  }
  return LBM_OK;
}

int launch_collide(const CollideArgs& a, int B, int odd, void* stream) {
  if (a.n_active == 0) return LBM_OK;
  if (B != 16 && B != 8) return LBM_EINVAL;
  if (a.zshift_even < 0 || a.zshift_odd < 0 || (B >> a.zshift_even) < 1 || (B >> a.zshift_odd) < 1)
    return LBM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (a.f64) collide_f64(a, B, odd, s);
  else if (a.half) collide_typed<__half>(a, B, odd, s);
  else collide_typed<float>(a, B, odd, s);
  return check_launch("collide");
}

int launch_collide_batch(const CollideArgs* lv, const int2* items, int n_items, int B, int odd, int odd_variant,
                         int even_variant, int half, int wide, int grid, int zshift, void* stream) {
  if (n_items == 0) return LBM_OK;
  if (B != 16 && B != 8) return LBM_EINVAL;
  if (zshift < 0 || (B >> zshift) < 1) return LBM_EINVAL;
  const bool odd_pairs = odd_variant == LBM_ODD_PAIRS || odd_variant == LBM_ODD_PAIRS_7 || odd_variant == LBM_ODD_PAIRS_8;
  const int kind = !odd ? (even_variant == LBM_EVEN_PAIRS ? 3 : 0)
                        : (odd_pairs ? 4 : (odd_variant == LBM_ODD_DIRECT ? 1 : 2));
  const int units = n_items << zshift;
  const int g = grid > 0 ? std::min(grid, units) : units;
  cudaStream_t s = (cudaStream_t)stream;
  if (half) batch_typed<__half>(lv, items, n_items, B, wide, kind, g, zshift, s);
  else batch_typed<float>(lv, items, n_items, B, wide, kind, g, zshift, s);
  return check_launch("collide_batch");
}

template <typename E>
void faces_typed(void* f, int esize, const E* e, int n, const double feq[27], const TurbArgs& turb,
                 cudaStream_t s) {
  if (turb.n_modes > 0 && esize != 8) {
    if (turb.n_cells > 0) {
      const size_t smem = (size_t)turb.n_modes * kModeCols * sizeof(float);
      k_turb_velocity<<<blocks_for(turb.n_cells, 128), 128, smem, s>>>(turb);
    }
    if (esize == 2) k_faces_turb<__half, E><<<blocks_for(n, 256), 256, 0, s>>>((__half*)f, e, n, turb);
    else k_faces_turb<float, E><<<blocks_for(n, 256), 256, 0, s>>>((float*)f, e, n, turb);
    return;
  }
  if (esize == 8) {
    Vals27 v;
    for (int i = 0; i < 27; ++i) v.v[i] = feq[i];
    k_faces<double, E, Vals27><<<blocks_for(n, 256), 256, 0, s>>>((double*)f, e, n, v);
    return;
  }
  Feq27 v;
  for (int i = 0; i < 27; ++i) v.v[i] = (float)feq[i];
  if (esize == 2) k_faces<__half, E, Feq27><<<blocks_for(n, 256), 256, 0, s>>>((__half*)f, e, n, v);
  else k_faces<float, E, Feq27><<<blocks_for(n, 256), 256, 0, s>>>((float*)f, e, n, v);
}

int launch_faces(void* f, int esize, const void* e, int narrow, int n, const double feq[27], const TurbArgs& turb,
                 void* stream) {
  if (n == 0) return LBM_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (narrow) faces_typed(f, esize, (const FaceEntryN*)e, n, feq, turb, s);
  else faces_typed(f, esize, (const FaceEntry*)e, n, feq, turb, s);
  return check_launch("faces");
}

int launch_friction(const void* f, int esize, float inv_scale, const Ref27& ref, int B, const int* nbr, int odd,
                    float omega1, const FrictionSample* e, int n, double* out, void* stream) {
  if (n == 0) return LBM_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned g = blocks_for(n, 128);
  by_storage(esize, [&](auto* tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    if (B == 16) k_friction<16, S><<<g, 128, 0, s>>>((const S*)f, e, n, nbr, odd, omega1, inv_scale, ref, out);
    else k_friction<8, S><<<g, 128, 0, s>>>((const S*)f, e, n, nbr, odd, omega1, inv_scale, ref, out);
  });
  return check_launch("friction");
}

int launch_tick(long long* tick, void* stream) {
  k_tick<<<1, 1, 0, (cudaStream_t)stream>>>(tick);
  return check_launch("tick");
}

int walls_partial_count(int n) { return (int)blocks_for(n, kWallThreads); }

template <typename E>
void walls_typed(void* f, int esize, const double* q64, float inv_scale, const Ref27& ref, const E* e, int n,
                 double* partials, double* link_force, unsigned* done, double* accum, double3 rest, cudaStream_t s) {
  const unsigned g = blocks_for(n, kWallThreads);
  by_storage(esize, [&](auto* tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    k_walls<S, E><<<g, kWallThreads, 0, s>>>((S*)f, e, n, q64, inv_scale, ref, partials, link_force, done, accum,
                                              rest);
  });
}

int launch_walls(void* f, int esize, const double* q64, float inv_scale, const Ref27& ref, const void* e, int narrow,
                 int n, double* partials, double* link_force, unsigned* done, double* accum, const double rest[3],
                 void* stream) {
  if (n == 0) return LBM_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const double3 r = make_double3(rest[0], rest[1], rest[2]);
  if (narrow)
    walls_typed(f, esize, q64, inv_scale, ref, (const WallEntryN*)e, n, partials, link_force, done, accum, r, s);
  else walls_typed(f, esize, q64, inv_scale, ref, (const WallEntry*)e, n, partials, link_force, done, accum, r, s);
  return check_launch("walls");
}

int launch_segments(const double* link_force, const int* seg_begin, int n_seg, double* seg_accum, void* stream) {
  if (n_seg == 0) return LBM_OK;
  k_segments<<<n_seg, 256, 0, (cudaStream_t)stream>>>(link_force, seg_begin, seg_accum);
  return check_launch("segments");
}

template <typename E, typename SE, typename IE>
void explode_typed(void* fine, const void* coarse, int esize, float ratio, const E* e, int ne, const SE* sv, int ns,
                   const IE* ie, int ni, void* saved, int parity, LedgerDev* ledger, int c3_log2, float inv_sf,
                   cudaStream_t s) {
  const unsigned g = blocks_for(std::max(ne, std::max(ns, ni)), 256);
  by_storage(esize, [&](auto* tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    using V = typename Store<S>::V;
    k_explode<S, E, SE, IE><<<g, 256, 0, s>>>((S*)fine, (const S*)coarse, e, ne, sv, ns, ie, ni, (V*)saved, parity,
                                               ratio, ledger, c3_log2, inv_sf);
  });
}

int launch_explode(void* fine, const void* coarse, int esize, float ratio, const void* e, int narrow, int ne,
                   const void* sv, int ns, const void* ie, int ni, void* saved, int parity, LedgerDev* ledger,
                   int c3_log2, float inv_sf, void* stream) {
  if (ne == 0 && ns == 0 && ni == 0) return LBM_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (narrow)
    explode_typed(fine, coarse, esize, ratio, (const ExplodeEntryN*)e, ne, (const SaveEntryN*)sv, ns,
                  (const InflowEntryN*)ie, ni, saved, parity, ledger, c3_log2, inv_sf, s);
  else
    explode_typed(fine, coarse, esize, ratio, (const ExplodeEntry*)e, ne, (const SaveEntry*)sv, ns,
                  (const InflowEntry*)ie, ni, saved, parity, ledger, c3_log2, inv_sf, s);
  return check_launch("explode");
}

template <typename E>
void coalesce_typed(void* coarse, const void* fine, int esize, float ratio, const E* e, int n, const void* saved,
                    int parity, LedgerDev* ledger, const LedgerConst& lc, int c3_log2, float inv_sc, float inv_sf,
                    cudaStream_t s) {
  by_storage(esize, [&](auto* tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    using V = typename Store<S>::V;
    k_coalesce<S, E><<<blocks_for(n, 256), 256, 0, s>>>((S*)coarse, (const S*)fine, e, n, (const V*)saved, parity,
                                                         ratio, ledger, lc, c3_log2, inv_sc, inv_sf);
  });
}

int launch_coalesce(void* coarse, const void* fine, int esize, float ratio, const void* e, int narrow, int n,
                    const void* saved, int parity, LedgerDev* ledger, const LedgerConst& lc, int c3_log2,
                    float inv_sc, float inv_sf, void* stream) {
  if (n == 0) return LBM_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (narrow)
    coalesce_typed(coarse, fine, esize, ratio, (const CoalesceEntryN*)e, n, saved, parity, ledger, lc, c3_log2,
                   inv_sc, inv_sf, s);
  else
    coalesce_typed(coarse, fine, esize, ratio, (const CoalesceEntry*)e, n, saved, parity, ledger, lc, c3_log2, inv_sc,
                   inv_sf, s);
  return check_launch("coalesce");
}

int launch_fill(void* f, int esize, long long n_blocks, int B, const double dev[27], void* stream) {
  Vals27 v;
  for (int i = 0; i < 27; ++i) v.v[i] = dev[i];
  const int c3 = B * B * B;
  const long long chunks = n_blocks * 27LL;
  if (chunks == 0) return LBM_OK;
  if (chunks > 0x7fffffffLL) return LBM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  by_storage(esize, [&](auto* tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    k_fill<S><<<(unsigned)chunks, 256, 0, s>>>((S*)f, c3, v);
  });
  return check_launch("fill");
}

int mass_partial_count(int n_active) { return n_active; }

int launch_mass(const void* f, int esize, float inv_scale, const Ref27& ref, const int* nbr, const int* maskoff,
                const uint8_t* masks, int n_active, int B, int parity, double* partials, void* stream) {
  if (n_active == 0) return LBM_OK;
  cudaStream_t s = (cudaStream_t)stream;
  by_storage(esize, [&](auto* tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    const float isc = Store<S>::scaled ? inv_scale : 1.0f;
    if (B == 16)
      k_mass<16, S><<<n_active, 256, 0, s>>>((const S*)f, nbr, maskoff, masks, parity, isc, ref, partials);
    else k_mass<8, S><<<n_active, 64, 0, s>>>((const S*)f, nbr, maskoff, masks, parity, isc, ref, partials);
  });
  return check_launch("mass");
}

int noalloc_max_blocks() { return kNoAllocMaxBlocks; }

// Device address of the static scratch for the current device (the domain's
// device must be current, as for every call of the library), looked up once
// per device with that device current.  std::call_once makes the first
// lookup race-free when several host threads make their first call at once;
// a failed lookup is retried by the next call.
int noalloc_scratch(double** out) {
  constexpr int kMaxDevices = 64;
  static std::once_flag once[kMaxDevices];
  static std::atomic<double*> ptr[kMaxDevices];
  static std::atomic<int> err[kMaxDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    snprintf(g_err, sizeof g_err, "cudaGetDevice: %s", cudaGetErrorString(e));
    return LBM_ECUDA;
  }
  std::call_once(once[dev], [dev] {
    void* p = nullptr;
    const cudaError_t r = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    err[dev].store((int)r);
    if (r == cudaSuccess) ptr[dev].store((double*)p);
  });
  double* p = ptr[dev].load();
  if (!p) {
    // the one-time lookup failed on this device: report it, try again directly
    void* q = nullptr;
    e = cudaGetSymbolAddress(&q, g_noalloc_scratch);
    if (e != cudaSuccess) {
      snprintf(g_err, sizeof g_err, "cudaGetSymbolAddress: %s (first lookup: %s)", cudaGetErrorString(e),
               cudaGetErrorString((cudaError_t)err[dev].load()));
      return LBM_ECUDA;
    }
    p = (double*)q;
  }
  *out = p;
  return LBM_OK;
}

int launch_mass_noalloc(const void* f, int esize, float inv_scale, const Ref27& ref, const int* nbr,
                        const int* maskoff,
                        const uint8_t* masks, int n_active, int B, int parity, double* scratch, void* stream) {
  if (n_active > kNoAllocMaxBlocks) return LBM_EINVAL;
  int rc = launch_mass(f, esize, inv_scale, ref, nbr, maskoff, masks, n_active, B, parity, scratch, stream);
  if (rc) return rc;
  k_sum5<<<1, 256, 0, (cudaStream_t)stream>>>(scratch, n_active, scratch + (size_t)kNoAllocMaxBlocks * 5);
  return check_launch("sum5");
}

}  // namespace lbm
