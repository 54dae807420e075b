// Collide-stream kernels of liblbm (included by kernels.cu): the fused
// cumulant collision and AA-pattern streaming of one active block, in the
// variants the schedules choose from - even step with direct loads and
// stores or a TMA bulk pipeline; odd step with per-thread column pointers,
// direct neighbour addressing or TMA/cp.async staging - and the batched
// persistent form that walks a (level, block) work list.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "cumulant.cuh"
#include "internal.h"

namespace lbm {
namespace {

__device__ __forceinline__ constexpr int dcx(int i) { return i % 3 - 1; }
__device__ __forceinline__ constexpr int dcy(int i) { return (i / 3) % 3 - 1; }
__device__ __forceinline__ constexpr int dcz(int i) { return i / 9 - 1; }

// neighbour-block digit (0, 1, 2) of a local coordinate shifted by s in [-1, 1]
template <int B>
__device__ __forceinline__ int block_digit(int c) {
  return c < 0 ? 0 : (c >= B ? 2 : 1);
}

// Population storage: FP32 deviations f - w, or FP16 deviations f - w - r
// from the inflow equilibrium (r_i = f_i^eq(1, U e_x) - w_i) times a
// per-level power-of-two scale.  ld/st move the stored (scaled) value.
template <typename S>
struct Store;
// V is the arithmetic type of the values moved (FP32 for both reduced forms).
template <>
struct Store<float> {
  using V = float;
  static constexpr bool scaled = false;
  static __device__ __forceinline__ float ld(const float* p, long long i) { return p[i]; }
  static __device__ __forceinline__ void st(float* p, long long i, float v) { p[i] = v; }
};
template <>
struct Store<__half> {
  using V = float;
  static constexpr bool scaled = true;
  static __device__ __forceinline__ float ld(const __half* p, long long i) { return __half2float(p[i]); }
  static __device__ __forceinline__ void st(__half* p, long long i, float v) { p[i] = __float2half_rn(v); }
};
// FP64 storage of f - w (the double-precision form): no scale, no reference
template <>
struct Store<double> {
  using V = double;
  static constexpr bool scaled = false;
  static __device__ __forceinline__ double ld(const double* p, long long i) { return p[i]; }
  static __device__ __forceinline__ void st(double* p, long long i, double v) { p[i] = v; }
};

#ifndef LBM_EVEN_MINB
#define LBM_EVEN_MINB 4
#endif
#ifndef LBM_ODD_MINB
#define LBM_ODD_MINB 4
#endif
#ifndef LBM_ODD_MINB_HALF
#define LBM_ODD_MINB_HALF 5  // the FP16 odd step fits 48 registers without spills
#endif
template <typename S>
constexpr int odd_minb() { return std::is_same<S, __half>::value ? LBM_ODD_MINB_HALF : LBM_ODD_MINB; }
// The one-CTA-per-block kernels can split a block's z walk over 2^zshift CTAs
// (CTA k of the block walks slabs k B / 2^zshift onwards): shorter CTAs fill
// the last partial wave of the grid and keep more blocks' rows in flight.
// Every cell update reads and writes only its own locations, so any split
// gives the same result.
struct ZSeg {
  int blk, z0, z1;
};
__device__ __forceinline__ ZSeg z_segment(int unit, int zshift, int B) {
  const int nz = B >> zshift, z0 = (unit & ((1 << zshift) - 1)) * nz;
  return ZSeg{unit >> zshift, z0, z0 + nz};
}
// the active block of launched block index b (a launch over a block subset)
__device__ __forceinline__ int block_of(const CollideArgs& a, int b) { return a.blocks ? a.blocks[b] : b; }
__device__ __forceinline__ ZSeg z_segment(const CollideArgs& a, int unit, int zshift, int B) {
  ZSeg z = z_segment(unit, zshift, B);
  z.blk = block_of(a, z.blk);
  return z;
}

// IDX: element-offset type, 32-bit when the level's array has < 2^31 elements
// One active block `blk` of a level: even step (own slots) or odd step with
// direct neighbour addressing.  s_base: 27 shared slots for the neighbour
// blocks' element offsets.
template <int B, bool ODD, typename IDX, typename S>
__device__ __forceinline__ void collide_block(const CollideArgs& a, const int blk, IDX* s_base, int z0 = 0,
                                              int z1 = B) {
  constexpr int C3 = B * B * B;
  if (threadIdx.x < 27) s_base[threadIdx.x] = (IDX)a.nbr[(size_t)blk * 27 + threadIdx.x] * (IDX)(27 * C3);
  __syncthreads();
  const int lx = threadIdx.x % B, ly = threadIdx.x / B;
  const int mo = a.maskoff[blk];
  const uint8_t* mask = mo >= 0 ? a.masks + (size_t)mo * C3 : nullptr;
  const Rates rates{a.omega1, a.omega2, a.galilean};
  S* __restrict__ f = reinterpret_cast<S*>(a.f);
  for (int lz = z0; lz < z1; ++lz) {
    const int cell = (lz * B + ly) * B + lx;
    if (mask && !mask[cell]) continue;
    float d[27];
    if (!ODD) {
      const S* p = f + s_base[13] + cell;
#pragma unroll
      for (int i = 0; i < 27; ++i) d[i] = Store<S>::ld(p, i * C3);
    } else {
#pragma unroll
      for (int i = 0; i < 27; ++i) {
        // pull f_i from (x - c_i, ibar)
        const int nx = lx - dcx(i), ny = ly - dcy(i), nz = lz - dcz(i);
        const int bd = block_digit<B>(nx) + 3 * block_digit<B>(ny) + 9 * block_digit<B>(nz);
        const int nc = ((nz & (B - 1)) * B + (ny & (B - 1))) * B + (nx & (B - 1));
        d[i] = Store<S>::ld(f, s_base[bd] + (IDX)((26 - i) * C3 + nc));
      }
    }
    // the FP16 even step runs the packed code in both lanes, so that it
    // equals the paired even step bit for bit
    if (Store<S>::scaled && !ODD) cumulant_collide_h_as_pair(d, rates, a.inv_scale, a.scale, &a.ref);
    else cumulant_collide_s<Store<S>::scaled>(d, rates, a.inv_scale, a.scale, &a.ref);
    if (!ODD) {
      S* p = f + s_base[13] + cell;
#pragma unroll
      for (int i = 0; i < 27; ++i) Store<S>::st(p, (26 - i) * C3, d[i]);
    } else {
#pragma unroll
      for (int i = 0; i < 27; ++i) {
        // push f*_i to (x + c_i, i)
        const int nx = lx + dcx(i), ny = ly + dcy(i), nz = lz + dcz(i);
        const int bd = block_digit<B>(nx) + 3 * block_digit<B>(ny) + 9 * block_digit<B>(nz);
        const int nc = ((nz & (B - 1)) * B + (ny & (B - 1))) * B + (nx & (B - 1));
        Store<S>::st(f, s_base[bd] + (IDX)(i * C3 + nc), d[i]);
      }
    }
  }
}

// Two x-neighbouring stored values (an even element index, so the pair is
// 4-byte aligned in FP16 and 8-byte aligned in FP32) as the two lanes of a
// packed FP32 register, and back.
template <typename S>
struct PairIO;
template <>
struct PairIO<float> {
  static __device__ __forceinline__ F2 ld(const float* p) {
    return F2{*reinterpret_cast<const unsigned long long*>(p)};
  }
  static __device__ __forceinline__ void st(float* p, F2 v) { *reinterpret_cast<unsigned long long*>(p) = v.v; }
};
template <>
struct PairIO<__half> {
  static __device__ __forceinline__ F2 ld(const __half* p) {
    const __half2 h = *reinterpret_cast<const __half2*>(p);
    return F2::pack(__low2float(h), __high2float(h));
  }
  static __device__ __forceinline__ void st(__half* p, F2 v) {
    *reinterpret_cast<__half2*>(p) = __floats2half2_rn(v.lo(), v.hi());
  }
};
// the collision of a pair in either storage form
template <typename S>
__device__ __forceinline__ void collide_pair(F2* d, const CollideArgs& a, const Rates& r) {
  collide_cell<F2, Store<S>::scaled>(d, r, a.inv_scale, a.scale, &a.ref);
}

// Even step with two x-neighbouring cells per thread: one 4-byte (FP16) or
// 8-byte (FP32) load or store moves a population of both cells, halving the
// load/store instructions of the one-cell-per-thread kernel, and the two
// collisions run as one in packed FP32 (two lanes per instruction); a pair
// with one non-fluid cell writes only the other.
#ifndef LBM_PAIR_MINB
#define LBM_PAIR_MINB 6
#endif
template <int B, typename IDX, typename S>
__device__ __forceinline__ void even_pair_block(const CollideArgs& a, const int blk, const ZSeg zg) {
  constexpr int C3 = B * B * B;
  const IDX own = (IDX)a.nbr[(size_t)blk * 27 + 13] * (IDX)(27 * C3);
  const int lx = 2 * (threadIdx.x % (B / 2)), ly = threadIdx.x / (B / 2);
  const int mo = a.maskoff[blk];
  const uint8_t* mask = mo >= 0 ? a.masks + (size_t)mo * C3 : nullptr;
  const Rates rates{a.omega1, a.omega2, a.galilean};
  S* __restrict__ f = reinterpret_cast<S*>(a.f);
  for (int lz = zg.z0; lz < zg.z1; ++lz) {
    const int cell = (lz * B + ly) * B + lx;
    const bool m0 = !mask || mask[cell], m1 = !mask || mask[cell + 1];
    if (!m0 && !m1) continue;
    S* p = f + own + cell;
    F2 d[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) d[i] = PairIO<S>::ld(p + i * C3);
    collide_pair<S>(d, a, rates);
    if (m0 && m1) {
#pragma unroll
      for (int i = 0; i < 27; ++i) PairIO<S>::st(p + (26 - i) * C3, d[i]);
    } else if (m0) {
#pragma unroll
      for (int i = 0; i < 27; ++i) Store<S>::st(p, (26 - i) * C3, d[i].lo());
    } else {
#pragma unroll
      for (int i = 0; i < 27; ++i) Store<S>::st(p, (26 - i) * C3 + 1, d[i].hi());
    }
  }
}
template <int B, typename IDX, typename S>
__global__ void __launch_bounds__(B * B / 2, LBM_PAIR_MINB) k_collide_even_p2(CollideArgs a) {
  const ZSeg zg = z_segment(a, blockIdx.x, a.zshift_even, B);
  even_pair_block<B, IDX, S>(a, zg.blk, zg);
}

// Odd step with two x-neighbouring cells (x0, x0 + 1), x0 even, per thread,
// collided as one in packed FP32.  A thread keeps 9 column pointers: for each
// of the rows y - 1, y, y + 1 the columns x0 - 1, x0 and x0 + 2 (each in
// whichever block holds it).  The pull of a population with c_x = 0 is one
// aligned pair load of both cells' values, with c_x = +-1 two single loads
// (x0 - 1 / x0, or x0 + 1 / x0 + 2); the push mirrors it.  Every
// neighbour of an active block has storage, so both lanes always load; only
// fluid cells store.  On the two z-face slabs the pointers are built per c_z
// group, for the slab (of this block or of its z neighbour) that the group
// reaches.
// MINB: resident CTAs per SM the registers are budgeted for (6: 80
// registers, no spills; 7: 72 registers, 24 bytes spilled; 8: 64 registers,
// ~170 bytes spilled) - more warps in flight against spill traffic, chosen
// by the autotuner (lbm_odd_variant LBM_ODD_PAIRS, _PAIRS_7, _PAIRS_8)
template <int B, typename IDX, typename S>
__device__ __forceinline__ void odd_pair_block(const CollideArgs& a, const int blk, IDX* s_base, const ZSeg zg) {
  constexpr int C3 = B * B * B, S2 = B * B, H = B / 2;
  const int t = threadIdx.x;
  if (t < 27) s_base[t] = (IDX)a.nbr[(size_t)blk * 27 + t] * (IDX)(27 * C3);
  __syncthreads();
  const int x0 = 2 * (t % H), ly = t / H;
  S* __restrict__ f = reinterpret_cast<S*>(a.f);
  // slab-lz column of cell (x, y), x and y within one block of the block's range
  auto colp = [&](int x, int y, int lz) -> S* {
    const int xyd = block_digit<B>(x) + 3 * block_digit<B>(y);
    return f + (s_base[xyd + 9] + (IDX)((lz * B + (y & (B - 1))) * B + (x & (B - 1))));
  };
  // slab-zs column of cell (x, y), zs in [-1, B] (this block or a z neighbour)
  auto colpz = [&](int x, int y, int zs) -> S* {
    const int bd = block_digit<B>(x) + 3 * block_digit<B>(y) + 9 * block_digit<B>(zs);
    return f + (s_base[bd] + (IDX)(((zs & (B - 1)) * B + (y & (B - 1))) * B + (x & (B - 1))));
  };
  const int mo = a.maskoff[blk];
  const uint8_t* mask = mo >= 0 ? a.masks + (size_t)mo * C3 : nullptr;
  const Rates rates{a.omega1, a.omega2, a.galilean};
  for (int lz = zg.z0; lz < zg.z1; ++lz) {
    const int cell = (lz * B + ly) * B + x0;
    const bool m0 = !mask || mask[cell], m1 = !mask || mask[cell + 1];
    if (!m0 && !m1) continue;
    const bool face = lz == 0 || lz == B - 1;
    F2 d[27];
    if (!face) {
      S *cL[3], *cC[3], *cR[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        cL[k] = colp(x0 - 1, ly + k - 1, lz);
        cC[k] = colp(x0, ly + k - 1, lz);
        cR[k] = colp(x0 + 2, ly + k - 1, lz);
      }
#pragma unroll
      for (int i = 0; i < 27; ++i) {  // pull f_i from (x - c_i, ibar) for both cells
        const int k = 1 - dcy(i);
        const int off = (26 - i) * C3 - dcz(i) * S2;
        if (dcx(i) == 0) d[i] = PairIO<S>::ld(cC[k] + off);
        else if (dcx(i) > 0) d[i] = F2::pack(Store<S>::ld(cL[k], off), Store<S>::ld(cC[k], off));
        else d[i] = F2::pack(Store<S>::ld(cC[k], off + 1), Store<S>::ld(cR[k], off));
      }
    } else {
#pragma unroll
      for (int g = -1; g <= 1; ++g) {  // directions pulling from slab lz + g (c_z = -g)
        S *cL[3], *cC[3], *cR[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          cL[k] = colpz(x0 - 1, ly + k - 1, lz + g);
          cC[k] = colpz(x0, ly + k - 1, lz + g);
          cR[k] = colpz(x0 + 2, ly + k - 1, lz + g);
        }
#pragma unroll
        for (int i = 0; i < 27; ++i) {
          if (-dcz(i) != g) continue;
          const int k = 1 - dcy(i);
          const int off = (26 - i) * C3;
          if (dcx(i) == 0) d[i] = PairIO<S>::ld(cC[k] + off);
          else if (dcx(i) > 0) d[i] = F2::pack(Store<S>::ld(cL[k], off), Store<S>::ld(cC[k], off));
          else d[i] = F2::pack(Store<S>::ld(cC[k], off + 1), Store<S>::ld(cR[k], off));
        }
      }
    }
    collide_pair<S>(d, a, rates);
    asm volatile("" ::: "memory");  // keep the pointer rebuild after the collision
    if (!face) {
      S *cL[3], *cC[3], *cR[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        cL[k] = colp(x0 - 1, ly + k - 1, lz);
        cC[k] = colp(x0, ly + k - 1, lz);
        cR[k] = colp(x0 + 2, ly + k - 1, lz);
      }
#pragma unroll
      for (int i = 0; i < 27; ++i) {  // push f*_i to (x + c_i, i) for both cells
        const int k = 1 + dcy(i);
        const int off = i * C3 + dcz(i) * S2;
        if (dcx(i) == 0) {
          if (m0 && m1) PairIO<S>::st(cC[k] + off, d[i]);
          else if (m0) Store<S>::st(cC[k], off, d[i].lo());
          else Store<S>::st(cC[k], off + 1, d[i].hi());
        } else if (dcx(i) > 0) {
          if (m0) Store<S>::st(cC[k], off + 1, d[i].lo());
          if (m1) Store<S>::st(cR[k], off, d[i].hi());
        } else {
          if (m0) Store<S>::st(cL[k], off, d[i].lo());
          if (m1) Store<S>::st(cC[k], off, d[i].hi());
        }
      }
    } else {
#pragma unroll
      for (int g = -1; g <= 1; ++g) {  // directions pushing into slab lz + g (c_z = g)
        S *cL[3], *cC[3], *cR[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          cL[k] = colpz(x0 - 1, ly + k - 1, lz + g);
          cC[k] = colpz(x0, ly + k - 1, lz + g);
          cR[k] = colpz(x0 + 2, ly + k - 1, lz + g);
        }
#pragma unroll
        for (int i = 0; i < 27; ++i) {
          if (dcz(i) != g) continue;
          const int k = 1 + dcy(i);
          const int off = i * C3;
          if (dcx(i) == 0) {
            if (m0 && m1) PairIO<S>::st(cC[k] + off, d[i]);
            else if (m0) Store<S>::st(cC[k], off, d[i].lo());
            else Store<S>::st(cC[k], off + 1, d[i].hi());
          } else if (dcx(i) > 0) {
            if (m0) Store<S>::st(cC[k], off + 1, d[i].lo());
            if (m1) Store<S>::st(cR[k], off, d[i].hi());
          } else {
            if (m0) Store<S>::st(cL[k], off, d[i].lo());
            if (m1) Store<S>::st(cC[k], off, d[i].hi());
          }
        }
      }
    }
  }
}

template <int B, typename IDX, typename S, int MINB>
__global__ void __launch_bounds__(B * B / 2, MINB) k_collide_odd_p2(CollideArgs a) {
  __shared__ IDX s_base[27];
  const ZSeg zg = z_segment(a, blockIdx.x, a.zshift_odd, B);
  odd_pair_block<B, IDX, S>(a, zg.blk, s_base, zg);
}

template <int B, bool ODD, typename IDX, typename S>
__global__ void __launch_bounds__(B * B, ODD ? LBM_ODD_MINB : LBM_EVEN_MINB) k_collide(CollideArgs a) {
  __shared__ IDX s_base[27];
  const ZSeg zg = z_segment(a, blockIdx.x, ODD ? a.zshift_odd : a.zshift_even, B);
  collide_block<B, ODD, IDX, S>(a, zg.blk, s_base, zg.z0, zg.z1);
}

// FP64 storage: the even or odd AA step of one block, one thread per (x, y)
// column walking its z segment, neighbour addressing through the 27-entry
// block table, the collision in FP64.  The double-precision form reproduces
// the FP64 method on the GPU (a reference and validation form: GB300's FP64
// rate is a small fraction of its FP32 rate, so this kernel is
// arithmetic-bound and is not tuned).
template <int B, bool ODD, typename IDX>
__global__ void __launch_bounds__(B * B) k_collide_f64(CollideArgs a) {
  constexpr int C3 = B * B * B;
  __shared__ IDX s_base[27];
  const ZSeg zg = z_segment(a, blockIdx.x, ODD ? a.zshift_odd : a.zshift_even, B);
  const int blk = zg.blk;
  if (threadIdx.x < 27) s_base[threadIdx.x] = (IDX)a.nbr[(size_t)blk * 27 + threadIdx.x] * (IDX)(27 * C3);
  __syncthreads();
  const int lx = threadIdx.x % B, ly = threadIdx.x / B;
  const int mo = a.maskoff[blk];
  const uint8_t* mask = mo >= 0 ? a.masks + (size_t)mo * C3 : nullptr;
  const RatesD rates{a.omega1d, a.omega2d, a.galilean};
  double* __restrict__ f = reinterpret_cast<double*>(a.f);
  for (int lz = zg.z0; lz < zg.z1; ++lz) {
    const int cell = (lz * B + ly) * B + lx;
    if (mask && !mask[cell]) continue;
    double d[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) {
      if (!ODD) {
        d[i] = f[s_base[13] + (IDX)(i * C3 + cell)];
      } else {  // pull f_i from (x - c_i, ibar)
        const int nx = lx - dcx(i), ny = ly - dcy(i), nz = lz - dcz(i);
        const int bd = block_digit<B>(nx) + 3 * block_digit<B>(ny) + 9 * block_digit<B>(nz);
        const int nc = ((nz & (B - 1)) * B + (ny & (B - 1))) * B + (nx & (B - 1));
        d[i] = f[s_base[bd] + (IDX)((26 - i) * C3 + nc)];
      }
    }
    cumulant_collide_d(d, rates);
#pragma unroll
    for (int i = 0; i < 27; ++i) {
      if (!ODD) {
        f[s_base[13] + (IDX)((26 - i) * C3 + cell)] = d[i];
      } else {  // push f*_i to (x + c_i, i)
        const int nx = lx + dcx(i), ny = ly + dcy(i), nz = lz + dcz(i);
        const int bd = block_digit<B>(nx) + 3 * block_digit<B>(ny) + 9 * block_digit<B>(nz);
        const int nc = ((nz & (B - 1)) * B + (ny & (B - 1))) * B + (nx & (B - 1));
        f[s_base[bd] + (IDX)(i * C3 + nc)] = d[i];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Odd step with the pulled values staged in shared memory (B = 16).
//
// At slab z the cell (x, y, z) pulls f_i from (x - c_i, z - cz_i) of plane
// ibar.  For each direction the 16 x 16 slab z - cz_i of plane ibar of the
// block (or of its z neighbour) is 1 KB of contiguous floats, fetched by one
// TMA bulk copy; the row that crosses a y face is a 64-byte bulk copy from the
// y neighbour; the column that crosses an x face and the corner value are
// strided, fetched with 4-byte cp.async.  Slabs are double-buffered so the
// copies for z + 1 run while slab z is collided.  The push to (x + c_i, i)
// stays a direct store.  Every wait on the copies is bounded; on time-out the
// CTA records an error word and leaves after a bounded wait for its copies.
struct Stage16 {
  float in[27][256];
  float xh[27][16];
  float yh[27][16];
  float cn[32];
};
#ifndef LBM_ODD_STAGES
#define LBM_ODD_STAGES 2
#endif
constexpr int kStages = LBM_ODD_STAGES;
constexpr int kStageBytes = kStages * (int)sizeof(Stage16) + 128 + 27 * 8;
constexpr uint32_t kStageTx = 27 * 1024 + 18 * 64;  // bulk bytes per slab

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void async_load4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// bounded wait; returns false on time-out
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase) {
  for (int it = 0; it < (1 << 22); ++it)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}

// One strided 4-byte halo copy of a slab: direction, x/y neighbour digit,
// offset inside the 16 x 16 slab and destination inside a stage (floats).
struct HaloItem {
  int dir, xyd, inslab, dst;
};

// k-th halo item: 18 x-halo columns of 16 (directions with cx != 0, in
// increasing order), then 12 corners (cx != 0 and cy != 0)
__device__ __forceinline__ HaloItem halo_item(int k) {
  int i, sy, by;
  if (k < 18 * 16) {
    const int q = k >> 4;
    i = (q >> 1) * 3 + ((q & 1) ? 2 : 0);
    sy = k & 15;
    by = 1;
  } else {
    const int q = k - 18 * 16, zc = q >> 2, r = q & 3;
    i = zc * 9 + (r >> 1) * 6 + ((r & 1) ? 2 : 0);
    sy = dcy(i) > 0 ? 15 : 0;
    by = dcy(i) > 0 ? 0 : 2;
  }
  const int bx = dcx(i) > 0 ? 0 : 2, col = dcx(i) > 0 ? 15 : 0;
  const int dst = k < 18 * 16 ? (int)(offsetof(Stage16, xh) / 4) + i * 16 + sy : (int)(offsetof(Stage16, cn) / 4) + i;
  return HaloItem{i, bx + 3 * by, sy * 16 + col, dst};
}

// issue the copies of slab z into stage st (thread-cooperative)
template <typename IDX>
__device__ __forceinline__ void stage_issue(Stage16& st, uint64_t* bar, const float* __restrict__ f, const IDX* s_base,
                                            int z, const HaloItem* items, int nitems) {
  constexpr int C3 = 4096;
  const int t = threadIdx.x;
  if (t < 32) {
    if (t == 0) mbar_arrive_tx(bar, kStageTx);
    __syncwarp();
    if (t < 27) {
      const int i = t;
      int zs = z - dcz(i);
      const int bz = zs < 0 ? 0 : (zs >= 16 ? 2 : 1);
      zs &= 15;
      const float* src = f + s_base[1 + 3 + 9 * bz] + (IDX)((26 - i) * C3 + zs * 256);
      bulk_load(st.in[i], src, 1024, bar);
      if (dcy(i) != 0) {
        const int by = dcy(i) > 0 ? 0 : 2, row = dcy(i) > 0 ? 15 : 0;
        const float* ys = f + s_base[1 + 3 * by + 9 * bz] + (IDX)((26 - i) * C3 + zs * 256 + row * 16);
        bulk_load(st.yh[i], ys, 64, bar);
      }
    }
  } else {
    float* sbase = reinterpret_cast<float*>(&st);
    for (int k = 0; k < nitems; ++k) {
      const HaloItem h = items[k];
      int zs = z - dcz(h.dir);
      const int bz = zs < 0 ? 0 : (zs >= 16 ? 2 : 1);
      zs &= 15;
      async_load4(sbase + h.dst, f + s_base[h.xyd + 9 * bz] + (IDX)((26 - h.dir) * C3 + zs * 256 + h.inslab));
    }
  }
  async_commit();
}

#ifndef LBM_STAGED_MINB
#define LBM_STAGED_MINB 3
#endif
template <typename IDX>
__global__ void __launch_bounds__(256, LBM_STAGED_MINB) k_collide_odd_staged(CollideArgs a) {
  constexpr int B = 16, C3 = 4096, NS = kStages;
  extern __shared__ __align__(128) unsigned char smem[];
  Stage16* st = reinterpret_cast<Stage16*>(smem);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + NS * sizeof(Stage16));
  IDX* s_base = reinterpret_cast<IDX*>(smem + NS * sizeof(Stage16) + 128);
  const int blk = block_of(a, blockIdx.x);
  const int t = threadIdx.x;
  if (t < 27) s_base[t] = (IDX)a.nbr[(size_t)blk * 27 + t] * (IDX)(27 * C3);
  if (t == 0) {
    for (int k = 0; k < NS; ++k) mbar_init(&bar[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int lx = t & 15, ly = t >> 4;
  const int mo = a.maskoff[blk];
  const uint8_t* mask = mo >= 0 ? a.masks + (size_t)mo * C3 : nullptr;
  const Rates rates{a.omega1, a.omega2, a.galilean};
  float* __restrict__ f = reinterpret_cast<float*>(a.f);
  // this thread's halo copies (threads 32..255 share 300 items)
  HaloItem items[2];
  int nitems = 0;
  if (t >= 32)
    for (int k = t - 32; k < 18 * 16 + 12; k += 256 - 32) items[nitems++] = halo_item(k);
  // prologue: slabs 0 .. NS-2 in flight
  for (int k = 0; k < NS - 1; ++k) stage_issue<IDX>(st[k], &bar[k], f, s_base, k, items, nitems);
  int failed_at = -1;
  for (int lz = 0; lz < B; ++lz) {
    const int cur = lz % NS;
    const int nxt = lz + NS - 1;  // slab to prefetch now
    if (nxt < B) {
      stage_issue<IDX>(st[nxt % NS], &bar[nxt % NS], f, s_base, nxt, items, nitems);
    } else {
      async_commit();
    }
    // one thread observes the bulk copies; the barrier below publishes them
    const bool ok = t != 0 || mbar_wait_bounded(&bar[cur], (uint32_t)((lz / NS) & 1));
    static_assert(NS == 2 || NS == 3, "two or three stages");
    // this thread's 4-byte copies of slab lz are done once at most NS-1 newer groups are pending
    if (NS == 2) asm volatile("cp.async.wait_group 1;" ::: "memory");
    else asm volatile("cp.async.wait_group 2;" ::: "memory");
    if (__syncthreads_or(!ok)) {
      failed_at = lz;
      break;
    }
    const int cell = (lz * B + ly) * B + lx;
    if (!mask || mask[cell]) {
      const Stage16& S = st[cur];
      float d[27];
#pragma unroll
      for (int i = 0; i < 27; ++i) {
        const int sx = lx - dcx(i), sy = ly - dcy(i);
        const bool inx = (unsigned)sx < 16u, iny = (unsigned)sy < 16u;
        float v;
        if (dcx(i) == 0 && dcy(i) == 0) v = S.in[i][t];
        else if (dcx(i) == 0) v = iny ? S.in[i][sy * 16 + lx] : S.yh[i][lx];
        else if (dcy(i) == 0) v = inx ? S.in[i][ly * 16 + sx] : S.xh[i][ly];
        else v = (inx && iny) ? S.in[i][sy * 16 + sx] : (iny ? S.xh[i][sy] : (inx ? S.yh[i][sx] : S.cn[i]));
        d[i] = v;
      }
      cumulant_collide(d, rates);
#pragma unroll
      for (int i = 0; i < 27; ++i) {
        const int nx = lx + dcx(i), ny = ly + dcy(i), nz = lz + dcz(i);
        const int bd = block_digit<B>(nx) + 3 * block_digit<B>(ny) + 9 * block_digit<B>(nz);
        const int nc = ((nz & (B - 1)) * B + (ny & (B - 1))) * B + (nx & (B - 1));
        f[s_base[bd] + (IDX)(i * C3 + nc)] = d[i];
      }
    }
    // every thread is done with stage cur before it is refilled
    __syncthreads();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (failed_at >= 0) {
    if (t == 0 && a.err) *a.err = 1.0;
    // bounded wait for the copies still in flight: slab failed_at and the
    // prefetched slab failed_at + 1
    if (t == 0)
      for (int z = failed_at; z < failed_at + NS - 1 + 1 && z < B; ++z)
        mbar_wait_bounded(&bar[z % NS], (uint32_t)((z / NS) & 1));
    async_wait_all();
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Even step through shared memory (B = 16): every population of a cell stays
// in its cell, so slab z of the 27 planes of the block (27 x 1 KB contiguous)
// is bulk-loaded, collided in place (f*_i goes to the position of plane ibar),
// and bulk-stored back.  Cells that are not updated keep their loaded values,
// so the store writes them back unchanged.  Four stages: slab z + 2 loads
// while slab z is collided and slab z - 1 is still being stored.
constexpr int kEvenStages = 4;
constexpr int kEvenBytes = kEvenStages * 27 * 1024 + 128;

__device__ __forceinline__ void bulk_store(void* gdst, const void* ssrc, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(smem_u32(ssrc)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

template <typename IDX>
__global__ void __launch_bounds__(256, 2) k_collide_even_tma(CollideArgs a) {
  constexpr int C3 = 4096, NS = kEvenStages;
  extern __shared__ __align__(128) unsigned char smem[];
  float(*st)[27][256] = reinterpret_cast<float(*)[27][256]>(smem);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + NS * 27 * 1024);
  const int blk = block_of(a, blockIdx.x);
  const int t = threadIdx.x;
  const IDX own = (IDX)a.nbr[(size_t)blk * 27 + 13] * (IDX)(27 * C3);
  float* __restrict__ fb = reinterpret_cast<float*>(a.f) + own;
  if (t == 0) {
    for (int k = 0; k < NS; ++k) mbar_init(&bar[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int mo = a.maskoff[blk];
  const uint8_t* mask = mo >= 0 ? a.masks + (size_t)mo * C3 : nullptr;
  const Rates rates{a.omega1, a.omega2, a.galilean};
  // warp 0 issues the bulk copies: lane i handles plane i, loads and stores.
  // Bulk store groups are per thread, so before reloading its plane's region
  // of a stage a lane waits until its own older store has read it (only its
  // newest store may still pend).
  auto issue_load = [&](int z) {
    if (t < 32) {
      const int s = z % NS;
      if (t < 27) bulk_wait_read1();
      if (t == 0) mbar_arrive_tx(&bar[s], 27 * 1024);
      __syncwarp();
      if (t < 27) bulk_load(st[s][t], fb + (IDX)(t * C3 + z * 256), 1024, &bar[s]);
    }
  };
  issue_load(0);
  issue_load(1);
  int failed_at = -1;
  for (int z = 0; z < 16; ++z) {
    const int cur = z % NS;
    // stage (z+2)%NS last held slab z-2, stored two iterations ago
    if (z + 2 < 16) issue_load(z + 2);
    const bool ok = t != 0 || mbar_wait_bounded(&bar[cur], (uint32_t)((z / NS) & 1));
    if (__syncthreads_or(!ok)) {
      failed_at = z;
      break;
    }
    const int cell = z * 256 + t;
    if (!mask || mask[cell]) {
      float d[27];
#pragma unroll
      for (int i = 0; i < 27; ++i) d[i] = st[cur][i][t];
      cumulant_collide(d, rates);
#pragma unroll
      for (int i = 0; i < 27; ++i) st[cur][26 - i][t] = d[i];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (t < 27) {
      bulk_store(fb + (IDX)(t * C3 + z * 256), st[cur][t], 1024);
      bulk_commit();
    }
  }
  if (failed_at >= 0) {
    if (t == 0 && a.err) *a.err = 1.0;
    // loads of slabs failed_at .. failed_at + 2 may still be in flight
    if (t == 0)
      for (int z = failed_at; z <= failed_at + 2 && z < 16; ++z)
        mbar_wait_bounded(&bar[z % NS], (uint32_t)((z / NS) & 1));
  }
  if (t < 27) bulk_wait_all();
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Odd step with per-thread column pointers.  A thread walks its (x, y) column
// through z.  Away from the block's z faces every neighbour x + c (and
// x - c) lies in one of 9 columns (dx, dy) of this block or of its x/y
// neighbours, at slab z + cz; with a pointer to each of those 9 columns,
// advanced by one slab per iteration, every pull and push is a single
// memory instruction with a constant offset (plane and dz).  On the two
// z-face slabs, where 9 directions reach into the z neighbours, the pointers
// are built per c_z group for the slab that group reaches (the branch is
// uniform across the CTA).
template <int B, typename IDX, typename S>
__device__ __forceinline__ void odd_cols_block(const CollideArgs& a, const int blk, IDX* s_base, IDX* s_col,
                                               int z0 = 0, int z1 = B) {
  constexpr int C3 = B * B * B, S2 = B * B;
  const int t = threadIdx.x;
  if (t < 27) s_base[t] = (IDX)a.nbr[(size_t)blk * 27 + t] * (IDX)(27 * C3);
  __syncthreads();
  const int lx = t % B, ly = t / B;
  S* __restrict__ f = reinterpret_cast<S*>(a.f);
  // FP16: element offsets of the thread's 9 neighbour columns at slab 0 kept
  // in shared memory (s_col[k * B * B + t], read only by this thread), which
  // makes each rebuild one load and one add per column; FP32 recomputes them
  // (measured: the 9 KB per CTA cost the FP32 step more L1 than it saved)
  constexpr bool kSmemCols = std::is_same<S, __half>::value;
  if (kSmemCols) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int nx = lx + (k % 3 - 1), ny = ly + (k / 3 - 1);
      const int xyd = block_digit<B>(nx) + 3 * block_digit<B>(ny);
      s_col[k * S2 + t] = s_base[xyd + 9] + (IDX)((ny & (B - 1)) * B + (nx & (B - 1)));
    }
  }
  // the 9 column pointers of the (x, y) neighbourhood at slab lz, rebuilt
  // from shared memory before the pull and again after the collision so
  // that none of them is live across it (saves ~20 registers per thread)
  auto cols = [&](S** col, int lz) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      if (kSmemCols) {
        col[k] = f + (s_col[k * S2 + t] + (IDX)(lz * S2));
      } else {
        const int nx = lx + (k % 3 - 1), ny = ly + (k / 3 - 1);
        const int xyd = block_digit<B>(nx) + 3 * block_digit<B>(ny);
        col[k] = f + s_base[xyd + 9] + (IDX)((lz * B + (ny & (B - 1))) * B + (nx & (B - 1)));
      }
    }
  };
  // the 9 column pointers at slab zs in [-1, B]: of this block's (x, y)
  // neighbourhood or of its z neighbour's (the z-face slabs, per c_z group)
  auto zcols = [&](S** col, int zs) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int nx = lx + (k % 3 - 1), ny = ly + (k / 3 - 1);
      const int bd = block_digit<B>(nx) + 3 * block_digit<B>(ny) + 9 * block_digit<B>(zs);
      col[k] = f + s_base[bd] + (IDX)(((zs & (B - 1)) * B + (ny & (B - 1))) * B + (nx & (B - 1)));
    }
  };
  const int mo = a.maskoff[blk];
  const uint8_t* mask = mo >= 0 ? a.masks + (size_t)mo * C3 : nullptr;
  const Rates rates{a.omega1, a.omega2, a.galilean};
  for (int lz = z0; lz < z1; ++lz) {
    const int cell = (lz * B + ly) * B + lx;
    const bool face = lz == 0 || lz == B - 1;
    if (!mask || mask[cell]) {
      float d[27];
      if (!face) {
        S* col[9];
        cols(col, lz);
#pragma unroll
        for (int i = 0; i < 27; ++i)  // pull f_i from (x - c_i, ibar)
          d[i] = Store<S>::ld(col[(1 - dcx(i)) + 3 * (1 - dcy(i))], (26 - i) * C3 - dcz(i) * S2);
      } else {
#pragma unroll
        for (int g = -1; g <= 1; ++g) {  // directions pulling from slab lz + g (c_z = -g)
          S* col[9];
          zcols(col, lz + g);
#pragma unroll
          for (int i = 0; i < 27; ++i)
            if (-dcz(i) == g) d[i] = Store<S>::ld(col[(1 - dcx(i)) + 3 * (1 - dcy(i))], (26 - i) * C3);
        }
      }
      cumulant_collide_s<Store<S>::scaled>(d, rates, a.inv_scale, a.scale, &a.ref);
      asm volatile("" ::: "memory");  // keep the pointer rebuild after the collision
      if (!face) {
        S* col[9];
        cols(col, lz);
#pragma unroll
        for (int i = 0; i < 27; ++i)  // push f*_i to (x + c_i, i)
          Store<S>::st(col[(1 + dcx(i)) + 3 * (1 + dcy(i))], i * C3 + dcz(i) * S2, d[i]);
      } else {
#pragma unroll
        for (int g = -1; g <= 1; ++g) {  // directions pushing into slab lz + g (c_z = g)
          S* col[9];
          zcols(col, lz + g);
#pragma unroll
          for (int i = 0; i < 27; ++i)
            if (dcz(i) == g) Store<S>::st(col[(1 + dcx(i)) + 3 * (1 + dcy(i))], i * C3, d[i]);
        }
      }
    }
  }
}

template <int B, typename IDX, typename S>
__global__ void __launch_bounds__(B * B, odd_minb<S>()) k_collide_odd_cols(CollideArgs a) {
  __shared__ IDX s_base[27];
  __shared__ IDX s_col[std::is_same<S, __half>::value ? 9 * B * B : 1];
  const ZSeg zg = z_segment(a, blockIdx.x, a.zshift_odd, B);
  odd_cols_block<B, IDX, S>(a, zg.blk, s_base, s_col, zg.z0, zg.z1);
}

// Batched, persistent form: the CTAs walk a work list of (level descriptor,
// block) pairs that spans several domains and levels, `gridDim.x` apart.
// KIND 0: even step; 1: odd step, direct addressing; 2: odd step, column
// pointers; 3: even step, two cells per thread; 4: odd step, two cells per
// thread (KIND 3 and 4 run B * B / 2 threads).
template <int KIND>
constexpr int batch_minb() {
  return KIND == 0 ? LBM_EVEN_MINB : (KIND >= 3 ? LBM_PAIR_MINB : LBM_ODD_MINB);
}
template <int B, int KIND, typename IDX, typename S>
__global__ void __launch_bounds__(KIND >= 3 ? B * B / 2 : B * B, batch_minb<KIND>())
    k_collide_batch(const CollideArgs* __restrict__ lv, const int2* __restrict__ items, int n, int zshift) {
  __shared__ IDX s_base[27];
  __shared__ IDX s_col[KIND == 2 && std::is_same<S, __half>::value ? 9 * B * B : 1];
  for (int it = blockIdx.x; it < (n << zshift); it += gridDim.x) {
    const ZSeg zg = z_segment(it, zshift, B);
    const int2 w = items[zg.blk];
    const CollideArgs a = lv[w.x];
    __syncthreads();  // the previous item's readers of s_base are done
    if (KIND == 2) odd_cols_block<B, IDX, S>(a, w.y, s_base, s_col, zg.z0, zg.z1);
    else if (KIND == 3) even_pair_block<B, IDX, S>(a, w.y, zg);
    else if (KIND == 4) odd_pair_block<B, IDX, S>(a, w.y, s_base, zg);
    else collide_block<B, KIND == 1, IDX, S>(a, w.y, s_base, zg.z0, zg.z1);
  }
}

}  // namespace
}  // namespace lbm
