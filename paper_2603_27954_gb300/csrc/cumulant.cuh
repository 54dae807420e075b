// D3Q27 cumulant collision (Sec. 2.2; Geier et al. 2015) on one cell, in
// FP32 (or FP64 for the double-precision storage form), for the rate set omega1 (shear), omega2 (bulk) and all third- to
// sixth-order cumulants relaxed fully to their zero equilibrium.
//
// Populations are carried as deviations d_i = f_i - w_i from the rest
// weights w_i (product weights 2/3, 1/6 per axis), so that the small
// quantities rho - 1, rho u and the non-equilibrium second moments keep
// full FP32 precision.
//
// With third and higher cumulants at zero after the collision, the
// post-collision distribution is fixed by rho, u and the six relaxed
// second-order cumulants: its central moments follow from the
// moment-cumulant relation (products of second-order cumulants, odd orders
// zero).  Writing m* for those normalised central moments and m_w for the
// central moments of the rest weights about u (a tensor product of the
// per-axis triplets 1, -u, 1/3 + u^2), the deviation of the result is
//      d*_i = rho * L_u(m* - m_w)_i + (rho - 1) w_i,
// where L_u maps central moments about u to populations (three passes of
// the 1-D map (M0, M1, M2) -> f_{-1}, f_0, f_{+1}).  Every entry of
// m* - m_w is formed from small quantities, so nothing cancels.
//
// The arithmetic is written once over a number type T:
//   Fp  plain FP32 (the compiler may contract a * b + c into one FMA);
//   Fd  plain FP64 (the FP64 storage form; all constants exact to double);
//   F2  two cells in one 64-bit register, Blackwell's packed FP32
//       instructions (add/sub/mul/fma .rn.f32x2): half the arithmetic
//       instructions of two one-cell collisions.  The assembler contracts a
//       packed multiply followed by a packed add into a packed FMA where it
//       sees fit (measured on sm_103a), so F2 results equal neither the
//       rounded-as-written nor the Fp ones bit for bit; a one-cell kernel that
//       must match a two-cell one runs the F2 code with the cell in both lanes.
#pragma once

#include <math.h>

#include "internal.h"  // RefShift

namespace lbm {

struct Rates {
  float omega1, omega2;
  int galilean;
};

#define LBM_DI __device__ __forceinline__

struct Fp {
  float v;
  static LBM_DI Fp make(float a) { return Fp{a}; }
  // constants written as double quotients (1.0 / 3.0 ...) round to the same
  // float as the float quotients for every constant below
  static LBM_DI Fp make(double a) { return Fp{(float)a}; }
};
LBM_DI Fp operator+(Fp a, Fp b) { return Fp{a.v + b.v}; }
LBM_DI Fp operator-(Fp a, Fp b) { return Fp{a.v - b.v}; }
LBM_DI Fp operator*(Fp a, Fp b) { return Fp{a.v * b.v}; }
LBM_DI Fp fma(Fp a, Fp b, Fp c) { return Fp{fmaf(a.v, b.v, c.v)}; }
LBM_DI Fp neg(Fp a) { return Fp{-a.v}; }
LBM_DI Fp recip(Fp a) { return Fp{1.0f / a.v}; }

struct F2 {
  unsigned long long v;
  static LBM_DI F2 pack(float lo, float hi) {
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
    return r;
  }
  static LBM_DI F2 make(float a) { return pack(a, a); }
  static LBM_DI F2 make(double a) { return pack((float)a, (float)a); }
  LBM_DI float lo() const {
    float a;
    asm("mov.b64 {%0, _}, %1;" : "=f"(a) : "l"(v));
    return a;
  }
  LBM_DI float hi() const {
    float b;
    asm("mov.b64 {_, %0}, %1;" : "=f"(b) : "l"(v));
    return b;
  }
};
LBM_DI F2 operator+(F2 a, F2 b) {
  F2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
LBM_DI F2 operator-(F2 a, F2 b) {
  F2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
LBM_DI F2 operator*(F2 a, F2 b) {
  F2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
LBM_DI F2 fma(F2 a, F2 b, F2 c) {
  F2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}
LBM_DI F2 neg(F2 a) { return a * F2::make(-1.0f); }
LBM_DI F2 recip(F2 a) { return F2::pack(__fdiv_rn(1.0f, a.lo()), __fdiv_rn(1.0f, a.hi())); }

// FP64 (the double-precision storage form): plain double arithmetic
struct Fd {
  double v;
  static LBM_DI Fd make(double a) { return Fd{a}; }
};
LBM_DI Fd operator+(Fd a, Fd b) { return Fd{a.v + b.v}; }
LBM_DI Fd operator-(Fd a, Fd b) { return Fd{a.v - b.v}; }
LBM_DI Fd operator*(Fd a, Fd b) { return Fd{a.v * b.v}; }
LBM_DI Fd fma(Fd a, Fd b, Fd c) { return Fd{::fma(a.v, b.v, c.v)}; }
LBM_DI Fd neg(Fd a) { return Fd{-a.v}; }
LBM_DI Fd recip(Fd a) { return Fd{1.0 / a.v}; }

// Coefficients of the relaxation formed from the rates: in FP32 each rate
// product rounded as written (uniform scalars, so that every FP32
// instantiation sees the same coefficients), in FP64 plain double products.
template <class T>
struct RelaxCoef {
  T mhw1, hw2, c15, r1, r2, g1, g2;  // -w1/2, w2/2, 3 w1/2, 1 - w1, 1 - w2, g (1 - w1/2), g (1 - w2/2)
};
struct RatesD {
  double omega1, omega2;
  int galilean;
};
template <class T>
LBM_DI RelaxCoef<T> relax_coef(const Rates& r) {
  const float w1 = r.omega1, w2 = r.omega2;
  const float g = r.galilean ? 3.0f : 0.0f;
  const float hw1 = __fmul_rn(0.5f, w1), hw2 = __fmul_rn(0.5f, w2);
  return RelaxCoef<T>{T::make(-hw1),
                      T::make(hw2),
                      T::make(__fmul_rn(1.5f, w1)),
                      T::make(__fsub_rn(1.0f, w1)),
                      T::make(__fsub_rn(1.0f, w2)),
                      T::make(__fmul_rn(g, __fsub_rn(1.0f, hw1))),
                      T::make(__fmul_rn(g, __fsub_rn(1.0f, hw2)))};
}
template <class T>
LBM_DI RelaxCoef<T> relax_coef(const RatesD& r) {
  const double w1 = r.omega1, w2 = r.omega2;
  const double g = r.galilean ? 3.0 : 0.0;
  return RelaxCoef<T>{T::make(-0.5 * w1),     T::make(0.5 * w2),
                      T::make(1.5 * w1),      T::make(1.0 - w1),
                      T::make(1.0 - w2),      T::make(g * (1.0 - 0.5 * w1)),
                      T::make(g * (1.0 - 0.5 * w2))};
}

// 1-D map from central moments (M0, M1, M2) about u to the three
// populations f(-1), f(0), f(+1): from the raw moments R1 = M1 + u M0 and
// R2 = M2 + 2u M1 + u^2 M0, f(+-1) = (R2 +- R1) / 2 and f(0) = M0 - R2.
// The coefficients depend on u only and are formed once per axis.
template <class T>
struct AxisMap {
  T a0, a1, ap, am, bp, bm;
};
template <class T>
LBM_DI AxisMap<T> axis_map(T u) {
  const T u2 = u * u, h = T::make(0.5f);
  return AxisMap<T>{T::make(1.0f) - u2, u * T::make(-2.0f), h * (u2 + u), h * (u2 - u), u + h, u - h};
}
// plain FP32: f(0) from its own two FMAs (the negation folds into the FMA)
LBM_DI void central_to_pop(Fp m0, Fp m1, Fp m2, const AxisMap<Fp>& A, Fp& fm, Fp& f0, Fp& fp) {
  const Fp h = Fp::make(0.5f) * m2;
  f0 = fma(A.a0, m0, fma(A.a1, m1, neg(m2)));
  fp = fma(A.ap, m0, fma(A.bp, m1, h));
  fm = fma(A.am, m0, fma(A.bm, m1, h));
}
// packed form: f(0) = M0 - f(+1) - f(-1), which needs no negated operand
// (the packed instructions have no operand negation)
template <class T>
LBM_DI void central_to_pop(T m0, T m1, T m2, const AxisMap<T>& A, T& fm, T& f0, T& fp) {
  const T h = T::make(0.5f) * m2;
  fp = fma(A.ap, m0, fma(A.bp, m1, h));
  fm = fma(A.am, m0, fma(A.bm, m1, h));
  f0 = m0 - (fp + fm);
}

// d holds the 27 deviations multiplied by a storage scale s_in on entry and
// receives the post-collision deviations multiplied by s_out (both 1 for FP32
// storage; the FP16 form folds its power-of-two scale into the moment sums
// and the final multiply-add instead of scaling every population, and keeps
// its values relative to the reference `ref`, whose moments j_x = U and
// Pi_xx - 1/3 = U^2 are added before the relaxation and whose populations
// are subtracted from the result).
template <class T, bool SCALED, class R>
LBM_DI void collide_cell(T* d, const R& r, float inv_s_in, float s_out, const RefShift* ref) {
  // ---- raw moments of the deviations: three passes (x, then y, then z)
  T x0[9], x1[9], x2[9];
#pragma unroll
  for (int yz = 0; yz < 9; ++yz) {
    const T a = d[3 * yz], b = d[3 * yz + 1], c = d[3 * yz + 2];
    x0[yz] = a + b + c;
    x1[yz] = c - a;
    x2[yz] = c + a;
  }
  T y00[3], y01[3], y02[3], y10[3], y11[3], y20[3];
#pragma unroll
  for (int z = 0; z < 3; ++z) {
    const int o = 3 * z;
    y00[z] = x0[o] + x0[o + 1] + x0[o + 2];
    y01[z] = x0[o + 2] - x0[o];
    y02[z] = x0[o + 2] + x0[o];
    y10[z] = x1[o] + x1[o + 1] + x1[o + 2];
    y11[z] = x1[o + 2] - x1[o];
    y20[z] = x2[o] + x2[o + 1] + x2[o + 2];
  }
  const T sc = T::make(inv_s_in);
  auto scl = [&](T v) { return SCALED ? v * sc : v; };
  const T drho = scl(y00[0] + y00[1] + y00[2]);
  const T jz = scl(y00[2] - y00[0]);
  const T szz = scl(y00[2] + y00[0]);
  const T jy = scl(y01[0] + y01[1] + y01[2]);
  const T syz = scl(y01[2] - y01[0]);
  const T syy = scl(y02[0] + y02[1] + y02[2]);
  const T jx = SCALED ? fma(y10[0] + y10[1] + y10[2], sc, T::make(ref->u)) : y10[0] + y10[1] + y10[2];
  const T sxz = scl(y10[2] - y10[0]);
  const T sxy = scl(y11[0] + y11[1] + y11[2]);
  const T sxx = SCALED ? fma(y20[0] + y20[1] + y20[2], sc, T::make(ref->u2)) : y20[0] + y20[1] + y20[2];

  const T rho = T::make(1.0f) + drho;
  const T ir = recip(rho);
  const T ux = jx * ir, uy = jy * ir, uz = jz * ir;
  const T ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
  const T third = T::make(1.0 / 3.0), mthird = T::make(-1.0 / 3.0);
  // second-order cumulants (normalised by rho), diagonal ones minus 1/3
  const T dxx = fma(fma(mthird, drho, sxx), ir, neg(ux2));
  const T dyy = fma(fma(mthird, drho, syy), ir, neg(uy2));
  const T dzz = fma(fma(mthird, drho, szz), ir, neg(uz2));
  const T kxy = sxy * ir - ux * uy;
  const T kxz = sxz * ir - ux * uz;
  const T kyz = syz * ir - uy * uz;

  // ---- relaxation (coefficients from the rates: relax_coef)
  const RelaxCoef<T> kc = relax_coef<T>(r);
  const T dxu = kc.mhw1 * (dxx + dxx - dyy - dzz) - kc.hw2 * (dxx + dyy + dzz);
  const T c15 = kc.c15;
  const T dyv = dxu + c15 * (dxx - dyy);
  const T dzw = dxu + c15 * (dxx - dzz);
  const T cx2 = ux2 * dxu, cy2 = uy2 * dyv, cz2 = uz2 * dzw;
  const T r1 = kc.r1, r2 = kc.r2;
  const T g1 = kc.g1, g2 = kc.g2;
  const T A = r1 * (dxx - dyy) - g1 * (cx2 - cy2);
  const T Bq = r1 * (dxx - dzz) - g1 * (cx2 - cz2);
  const T Tr = r2 * (dxx + dyy + dzz) - g2 * (cx2 + cy2 + cz2);
  const T pxx = (A + Bq + Tr) * third;
  const T pyy = pxx - A;
  const T pzz = pxx - Bq;
  const T qxy = r1 * kxy, qxz = r1 * kxz, qyz = r1 * kyz;

  // ---- m* - m_w, indexed a + 3b + 9c
  const T ax = third + ux2, ay = third + uy2, az = third + uz2;
  const T ex = pxx - ux2, ey = pyy - uy2, ez = pzz - uz2;
  const T sxx2 = ax + ex, syy2 = ay + ey, szz2 = az + ez;
  const T two = T::make(2.0f);
  T m[27];
  m[0] = T::make(0.0f);
  m[1] = ux;
  m[3] = uy;
  m[9] = uz;
  m[2] = ex;
  m[6] = ey;
  m[18] = ez;
  m[4] = qxy - ux * uy;
  m[10] = qxz - ux * uz;
  m[12] = qyz - uy * uz;
  m[5] = uy * ax;   // 210
  m[11] = uz * ax;  // 201
  m[7] = ux * ay;   // 120
  m[15] = uz * ay;  // 021
  m[19] = ux * az;  // 102
  m[21] = uy * az;  // 012
  m[13] = ux * uy * uz;  // 111
  m[8] = ax * ey + ay * ex + ex * ey + two * qxy * qxy;    // 220
  m[20] = ax * ez + az * ex + ex * ez + two * qxz * qxz;   // 202
  m[24] = ay * ez + az * ey + ey * ez + two * qyz * qyz;   // 022
  m[14] = ax * m[12] + ex * qyz + two * qxy * qxz;         // 211
  m[16] = ay * m[10] + ey * qxz + two * qxy * qyz;         // 121
  m[22] = az * m[4] + ez * qxy + two * qxz * qyz;          // 112
  m[17] = ax * ay * uz;  // 221
  m[23] = ax * az * uy;  // 212
  m[25] = ay * az * ux;  // 122
  m[26] = ax * ay * ez + ax * ey * az + ex * ay * az + ax * ey * ez + ex * ay * ez + ex * ey * az + ex * ey * ez +
          two * (sxx2 * qyz * qyz + syy2 * qxz * qxz + szz2 * qxy * qxy) + T::make(8.0f) * qxy * qxz * qyz;  // 222

  // ---- back to populations: z pass, y pass, x pass
  const AxisMap<T> Mx = axis_map(ux), My = axis_map(uy), Mz = axis_map(uz);
  T t[27];
#pragma unroll
  for (int ab = 0; ab < 9; ++ab)  // moment index a + 3b, population cz
    central_to_pop(m[ab], m[ab + 9], m[ab + 18], Mz, t[ab], t[ab + 9], t[ab + 18]);
#pragma unroll
  for (int zc = 0; zc < 3; ++zc)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int o = 9 * zc + a;  // moment a, moment b (stride 3), population cz
      T p0, p1, p2;
      central_to_pop(t[o], t[o + 3], t[o + 6], My, p0, p1, p2);
      t[o] = p0;
      t[o + 3] = p1;
      t[o + 6] = p2;
    }
  // (rho - 1) w_i for the four distinct rest weights (number of zero
  // components), minus the scaled reference r_i s for the FP16 form
  const T so = T::make(SCALED ? s_out : 1.0f);
  const T rs = rho * so, ds = drho * so;
  const T dw[4] = {ds * T::make(1.0 / 216.0), ds * T::make(1.0 / 54.0), ds * T::make(2.0 / 27.0),
                   ds * T::make(8.0 / 27.0)};
#pragma unroll
  for (int yz = 0; yz < 9; ++yz) {
    const int o = 3 * yz;  // moment a, population cy, cz
    T p0, p1, p2;
    central_to_pop(t[o], t[o + 1], t[o + 2], Mx, p0, p1, p2);
    const int zeros = (yz % 3 == 1) + (yz / 3 == 1);
    if (SCALED) {
      d[o] = fma(rs, p0, dw[zeros] - T::make(ref->out[3 * zeros]));
      d[o + 1] = fma(rs, p1, dw[zeros + 1] - T::make(ref->out[3 * zeros + 1]));
      d[o + 2] = fma(rs, p2, dw[zeros] - T::make(ref->out[3 * zeros + 2]));
    } else {
      d[o] = fma(rs, p0, dw[zeros]);
      d[o + 1] = fma(rs, p1, dw[zeros + 1]);
      d[o + 2] = fma(rs, p2, dw[zeros]);
    }
  }
}

// FP64 storage: plain FP64 arithmetic on one cell (deviations from the rest
// weights, no scale, no reference)
LBM_DI void cumulant_collide_d(double* d, const RatesD& r) {
  collide_cell<Fd, false>(reinterpret_cast<Fd*>(d), r, 1.0f, 1.0f, nullptr);
}
// FP32 storage: plain FP32 arithmetic on one cell
LBM_DI void cumulant_collide(float* d, const Rates& r) {
  collide_cell<Fp, false>(reinterpret_cast<Fp*>(d), r, 1.0f, 1.0f, nullptr);
}
// FP16 storage, one cell, plain FP32 arithmetic
LBM_DI void cumulant_collide_h(float* d, const Rates& r, float inv_s_in, float s_out, const RefShift* ref) {
  collide_cell<Fp, true>(reinterpret_cast<Fp*>(d), r, inv_s_in, s_out, ref);
}
// FP16 storage, one cell run through the packed code in both lanes: the
// result of the two-cell form for this cell, bit for bit
LBM_DI void cumulant_collide_h_as_pair(float* d, const Rates& r, float inv_s_in, float s_out,
                                       const RefShift* ref) {
  F2 p[27];
#pragma unroll
  for (int i = 0; i < 27; ++i) p[i] = F2::make(d[i]);
  collide_cell<F2, true>(p, r, inv_s_in, s_out, ref);
#pragma unroll
  for (int i = 0; i < 27; ++i) d[i] = p[i].lo();
}
// one cell, storage form chosen at compile time
template <bool SCALED>
LBM_DI void cumulant_collide_s(float* d, const Rates& r, float inv_s_in, float s_out, const RefShift* ref = nullptr) {
  if (SCALED) cumulant_collide_h(d, r, inv_s_in, s_out, ref);
  else cumulant_collide(d, r);
}

}  // namespace lbm
