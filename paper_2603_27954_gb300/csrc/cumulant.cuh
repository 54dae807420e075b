// D3Q27 cumulant collision (Sec. 2.2; Geier et al. 2015) on one cell, in
// FP32, for the rate set omega1 (shear), omega2 (bulk) and all third- to
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
#pragma once

#include <math.h>

#include "internal.h"  // RefShift

#ifndef LBM_HD
#define LBM_HD __host__ __device__ __forceinline__
#endif

namespace lbm {

struct Rates {
  float omega1, omega2;
  int galilean;
};


// 1-D map from central moments (M0, M1, M2) about u to the three
// populations f(-1), f(0), f(+1): from the raw moments R1 = M1 + u M0 and
// R2 = M2 + 2u M1 + u^2 M0, f(+-1) = (R2 +- R1) / 2 and f(0) = M0 - R2.
// The coefficients depend on u only and are formed once per axis.
struct AxisMap {
  float a0, a1, ap, am, bp, bm;
};
LBM_HD AxisMap axis_map(float u) {
  const float u2 = u * u;
  return AxisMap{1.0f - u2, -2.0f * u, 0.5f * (u2 + u), 0.5f * (u2 - u), u + 0.5f, u - 0.5f};
}
LBM_HD void central_to_pop(float m0, float m1, float m2, const AxisMap& A, float& fm, float& f0, float& fp) {
  const float h = 0.5f * m2;
  f0 = fmaf(A.a0, m0, fmaf(A.a1, m1, -m2));
  fp = fmaf(A.ap, m0, fmaf(A.bp, m1, h));
  fm = fmaf(A.am, m0, fmaf(A.bm, m1, h));
}

// d holds the 27 deviations multiplied by a storage scale s_in on entry and
// receives the post-collision deviations multiplied by s_out (both 1 for FP32
// storage; the FP16 form folds its power-of-two scale into the moment sums
// and the final multiply-add instead of scaling every population).
template <bool SCALED>
LBM_HD void cumulant_collide_s(float* d, const Rates& r, float inv_s_in, float s_out,
                               const RefShift* ref = nullptr) {
  // ---- raw moments of the deviations: three passes (x, then y, then z)
  float x0[9], x1[9], x2[9];
#pragma unroll
  for (int yz = 0; yz < 9; ++yz) {
    float a = d[3 * yz], b = d[3 * yz + 1], c = d[3 * yz + 2];
    x0[yz] = a + b + c;
    x1[yz] = c - a;
    x2[yz] = c + a;
  }
  float y00[3], y01[3], y02[3], y10[3], y11[3], y20[3];
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
  const float sc = SCALED ? inv_s_in : 1.0f;
  const float drho = (y00[0] + y00[1] + y00[2]) * sc;
  const float jz = (y00[2] - y00[0]) * sc;
  const float szz = (y00[2] + y00[0]) * sc;
  const float jy = (y01[0] + y01[1] + y01[2]) * sc;
  const float syz = (y01[2] - y01[0]) * sc;
  const float syy = (y02[0] + y02[1] + y02[2]) * sc;
  const float jx = SCALED ? fmaf(y10[0] + y10[1] + y10[2], sc, ref->u) : (y10[0] + y10[1] + y10[2]) * sc;
  const float sxz = (y10[2] - y10[0]) * sc;
  const float sxy = (y11[0] + y11[1] + y11[2]) * sc;
  const float sxx = SCALED ? fmaf(y20[0] + y20[1] + y20[2], sc, ref->u2) : (y20[0] + y20[1] + y20[2]) * sc;

  const float rho = 1.0f + drho;
  const float ir = 1.0f / rho;
  const float ux = jx * ir, uy = jy * ir, uz = jz * ir;
  const float ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
  const float third = 1.0f / 3.0f;
  // second-order cumulants (normalised by rho), diagonal ones minus 1/3
  const float dxx = (sxx - third * drho) * ir - ux2;
  const float dyy = (syy - third * drho) * ir - uy2;
  const float dzz = (szz - third * drho) * ir - uz2;
  const float kxy = sxy * ir - ux * uy;
  const float kxz = sxz * ir - ux * uz;
  const float kyz = syz * ir - uy * uz;

  // ---- relaxation
  const float w1 = r.omega1, w2 = r.omega2;
  const float g = r.galilean ? 3.0f : 0.0f;
  const float dxu = -0.5f * w1 * (2.0f * dxx - dyy - dzz) - 0.5f * w2 * (dxx + dyy + dzz);
  const float dyv = dxu + 1.5f * w1 * (dxx - dyy);
  const float dzw = dxu + 1.5f * w1 * (dxx - dzz);
  const float cx2 = ux2 * dxu, cy2 = uy2 * dyv, cz2 = uz2 * dzw;
  const float A = (1.0f - w1) * (dxx - dyy) - g * (1.0f - 0.5f * w1) * (cx2 - cy2);
  const float Bq = (1.0f - w1) * (dxx - dzz) - g * (1.0f - 0.5f * w1) * (cx2 - cz2);
  const float T = (1.0f - w2) * (dxx + dyy + dzz) - g * (1.0f - 0.5f * w2) * (cx2 + cy2 + cz2);
  const float pxx = (A + Bq + T) * third;
  const float pyy = pxx - A;
  const float pzz = pxx - Bq;
  const float qxy = (1.0f - w1) * kxy, qxz = (1.0f - w1) * kxz, qyz = (1.0f - w1) * kyz;

  // ---- m* - m_w, indexed a + 3b + 9c
  const float ax = third + ux2, ay = third + uy2, az = third + uz2;
  const float ex = pxx - ux2, ey = pyy - uy2, ez = pzz - uz2;
  const float sxx2 = ax + ex, syy2 = ay + ey, szz2 = az + ez;
  float m[27];
  m[0] = 0.0f;
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
  m[8] = ax * ey + ay * ex + ex * ey + 2.0f * qxy * qxy;    // 220
  m[20] = ax * ez + az * ex + ex * ez + 2.0f * qxz * qxz;   // 202
  m[24] = ay * ez + az * ey + ey * ez + 2.0f * qyz * qyz;   // 022
  m[14] = ax * m[12] + ex * qyz + 2.0f * qxy * qxz;         // 211
  m[16] = ay * m[10] + ey * qxz + 2.0f * qxy * qyz;         // 121
  m[22] = az * m[4] + ez * qxy + 2.0f * qxz * qyz;          // 112
  m[17] = ax * ay * uz;  // 221
  m[23] = ax * az * uy;  // 212
  m[25] = ay * az * ux;  // 122
  m[26] = ax * ay * ez + ax * ey * az + ex * ay * az + ax * ey * ez + ex * ay * ez + ex * ey * az + ex * ey * ez +
          2.0f * (sxx2 * qyz * qyz + syy2 * qxz * qxz + szz2 * qxy * qxy) + 8.0f * qxy * qxz * qyz;  // 222

  // ---- back to populations: z pass, y pass, x pass
  const AxisMap Mx = axis_map(ux), My = axis_map(uy), Mz = axis_map(uz);
  float t[27];
#pragma unroll
  for (int ab = 0; ab < 9; ++ab)  // moment index a + 3b, population cz
    central_to_pop(m[ab], m[ab + 9], m[ab + 18], Mz, t[ab], t[ab + 9], t[ab + 18]);
#pragma unroll
  for (int zc = 0; zc < 3; ++zc)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int o = 9 * zc + a;  // moment a, moment b (stride 3), population cz
      float p0, p1, p2;
      central_to_pop(t[o], t[o + 3], t[o + 6], My, p0, p1, p2);
      t[o] = p0;
      t[o + 3] = p1;
      t[o + 6] = p2;
    }
  // (rho - 1) w_i for the four distinct rest weights (number of zero components)
  const float so = SCALED ? s_out : 1.0f;
  const float rs = rho * so, ds = drho * so;
  const float dw[4] = {ds * (1.0f / 216.0f), ds * (1.0f / 54.0f), ds * (2.0f / 27.0f), ds * (8.0f / 27.0f)};
#pragma unroll
  for (int yz = 0; yz < 9; ++yz) {
    const int o = 3 * yz;  // moment a, population cy, cz
    float p0, p1, p2;
    central_to_pop(t[o], t[o + 1], t[o + 2], Mx, p0, p1, p2);
    const int zeros = (yz % 3 == 1) + (yz / 3 == 1);
    if (SCALED) {  // back to the stored reference: minus r_i s
      d[o] = fmaf(rs, p0, dw[zeros] - ref->out[3 * zeros]);
      d[o + 1] = fmaf(rs, p1, dw[zeros + 1] - ref->out[3 * zeros + 1]);
      d[o + 2] = fmaf(rs, p2, dw[zeros] - ref->out[3 * zeros + 2]);
    } else {
      d[o] = fmaf(rs, p0, dw[zeros]);
      d[o + 1] = fmaf(rs, p1, dw[zeros + 1]);
      d[o + 2] = fmaf(rs, p2, dw[zeros]);
    }
  }
}

LBM_HD void cumulant_collide(float* d, const Rates& r) { cumulant_collide_s<false>(d, r, 1.0f, 1.0f); }

}  // namespace lbm
