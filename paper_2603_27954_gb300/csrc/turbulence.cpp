// Synthetic turbulent inflow: a random-Fourier-mode velocity field (Kraichnan
// 1970; Smirnov, Shi & Celik 2001) with a von Karman energy spectrum, frozen
// and carried through the inflow plane at the mean speed (Taylor's
// hypothesis).  The paper uses the inflow turbulence intensity I_u (Sec. 4.2)
// only in its analytical model; this field lets the LBM see the same intensity.
//
//   u'(x) = sum_n a_n cos(k_n . x + psi_n),  a_n = 2 u_n sigma_n,  sigma_n . k_n = 0
//
// Mode n takes four uniforms r0..r3 from SplitMix64 in counter form (counter
// 2^40 + 4 n + j, the domain's seed): direction of k_n with cos(theta) =
// 2 r0 - 1 and phi = 2 pi r1; sigma_n = cos(2 pi r2) e1 + sin(2 pi r2) e2 with
// e1 = (-sin phi, cos phi, 0), e2 = d x e1; psi_n = 2 pi r3.  Magnitudes are
// log-spaced over [k_e / 4, min(16 k_e, pi / 4)] with k_e = 0.747 / L_int, and
// u_n^2 = (3/2) I_u^2 U^2 E(k_n) dk_n / sum_m E(k_m) dk_m with the von Karman
// shape E(k) = (k/k_e)^4 / (1 + (k/k_e)^2)^(17/6): the expected stream-wise
// variance (2/3) sum u_n^2 is then (I_u U)^2.  Lengths in level-0 cells.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace lbm {

void rfm_modes(uint64_t seed, int n, double i_u, double u, double l_int, std::vector<double>* out) {
  out->assign((size_t)n * kModeCols, 0.0);
  if (n <= 0) return;
  const double kPi = 3.14159265358979323846;
  const double ke = 0.747 / l_int;
  const double klo = 0.25 * ke, khi = std::max(klo * 1.0001, std::min(16.0 * ke, 0.25 * kPi));
  const double span = std::log(khi / klo);
  std::vector<double> w(n);
  double wsum = 0;
  for (int m = 0; m < n; ++m) {
    const double k = klo * std::exp(span * (m + 0.5) / n);
    const double dk = k * span / n;
    const double r = k / ke;
    w[m] = std::pow(r, 4) / std::pow(1.0 + r * r, 17.0 / 6.0) * dk;
    wsum += w[m];
  }
  auto uni = [&](int m, int j) {
    const uint64_t z = splitmix(seed, (1ULL << 40) + 4ULL * (uint64_t)m + (uint64_t)j);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  for (int m = 0; m < n; ++m) {
    const double k = klo * std::exp(span * (m + 0.5) / n);
    const double ct = 2.0 * uni(m, 0) - 1.0, st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
    const double ph = 2.0 * kPi * uni(m, 1), al = 2.0 * kPi * uni(m, 2), psi = 2.0 * kPi * uni(m, 3);
    const double d[3] = {st * std::cos(ph), st * std::sin(ph), ct};
    const double e1[3] = {-std::sin(ph), std::cos(ph), 0.0};
    const double e2[3] = {-ct * std::cos(ph), -ct * std::sin(ph), st};
    const double un = std::sqrt(1.5 * i_u * i_u * u * u * w[m] / wsum);
    double* row = &(*out)[(size_t)m * kModeCols];
    for (int a = 0; a < 3; ++a) {
      row[a] = k * d[a];
      row[3 + a] = 2.0 * un * (std::cos(al) * e1[a] + std::sin(al) * e2[a]);
    }
    row[6] = psi;
  }
}

}  // namespace lbm
