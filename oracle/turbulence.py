"""Oracle of the synthetic turbulent inflow.

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the CPU
baseline of the benchmark, never by the product path.

Sec. 4.2 defines the inflow turbulence intensity I_u = u'_rms / U; the paper
uses it only in its analytical model.  The LBM inflow here is a random-
Fourier-mode field (Kraichnan 1970; Smirnov, Shi & Celik 2001):

    u'(x) = sum_n 2 u_n sigma_n cos(kappa_n d_n . x + psi_n)

d_n a random unit vector, sigma_n a random unit vector normal to d_n (so the
field is divergence-free), psi_n a random phase, kappa_n log-spaced over
[kappa_e / 4, min(16 kappa_e, pi / 4)] with kappa_e = 0.747 / L_int, and
u_n^2 proportional to the von Karman shape E(kappa) = (kappa/kappa_e)^4 /
(1 + (kappa/kappa_e)^2)^(17/6) times the bin width, normalised so that
sum_n u_n^2 = (3/2) I_u^2 U^2 (expected stream-wise variance (I_u U)^2).
The four uniforms of mode n are SplitMix64 outputs 2^40 + 4 n + j of the
domain's seed (top 53 bits / 2^53): cos(theta) = 2 r0 - 1, phi = 2 pi r1,
polarisation angle 2 pi r2 in the basis e1 = (-sin phi, cos phi, 0),
e2 = d x e1, psi = 2 pi r3.  At the inflow the frozen field is carried at U
(Taylor's hypothesis): u(p, t) = U e_x + u'(p - U t e_x).
"""
import math

import numpy as np

from . import lib


def uniform(seed, k):
    """Output k of SplitMix64 (counter form) as a double in [0, 1)."""
    return (lib().orc_splitmix64(seed, k) >> 11) / 9007199254740992.0


def von_karman(r):
    return r ** 4 / (1.0 + r * r) ** (17.0 / 6.0)


def rfm_modes(seed, n, i_u, u, l_int):
    """Mode table, n x 7: wavevector k (3), amplitude vector a = 2 u_n sigma_n (3), phase psi."""
    ke = 0.747 / l_int
    klo = 0.25 * ke
    khi = max(klo * 1.0001, min(16.0 * ke, 0.25 * math.pi))
    span = math.log(khi / klo)
    kap = klo * np.exp(span * (np.arange(n) + 0.5) / n)
    w = von_karman(kap / ke) * kap * span / n
    un = np.sqrt(1.5 * (i_u * u) ** 2 * w / w.sum())
    out = np.zeros((n, 7))
    for m in range(n):
        r = [uniform(seed, (1 << 40) + 4 * m + j) for j in range(4)]
        ct = 2.0 * r[0] - 1.0
        st = math.sqrt(max(0.0, 1.0 - ct * ct))
        ph, al, psi = 2 * math.pi * r[1], 2 * math.pi * r[2], 2 * math.pi * r[3]
        d = np.array([st * math.cos(ph), st * math.sin(ph), ct])
        e1 = np.array([-math.sin(ph), math.cos(ph), 0.0])
        e2 = np.cross(d, e1)
        out[m, 0:3] = kap[m] * d
        out[m, 3:6] = 2.0 * un[m] * (math.cos(al) * e1 + math.sin(al) * e2)
        out[m, 6] = psi
    return out


def fluctuation(modes, x):
    """u'(x) for points x (..., 3)."""
    x = np.asarray(x, dtype=np.float64)
    ph = x @ modes[:, 0:3].T + modes[:, 6]
    return np.cos(ph) @ modes[:, 3:6]
