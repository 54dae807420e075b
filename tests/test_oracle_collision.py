"""Pins of the oracle's D3Q27 cumulant collision (Sec. 2.2, Geier et al. 2015).

* cumulants against a brute-force exact Taylor expansion of
  log sum_i f_i exp(Xi . c_i) in rational arithmetic (independent of the
  oracle's set-partition formulas);
* the equilibrium against its defining moments;
* textbook special cases of the collision: all rates one gives the
  factorised equilibrium, all rates zero gives the identity, the rest state
  is a fixed point, mass and momentum are conserved;
* with ten distinct rates, every cumulant group (measured by the brute-force
  expansion) relaxes by its own rate.
"""
from fractions import Fraction
from itertools import product
import math

import numpy as np
import pytest

import oracle as O

C27 = np.array([[i % 3 - 1, (i // 3) % 3 - 1, i // 9 - 1] for i in range(27)])


def _mul(a, b):
    out = {}
    for (ea, ca) in a.items():
        for (eb, cb) in b.items():
            e = (ea[0] + eb[0], ea[1] + eb[1], ea[2] + eb[2])
            if max(e) > 2:
                continue  # only exponents <= 2 per variable are needed
            out[e] = out.get(e, 0) + ca * cb
    return out


def brute_force_cumulants(f):
    """k_abc = a! b! c! [x^a y^b z^c] log( sum_i f_i exp(x cx + y cy + z cz) )."""
    M = {}
    for i, fi in enumerate(f):
        term = {(0, 0, 0): Fraction(fi)}
        for ax in range(3):
            c = int(C27[i, ax])
            e1 = [0, 0, 0]
            e2 = [0, 0, 0]
            e1[ax] = 1
            e2[ax] = 2
            fac = {(0, 0, 0): Fraction(1), tuple(e1): Fraction(c), tuple(e2): Fraction(c * c, 2)}
            term = _mul(term, fac)
        for e, v in term.items():
            M[e] = M.get(e, 0) + v
    m0 = M[(0, 0, 0)]
    X = {e: v / m0 for e, v in M.items() if e != (0, 0, 0)}
    logm = {}
    P = {(0, 0, 0): Fraction(1)}
    for k in range(1, 7):
        P = _mul(P, X)
        for e, v in P.items():
            logm[e] = logm.get(e, 0) + Fraction((-1) ** (k + 1), k) * v
    out = np.zeros(27)
    out[0] = float(m0)
    for a, b, c in product(range(3), repeat=3):
        if (a, b, c) == (0, 0, 0):
            continue
        out[a + 3 * b + 9 * c] = float(logm.get((a, b, c), 0) * math.factorial(a) * math.factorial(b) * math.factorial(c))
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cumulants_match_brute_force_log_expansion(seed):
    rng = np.random.default_rng(seed)
    w = O.equilibrium(1.0, [0.0, 0.0, 0.0])
    fr = [Fraction(int(round(1e6 * wi * (1 + 0.2 * rng.standard_normal()))), 10 ** 6) for wi in w]
    want = brute_force_cumulants(fr)
    got = O.cumulants(np.array([float(x) for x in fr]))
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("u", [(0, 0, 0), (0.05, -0.02, 0.03), (0.2, 0.1, -0.15)])
def test_equilibrium_moments(u):
    rho = 1.03
    f = O.equilibrium(rho, u)
    u = np.array(u)
    assert f.sum() == pytest.approx(rho, rel=1e-14)
    np.testing.assert_allclose(f @ C27, rho * u, atol=1e-15)
    second = np.einsum("i,ia,ib->ab", f, C27, C27)
    np.testing.assert_allclose(second, rho * (np.eye(3) / 3 + np.outer(u, u)), atol=1e-15)
    k = O.cumulants(f)
    np.testing.assert_allclose([k[2], k[6], k[18]], 1.0 / 3.0, atol=1e-14)
    mask = np.ones(27, bool)
    mask[[0, 1, 3, 9, 2, 6, 18]] = False
    np.testing.assert_allclose(k[mask], 0.0, atol=1e-14)


def _perturbed(seed, amp=0.05, u=(0.03, -0.01, 0.02)):
    rng = np.random.default_rng(seed)
    return O.equilibrium(1.0, u) * (1 + amp * rng.standard_normal(27))


@pytest.mark.parametrize("galilean", [True, False])
def test_collision_conserves_mass_and_momentum(galilean):
    for seed in range(5):
        f = _perturbed(seed)
        out = O.collide(f, O.rates(1.83, 1.0, galilean=galilean))
        assert out.sum() == pytest.approx(f.sum(), abs=1e-15)
        np.testing.assert_allclose(out @ C27, f @ C27, atol=1e-15)


def test_rest_state_is_fixed_point():
    w = O.equilibrium(1.0, [0, 0, 0])
    for w1 in (0.6, 1.0, 1.95):
        np.testing.assert_allclose(O.collide(w, O.rates(w1)), w, atol=1e-16)


def test_all_rates_one_gives_factorised_equilibrium():
    """Full relaxation of every cumulant yields rho * prod_a Phi(c_a, u_a)."""
    for seed in range(5):
        f = _perturbed(seed, 0.1)
        rho = f.sum()
        u = f @ C27 / rho
        out = O.collide(f, O.rates(1.0, 1.0, galilean=False))
        np.testing.assert_allclose(out, O.equilibrium(rho, u), atol=1e-15)


def test_galilean_correction_vanishes_for_isotropic_second_moments():
    """The correction is proportional to strain-rate estimates built from the
    second-order cumulants; an equilibrium input has none."""
    f = O.equilibrium(1.01, [0.1, -0.05, 0.07])
    out = O.collide(f, O.rates(1.0, 1.0, galilean=True))
    np.testing.assert_allclose(out, f, atol=1e-15)


def test_all_rates_zero_is_identity():
    for seed in range(3):
        f = _perturbed(seed, 0.1)
        out = O.collide(f, O.rates(0.0, 0.0, (0.0,) * 8, galilean=True))
        np.testing.assert_allclose(out, f, atol=2e-15)


def test_shear_cumulant_relaxes_by_one_minus_omega():
    """An off-diagonal second-order cumulant decays by (1 - omega1); the
    others are set to equilibrium when their rates are one."""
    f = _perturbed(7, 0.1)
    k0 = O.cumulants(f)
    w1 = 1.6
    k1 = O.cumulants(O.collide(f, O.rates(w1, 1.0, galilean=False)))
    for idx in (4, 10, 12):  # k110, k101, k011
        assert k1[idx] == pytest.approx((1 - w1) * k0[idx], rel=1e-11, abs=1e-16)
    for idx in (13, 8, 26):  # k111, k220, k222
        assert abs(k1[idx]) < 1e-14


def test_body_force_adds_momentum():
    f = _perturbed(3)
    F = (1e-4, -2e-4, 3e-5)
    out = O.collide(f, O.rates(1.7), force=F)
    np.testing.assert_allclose(out @ C27 - f @ C27, F, atol=1e-16)
    assert out.sum() == pytest.approx(f.sum(), abs=1e-15)


def test_each_cumulant_group_relaxes_by_its_own_rate():
    """Geier et al. (2015), the relaxation the paper's cumulant LBM uses
    (Sec. 2.2): with ten distinct rates and no Galilean correction, each
    group of cumulants moves toward its equilibrium by (1 - omega) of its own
    rate - omega1 the off-diagonal and deviatoric second order, omega2 the
    trace (equilibrium 1 = 3 c_s^2), omega3 / omega4 the sums / differences
    of the third-order pairs, omega5 k111, omega6 the two fourth-order
    differences, omega7 their sum, omega8 k211 and its permutations, omega9
    fifth order, omega10 sixth order.  Both sides are cumulants from the
    brute-force rational expansion, so this pins the general-rate branches
    of the oracle's relaxation independently of its own transform."""
    f = _perturbed(11, 0.1)
    w1, w2 = 1.37, 0.61
    hi = (0.23, 1.71, 0.48, 1.29, 0.87, 1.53, 0.35, 1.91)  # omega3 .. omega10
    out = O.collide(f, O.rates(w1, w2, hi, galilean=False))
    kb = brute_force_cumulants([Fraction(x) for x in f])
    ka = brute_force_cumulants([Fraction(x) for x in out])

    def K(k, a, b, c):
        return k[a + 3 * b + 9 * c]

    def check(expr, omega, eq=0.0):
        before, after = expr(kb), expr(ka)
        assert after - eq == pytest.approx((1 - omega) * (before - eq), rel=1e-9, abs=1e-15)

    for (a, b, c) in ((1, 1, 0), (1, 0, 1), (0, 1, 1)):
        check(lambda k: K(k, a, b, c), w1)
    check(lambda k: K(k, 2, 0, 0) - K(k, 0, 2, 0), w1)
    check(lambda k: K(k, 2, 0, 0) - K(k, 0, 0, 2), w1)
    check(lambda k: K(k, 2, 0, 0) + K(k, 0, 2, 0) + K(k, 0, 0, 2), w2, eq=1.0)
    for (p, q) in (((1, 2, 0), (1, 0, 2)), ((2, 1, 0), (0, 1, 2)), ((2, 0, 1), (0, 2, 1))):
        check(lambda k: K(k, *p) + K(k, *q), hi[0])
        check(lambda k: K(k, *p) - K(k, *q), hi[1])
    check(lambda k: K(k, 1, 1, 1), hi[2])
    check(lambda k: K(k, 2, 2, 0) - 2 * K(k, 2, 0, 2) + K(k, 0, 2, 2), hi[3])
    check(lambda k: K(k, 2, 2, 0) + K(k, 2, 0, 2) - 2 * K(k, 0, 2, 2), hi[3])
    check(lambda k: K(k, 2, 2, 0) + K(k, 2, 0, 2) + K(k, 0, 2, 2), hi[4])
    for idx in ((2, 1, 1), (1, 2, 1), (1, 1, 2)):
        check(lambda k: K(k, *idx), hi[5])
    for idx in ((2, 2, 1), (2, 1, 2), (1, 2, 2)):
        check(lambda k: K(k, *idx), hi[6])
    check(lambda k: K(k, 2, 2, 2), hi[7])
    # mass and momentum (first-order cumulants are the velocity) unchanged
    assert ka[0] == pytest.approx(kb[0], rel=1e-14)
    np.testing.assert_allclose([ka[1], ka[3], ka[9]], [kb[1], kb[3], kb[9]], rtol=1e-12, atol=1e-16)
