"""Pins for the friction-force oracle (no GPU): the stress of a Chapman-Enskog
state is 2 rho nu S exactly; a simple shear drags a wall along the flow with
rho nu gamma per area; the quadrature areas add up to the analytic surface;
in a body-force channel the friction on the two walls balances the body force
on the fluid between the true wall positions (no pressure drag in a periodic
channel); the library's
quadrature points (host code) equal the oracle's restatement."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import friction as Fr
from paper_2603_27954_gb300 import lbm as L
from paper_2603_27954_gb300 import workloads as W

W27 = O.equilibrium(1.0, np.zeros(3))
CS2 = 1.0 / 3.0


def ce_state(rho, u, S, omega):
    """f = f_eq + f1 with f1_i = -(rho w_i / (cs^2 omega)) (c_i c_i - cs^2 I) : S."""
    feq = O.equilibrium(rho, np.asarray(u, float))
    Q = np.einsum("ia,ib->iab", Fr.C27, Fr.C27) - CS2 * np.eye(3)
    f1 = -(rho * W27 / (CS2 * omega)) * np.einsum("iab,ab->i", Q, S)
    return feq + f1


def test_chapman_enskog_stress_is_two_rho_nu_s():
    rng = np.random.default_rng(1)
    for _ in range(5):
        A = rng.standard_normal((3, 3)) * 1e-3
        S = 0.5 * (A + A.T)
        S -= np.trace(S) / 3 * np.eye(3)
        rho, u, om = 1.0 + 0.01 * rng.standard_normal(), 0.05 * rng.standard_normal(3), rng.uniform(0.6, 1.9)
        nu = CS2 * (1.0 / om - 0.5)
        sig = Fr.cell_stress(ce_state(rho, u, S, om), om)
        np.testing.assert_allclose(sig, 2 * rho * nu * S, atol=1e-15)


def test_shear_drags_the_wall_along_the_flow():
    """u_x = gamma y above a wall with normal +y: friction rho nu gamma dA along +x."""
    gamma, om, rho = 2e-3, 1.2, 1.0
    S = np.zeros((3, 3))
    S[0, 1] = S[1, 0] = gamma / 2
    f = ce_state(rho, (0.01, 0.0, 0.0), S, om)
    rows = np.array([[0, 1, 0, -1e9, -1e9, -1e9, 0, 1, 0, 0.25, 1.5, 0, 0]], float)
    F = Fr.friction(rows, lambda c: np.repeat(f[None, :], len(c), axis=0), om)
    nu = CS2 * (1 / om - 0.5)
    np.testing.assert_allclose(F[0], [rho * nu * gamma * 0.25, 0, 0], atol=1e-16)


def test_quadrature_areas():
    seg = (3.0, 4.0, 5.0, 3.0 + 7.0, 4.0 + 2.0, 5.0 + 9.0, 2.6, 0)
    pts = Fr.cylinder_points(seg)
    L_ = math.sqrt(49 + 4 + 81)
    r = 1.3
    assert sum(p[2] for p in pts) == pytest.approx(2 * math.pi * r * L_ + 2 * math.pi * r * r, rel=1e-12)
    for x, n, _ in pts:  # every point on the surface, unit normal
        assert abs(np.linalg.norm(n) - 1) < 1e-12
    pl = Fr.plane_points((0.0, 1.0, 0.0, 2.5), (0, 0, 0), (6, 10, 4))
    assert sum(p[2] for p in pl) == pytest.approx(24.0, rel=1e-12)
    assert all(abs(x[1] - 2.5) < 1e-12 for x, _, _ in pl)


@pytest.mark.parametrize("o", [0.0, 0.3])
def test_channel_wall_friction_balances_the_body_force(o):
    nu, g, N = 1.0 / 6.0, 1e-5, 16
    ny = N + 4
    ya, yb = 2.0 + o, ny - 2.0 - o
    items = [(1, (0, 1, 0, ya)), (1, (0, -1, 0, -yb))]
    s = O.Sim(1, ny, 1, bc=("periodic",) * 3, nu0=nu, u_in=0.0, force=(g, 0, 0))
    s.set_prims(O.prims(items))
    s.step(int(8 * (yb - ya) ** 2 / nu))
    types = s.cell_type(0)
    f = s.f(0)

    def fluid(c):
        c = np.asarray(c) % np.array([1, ny, 1])
        return types[c[2], c[1], c[0]] == 0

    def pops(c):
        c = np.asarray(c) % np.array([1, ny, 1])
        return f[c[:, 2], c[:, 1], c[:, 0]]

    rows = Fr.samples(items, (0, 0, 0), (1, ny, 1), fluid)
    assert len(rows) == 8 and np.allclose(rows[:, 9].sum(), 2.0)
    F = Fr.friction(rows, pops, 1.0 / (3 * nu + 0.5)).sum(axis=0)
    # the shear at the true walls carries the body force on the fluid between
    # them: g (yb - ya) per unit wall area (the bounce-back places the walls
    # at ya and yb whatever the node count)
    np.testing.assert_allclose(F, [g * (yb - ya), 0, 0], rtol=2e-3, atol=1e-12)


@pytest.mark.parametrize("case", ["tiny", "amr2_small", "amr2_quarter"])
def test_library_quadrature_matches_oracle(case):
    c = W.CASES[case]
    d = L.domain_desc(*c["n0"], levels=c["levels"], block=c["block"], bc=c["bc"], u_in=c["u_in"],
                      re_h=c["re_h"])
    h = L.lbm_create_domain(d)
    L.lbm_set_geometry(h, L.tree_desc(**c["tree"]))
    lib_rows = L.lbm_friction_samples(h)
    seg = L.lbm_get_segments(h)
    lv = c["levels"] - 1
    info = L.lbm_level_info(h, lv)
    types = L.lbm_get_cell_types(h, lv)
    L.lbm_destroy(h)
    lo, hi = np.array(info["lo"]), np.array(info["hi"])

    def fluid(cc):
        cc = np.asarray(cc)
        if np.any(cc < lo) or np.any(cc >= hi):
            return False
        q = cc - lo
        return types[q[2], q[1], q[0]] == 0

    ref = Fr.samples([(0, s) for s in seg], lo, hi, fluid)
    assert lib_rows.shape == ref.shape
    np.testing.assert_array_equal(lib_rows[:, [0, 1, 2, 3, 4, 5, 12]], ref[:, [0, 1, 2, 3, 4, 5, 12]])
    np.testing.assert_allclose(lib_rows[:, 6:12], ref[:, 6:12], rtol=1e-6, atol=1e-6)
