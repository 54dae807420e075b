"""Pins for the synthetic turbulent inflow (no GPU): every mode is
divergence-free, the amplitudes carry exactly (3/2) (I_u U)^2, the sampled
field has zero mean, the stream-wise variance its modes predict and zero
numerical divergence, the von Karman shape peaks at sqrt(12/5) kappa_e, the
library's mode table (host code) equals the oracle's restatement, and the
inflow face pulls the equilibrium of the frozen field exactly."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import turbulence as T
from paper_2603_27954_gb300 import lbm as L

I_U, U, LINT, SEED = 0.08, 0.05, 24.0, 77


@pytest.fixture(scope="module")
def modes():
    return T.rfm_modes(SEED, 256, I_U, U, LINT)


def test_modes_are_divergence_free_and_normalised(modes):
    k, a = modes[:, 0:3], modes[:, 3:6]
    np.testing.assert_allclose((k * a).sum(axis=1), 0.0, atol=1e-15)
    assert (a * a).sum() / 4.0 == pytest.approx(1.5 * (I_U * U) ** 2, rel=1e-12)
    kap = np.linalg.norm(k, axis=1)
    assert np.all(np.diff(kap) > 0)
    assert kap[0] > 0.25 * 0.747 / LINT and kap[-1] < min(16 * 0.747 / LINT, math.pi / 4)


def test_von_karman_peak():
    r = np.linspace(0.5, 3.0, 250001)
    assert r[np.argmax(T.von_karman(r))] == pytest.approx(math.sqrt(12 / 5), abs=1e-4)


def test_sampled_field_statistics(modes):
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 4000, (200000, 3))
    u = T.fluctuation(modes, x)
    var_x_modes = 0.5 * (modes[:, 3] ** 2).sum()  # spatial mean of the x-component's square
    assert np.abs(u.mean(axis=0)).max() < 0.02 * I_U * U
    assert (u[:, 0] ** 2).mean() == pytest.approx(var_x_modes, rel=0.03)
    # isotropy: the three components share the energy within the draw's spread
    comp = 0.5 * (modes[:, 3:6] ** 2).sum(axis=0)
    assert comp.sum() == pytest.approx(3 * (I_U * U) ** 2, rel=1e-12)
    assert np.all(np.abs(comp / (I_U * U) ** 2 - 1.0) < 0.35)
    # central-difference divergence is zero up to the O(h^2) truncation
    h = 1e-3
    pts = x[:200]
    div = sum((T.fluctuation(modes, pts + h * np.eye(3)[a]) - T.fluctuation(modes, pts - h * np.eye(3)[a]))[:, a]
              for a in range(3)) / (2 * h)
    grad = np.abs(T.fluctuation(modes, pts + h * np.eye(3)[0]) - T.fluctuation(modes, pts)).max() / h
    assert np.abs(div).max() < 1e-6 * grad


@pytest.mark.parametrize("seed,n,i_u,u,lint", [(SEED, 256, I_U, U, LINT), (0, 64, 0.15, 0.08, 6.0),
                                                (2 ** 40 + 3, 128, 0.02, 0.03, 180.0)])
def test_library_mode_table_matches_oracle(seed, n, i_u, u, lint):
    """The library's mode table (host code) is the oracle's, for several seeds,
    mode counts, intensities, speeds and integral lengths (down to the
    wavenumber cap pi / 4 for short integral lengths)."""
    desc = L.domain_desc(64, 32, 32, bc=("inout", "slip", "slip"), u_in=u, nu_finest=0.02, i_u=i_u, seed=seed)
    h = L.lbm_create_domain(desc)
    L.lbm_set_geometry_prims(h, [], np.zeros((0, 8)))
    L.lbm_set_inflow_turbulence(h, n, lint)
    lib_modes = L.lbm_inflow_modes(h)
    L.lbm_destroy(h)
    np.testing.assert_allclose(lib_modes, T.rfm_modes(seed, n, i_u, u, lint), rtol=1e-12, atol=1e-15)


def test_uniform_inflow_domain_has_no_modes():
    h = L.lbm_create_domain(L.domain_desc(32, 32, 32, bc=("inout", "slip", "slip"), nu_finest=0.02))
    L.lbm_set_geometry_prims(h, [], np.zeros((0, 8)))
    assert len(L.lbm_inflow_modes(h)) == 0
    with pytest.raises(L.LbmError) as e:
        L.lbm_set_inflow_turbulence(h, 256, 10.0)
    assert e.value.code == L.LBM_ESTATE
    L.lbm_destroy(h)
    with pytest.raises(L.LbmError):
        L.lbm_create_domain(L.domain_desc(32, 32, 32, bc=("periodic",) * 3, nu_finest=0.02, i_u=0.08))


def test_oracle_turbulent_inflow_reaches_the_interior():
    """The oracle's inflow cells see the mode field: after a few steps the
    first fluid plane's velocity differs from uniform by about I_u U."""
    sim = O.Sim(32, 24, 24, bc=("inout", "slip", "slip"), nu0=0.02, u_in=U)
    sim.set_turbulence(T.rfm_modes(SEED, 64, I_U, U, 8.0), U)
    sim.step(6)
    _, u = sim.macro(0)
    dev = u[:, :, 0, :] - np.array([U, 0, 0])
    rms = np.sqrt((dev ** 2).mean())
    assert 0.1 * I_U * U < rms < 3 * I_U * U


def test_inflow_face_pulls_the_equilibrium_of_the_frozen_field(modes):
    """Taylor's hypothesis at the inflow face: at coarse step t every
    population a first-plane cell pulls across x = 0, from the outside cell
    g = (-1, y - c_y, z - c_z), is f^eq(1, U e_x + u'(g + 1/2 - U t e_x)) with
    u' the mode sum, to round-off - the outside cell's centre, not the
    pulling cell's, and the field carried by U t, not U (t + 1)."""
    C27 = np.array([[i % 3 - 1, (i // 3) % 3 - 1, i // 9 - 1] for i in range(27)])
    nx, ny, nz = 6, 7, 5
    sim = O.Sim(nx, ny, nz, bc=("inout", "periodic", "periodic"), nu0=0.02, u_in=U)
    sim.set_turbulence(modes, U)
    for t in range(3):
        sim.step(1)
        f = sim.f(0)
        checked = 0
        for i in np.flatnonzero(C27[:, 0] == 1):
            cx, cy, cz = C27[i]
            for z in range(nz):
                for y in range(ny):
                    g = np.array([-1.0, (y - cy) % ny, (z - cz) % nz]) + 0.5
                    u = np.array([U, 0.0, 0.0]) + T.fluctuation(modes, g - np.array([U * t, 0.0, 0.0]))
                    assert f[z, y, 0, i] == pytest.approx(O.equilibrium(1.0, u)[i], rel=0, abs=1e-15)
                    checked += 1
        assert checked == 9 * ny * nz
