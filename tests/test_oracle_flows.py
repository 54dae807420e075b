"""Physics pins of the oracle's time stepping (Sec. 2.2-2.3).

Closed forms: Taylor-Green decay exp(-2 nu k^2 t), the Poiseuille parabola
(with second-order convergence of the interpolated bounce-back for several
wall fractions q), Lamb's low-Re cylinder drag.  Invariants: the
momentum-exchange balance per step, mass and momentum conservation across a
refinement interface, uniform flow left unchanged by the face conditions and
by the interface.  Exact special cases: the outflow and inflow faces cell by
cell, slip walls as mirror planes, the refined levels as an exact shift when
every rate is zero, simple bounce-back where a link has no second fluid node,
and one coarse step as 2^l one-cell updates per level.
"""
import numpy as np
import pytest

import oracle as O

C27 = np.array([[i % 3 - 1, (i // 3) % 3 - 1, i // 9 - 1] for i in range(27)])


def _tgv_field(lo, hi, scale, k, U, U0=0.0):
    z, y, x = np.meshgrid(*(np.arange(lo[a], hi[a]) + 0.5 for a in (2, 1, 0)), indexing="ij")
    x = x / scale - 0.5
    y = y / scale - 0.5
    ux = U0 + U * np.sin(k * x) * np.cos(k * y)
    uy = -U * np.cos(k * x) * np.sin(k * y)
    rho = 1 - 0.75 * U * U * (np.cos(2 * k * x) + np.cos(2 * k * y))
    return rho, np.stack([ux, uy, 0 * ux], -1), x, y


def _tgv_rate(N, nu, U, U0, steps, galilean=True):
    k = 2 * np.pi / N
    s = O.Sim(N, N, 2, bc=("periodic",) * 3, nu0=nu, u_in=0.0, galilean=galilean)
    lo, hi = s.box(0)
    rho, u, x, y = _tgv_field(lo, hi, 1, k, U, U0)
    s.init_field(0, rho, u)

    def amp(t):
        _, uu = s.macro(0)
        a = np.sin(k * (x - U0 * t)) * np.cos(k * y)
        b = np.cos(k * (x - U0 * t)) * np.cos(k * y)
        return np.hypot(((uu[..., 0] - U0) * a).sum() / (a * a).sum(), ((uu[..., 0] - U0) * b).sum() / (b * b).sum())

    t0 = steps // 4
    s.step(t0)
    a0 = amp(t0)
    s.step(steps)
    a1 = amp(t0 + steps)
    return -np.log(a1 / a0) / steps / (2 * nu * k * k) - 1


@pytest.mark.parametrize("N,nu", [(32, 0.01), (32, 0.002), (64, 0.02)])
def test_taylor_green_decay_rate(N, nu):
    """Amplitude decays as exp(-2 nu k^2 t), nu = (1/omega1 - 1/2)/3."""
    assert abs(_tgv_rate(N, nu, 0.02, 0.0, 400 * N // 32)) < 0.01


def test_galilean_correction_restores_decay_rate_under_mean_flow():
    """With a mean flow U0 = 0.15 the D3Q27 lattice's missing u^3 moment biases
    the viscosity; the correction of the diagonal cumulants removes it."""
    with_corr = _tgv_rate(32, 0.01, 0.01, 0.15, 400, True)
    without = _tgv_rate(32, 0.01, 0.01, 0.15, 400, False)
    assert abs(with_corr) < 0.01
    assert abs(without) > 0.03


def _poiseuille_error(N, o, nu=1.0 / 6.0, g=1e-5):
    ny = N + 4
    ya, yb = 2.0 + o, ny - 2.0 - o
    s = O.Sim(1, ny, 1, bc=("periodic",) * 3, nu0=nu, u_in=0.0, force=(g, 0, 0))
    s.set_prims(O.prims([(1, (0, 1, 0, ya)), (1, (0, -1, 0, -yb))]))
    s.step(int(6 * (yb - ya) ** 2 / nu))
    _, u = s.macro(0)
    y = np.arange(ny) + 0.5
    ux = u[0, :, 0, 0]
    fl = ~np.isnan(ux)
    exact = g / (2 * nu) * (y - ya) * (yb - y)
    return np.sqrt(((ux[fl] - exact[fl]) ** 2).sum() / (exact[fl] ** 2).sum())


@pytest.mark.parametrize("o,q", [(0.0, 0.5), (0.3, 0.2), (-0.2, 0.7)])
def test_poiseuille_second_order_bounce_back(o, q):
    """Body-force channel between walls a fraction q beyond the last fluid
    node: the parabola g (y-ya)(yb-y) / (2 nu), error falling as N^-2."""
    e = [_poiseuille_error(N, o) for N in (8, 16, 32)]
    assert e[2] < 4e-3
    for a, b in zip(e, e[1:]):
        assert 3.3 < a / b < 4.8


def test_momentum_exchange_balances_fluid_momentum_every_step():
    """Periodic box, body force g on every fluid cell, a solid block: per step
    the fluid momentum changes by N_f g - F_ME exactly."""
    N, g = 16, 2e-6
    s = O.Sim(N, N, N, bc=("periodic",) * 3, nu0=0.05, u_in=0.0, force=(g, 0, 0))
    s.set_prims(O.prims([(2, (6, 6.3, 5.7, 10, 9.6, 10.2))]))
    nf = int((s.cell_type(0) == 0).sum())
    cell, d, q = s.links(0)
    assert (q < 0.5).any() and (q >= 0.5).any()  # both Bouzidi branches

    def P():
        return np.nansum(s.f(0) @ C27, axis=(0, 1, 2))

    p0 = P()
    for _ in range(10):
        s.step(1)
        p1 = P()
        F, _, _ = s.force()
        np.testing.assert_allclose(p1 - p0, nf * np.array([g, 0, 0]) - F, atol=1e-12)
        p0 = p1


def _refined_box_sim(N=32, levels=2, nu=0.01):
    boxes = [None, [16, 16, 16, 48, 48, 48]]
    return O.Sim(N, N, N, levels=levels, boxes=boxes, bc=("periodic",) * 3, nu0=nu, u_in=0.0)


def test_refinement_conserves_mass_and_momentum():
    """Closed periodic box with a refined patch; a non-uniform flow crosses
    the interface.  Volume-weighted mass and momentum stay constant."""
    s = _refined_box_sim()
    for l in range(2):
        lo, hi = s.box(l)
        z, y, x = np.meshgrid(*(np.arange(lo[a], hi[a]) / 2.0 ** l for a in (2, 1, 0)), indexing="ij")
        u = np.stack([0.03 * np.sin(2 * np.pi * y / 32), 0.02 * np.cos(2 * np.pi * x / 32),
                      0.01 * np.sin(2 * np.pi * (x + y) / 32)], -1)
        rho = 1 + 0.01 * np.cos(2 * np.pi * z / 32)
        s.init_field(l, rho, u)
    m0, p0 = s.mass()
    s.step(30)
    m1, p1 = s.mass()
    assert abs(m1 - m0) / m0 < 1e-12
    np.testing.assert_allclose(p1, p0, atol=1e-12 * m0)
    for l in range(2):
        f = s.f(l)
        assert not np.isnan(f[s.cell_type(l) == 0]).any()


def test_uniform_flow_crosses_refinement_unchanged():
    s = _refined_box_sim()
    u = [0.05, 0.02, -0.01]
    s.init_uniform(1.0, u)
    s.step(8)
    feq = O.equilibrium(1.0, u)
    for l in range(2):
        f = s.f(l)
        ok = s.cell_type(l) == 0
        np.testing.assert_allclose(f[ok], np.broadcast_to(feq, f[ok].shape), atol=2e-15)


def test_face_conditions_keep_uniform_inflow_uniform():
    """Inflow equilibrium at x = 0, zero-gradient outflow, slip or inflow
    lateral faces: the uniform state U x is a steady solution."""
    for lateral in ("slip", "inflow"):
        s = O.Sim(16, 12, 10, bc=("inout", lateral, lateral), nu0=0.02, u_in=0.05)
        s.step(20)
        feq = O.equilibrium(1.0, [0.05, 0, 0])
        f = s.f(0)
        np.testing.assert_allclose(f, np.broadcast_to(feq, f.shape), atol=2e-15)


def test_slip_walls_conserve_mass():
    """Periodic in x, specular slip in y and z: a closed system."""
    s = O.Sim(8, 10, 12, bc=("periodic", "slip", "slip"), nu0=0.02, u_in=0.0)
    lo, hi = s.box(0)
    rho, u, _, _ = _tgv_field(lo, hi, 1, 2 * np.pi / 8, 0.03)
    u[..., 2] = 0.02
    s.init_field(0, rho, u)
    m0, p0 = s.mass()
    s.step(40)
    m1, p1 = s.mass()
    assert abs(m1 - m0) / m0 < 1e-13
    assert p1[0] == pytest.approx(p0[0], abs=1e-11)


def test_taylor_green_across_refined_patch():
    """Kinetic energy decays as exp(-4 nu k^2 t) with a refined patch in the
    middle of the box; the interface (no non-equilibrium rescaling) adds an
    error of a few per cent at this resolution, the uniform grid none, and
    the two-level error shrinks as the resolution grows (the same flow at
    half the resolution, acoustic scaling: nu and the step counts halve)."""
    def rate(levels, N=32):
        nu, U = 0.01 * N / 32, 0.01
        k = 2 * np.pi / N
        f = N // 16
        boxes = [None, [10 * f, 10 * f, 4 * f, 22 * f, 22 * f, 12 * f]] if levels == 2 else None
        s = O.Sim(N, N, N // 2, levels=levels, boxes=boxes, bc=("periodic",) * 3, nu0=nu, u_in=0.0)
        for l in range(levels):
            lo, hi = s.box(l)
            rho, u, _, _ = _tgv_field(lo, hi, 2 ** l, k, U)
            s.init_field(l, rho, u)

        def E():
            tot = 0.0
            for l in range(levels):
                r, u = s.macro(l)
                tot += 8.0 ** -l * np.nansum(r * (u ** 2).sum(-1))
            return tot

        s.step(100 * N // 32)
        e0 = E()
        n = 400 * N // 32
        s.step(n)
        return -np.log(E() / e0) / n / (4 * nu * k * k) - 1

    assert abs(rate(1)) < 0.002
    fine, coarse = rate(2), rate(2, N=16)
    assert abs(fine) < 0.05
    # measured: 0.069 at N = 16, 0.023 at N = 32
    assert abs(fine) < 0.5 * abs(coarse), (fine, coarse)


def _post_collision(s, nu):
    """Post-collision populations of every cell of a single-level Sim, by the
    separately pinned one-cell collision (orc_collide), in (z, y, x, i) order."""
    f = s.f(0)
    r = O.rates(1.0 / (3.0 * nu + 0.5))
    out = np.empty_like(f)
    for z in range(f.shape[0]):
        for y in range(f.shape[1]):
            for x in range(f.shape[2]):
                out[z, y, x] = O.collide(f[z, y, x], r)
    return out


def test_outflow_takes_the_last_plane_cell_by_cell():
    """Zero-gradient outflow (Sec. 2.3): a population that a cell of the last
    plane x = n - 1 pulls from beyond the outlet, x - c_i = (n, y - c_y, z - c_z),
    is the post-collision value of the same direction at (n - 1, y - c_y, z - c_z):
    the post-collision field continued with zero x-gradient.  A non-uniform
    field in y and z makes a copy from another plane, another row or another
    direction fail; the inflow face pulls the inflow equilibrium exactly."""
    nx, ny, nz, nu, U = 6, 5, 4, 0.02, 0.05
    s = O.Sim(nx, ny, nz, bc=("inout", "periodic", "periodic"), nu0=nu, u_in=U)
    rng = np.random.default_rng(11)
    rho = 1.0 + 0.01 * rng.standard_normal((nz, ny, nx))
    u = 0.03 * rng.standard_normal((nz, ny, nx, 3))
    s.init_field(0, rho, u)
    A = _post_collision(s, nu)
    s.step(1)
    B = s.f(0)
    feq_in = O.equilibrium(1.0, [U, 0.0, 0.0])
    checked = 0
    for i in range(27):
        cx, cy, cz = C27[i]
        for z in range(nz):
            for y in range(ny):
                sy, sz = (y - cy) % ny, (z - cz) % nz
                if cx == -1:  # pulled across the outlet
                    assert B[z, y, nx - 1, i] == A[sz, sy, nx - 1, i]
                    # a copy from plane n - 2, from the unshifted row or from the opposite direction differs
                    assert B[z, y, nx - 1, i] != A[sz, sy, nx - 2, i]
                    checked += 1
                if cx == 1:  # pulled across the inflow face
                    assert B[z, y, 0, i] == feq_in[i]
    assert checked == 9 * ny * nz
    # the rows: for some population the unshifted row must give a different value
    assert any(B[z, y, nx - 1, i] != A[z, y, nx - 1, i] for i in range(27) if C27[i][0] == -1 and (C27[i][1] or C27[i][2])
               for z in range(nz) for y in range(ny))


def test_outflow_keeps_a_sheared_stream_x_invariant():
    """A stream sheared in y and z and uniform in x, convected out through the
    zero-gradient outlet: until the disturbance of the uniform inflow face
    (one cell per step) arrives, every plane from x = k to the outlet stays
    identical to the others bit for bit - the outlet plane pulls exactly what
    an interior plane would (a wrong row, direction or sign breaks it)."""
    nx, ny, nz, nu = 24, 8, 6, 0.02
    s = O.Sim(nx, ny, nz, bc=("inout", "periodic", "periodic"), nu0=nu, u_in=0.05)
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    u = np.stack([0.05 + 0.02 * np.sin(2 * np.pi * y / ny), 0.01 * np.cos(2 * np.pi * z / nz),
                  0.015 * np.sin(2 * np.pi * (y / ny + z / nz))], -1)
    s.init_field(0, 1.0 + 0.002 * np.cos(2 * np.pi * y / ny), u)
    for k in range(1, 12):
        s.step(1)
        f = s.f(0)
        for xx in range(k, nx):
            np.testing.assert_array_equal(f[:, :, xx], f[:, :, nx - 1], err_msg="plane %d after %d steps" % (xx, k))
        assert not np.array_equal(f[:, :, 0], f[:, :, nx - 1])  # the inflow face does disturb


def _lamb_cd(re):
    """Lamb's Oseen drag per unit length of a circular cylinder at small Re:
    C_D = 8 pi / (Re (1/2 - gamma + ln(8 / Re)))."""
    return 8.0 * np.pi / (re * (0.5 - 0.5772156649015329 + np.log(8.0 / re)))


@pytest.mark.slow
def test_low_re_cylinder_momentum_exchange_near_lamb():
    """The oracle's momentum-exchange force (Sec. 2.2, Wen et al. 2014) on a
    spanwise-periodic cylinder of diameter D = 6 cells at Re = U D / nu = 1,
    uniform inflow, slip walls 12 D either side, a stream-wise box of 36 D:
    the steady drag per unit length within 10 % of Lamb's Oseen value (the
    bound of the same check on the CUDA path; finite Re, confinement and the
    coarse cylinder move a converged lattice result by a few per cent:
    measured -1.8 % here).  The drag has settled (under 1 % change over the
    last 400 steps) and the symmetric flow carries no lift."""
    D, U, re = 6.0, 0.05, 1.0
    nx, ny = int(36 * D), int(24 * D)
    s = O.Sim(nx, ny, 1, bc=("inout", "slip", "periodic"), nu0=U * D / re, u_in=U)
    xc, yc = nx / 3.0, ny / 2.0
    s.set_prims(O.prims([(0, (xc, yc, -2.0, xc, yc, 3.0, D, 0.0))]))
    s.step(1200)
    f0, _, _ = s.force()
    s.step(400)
    f1, _, _ = s.force()
    cd0, cd1 = (f[0] / (0.5 * U * U * D * 1.0) for f in (f0, f1))
    assert abs(cd1 - cd0) < 0.01 * abs(cd1)
    assert abs(f1[1]) < 1e-3 * abs(f1[0])
    assert abs(cd1 - _lamb_cd(re)) <= 0.10 * _lamb_cd(re), (cd1, _lamb_cd(re))


@pytest.mark.parametrize("axis", [1, 2])
def test_slip_walls_equal_the_mirrored_periodic_domain(axis):
    """Specular (free-slip) walls halfway between cells (the lateral faces of
    Sec. 2.3's box in the slip reading) are mirror planes: a box with slip
    walls normal to `axis` evolves exactly as the first half of a periodic box
    of twice the width whose second half is the mirror image of the first
    (position reflected, the normal velocity reversed).  A non-uniform random
    field makes a reflection of the wrong component, an unreflected copy or a
    wall placed on a cell centre fail."""
    n = (6, 5, 4)
    dbl = list(n)
    dbl[axis] *= 2
    bc_slip = ["periodic"] * 3
    bc_slip[axis] = "slip"
    a = O.Sim(*n, bc=tuple(bc_slip), nu0=0.03, u_in=0.0)
    b = O.Sim(*dbl, bc=("periodic",) * 3, nu0=0.03, u_in=0.0)
    rng = np.random.default_rng(5 + axis)
    shape = (n[2], n[1], n[0])
    rho = 1.0 + 0.01 * rng.standard_normal(shape)
    u = 0.04 * rng.standard_normal(shape + (3,))
    ax_np = 2 - axis  # numpy axis of the lattice axis (arrays are z, y, x)
    rho_m = np.flip(rho, ax_np)
    u_m = np.flip(u, ax_np).copy()
    u_m[..., axis] *= -1
    a.init_field(0, rho, u)
    b.init_field(0, np.concatenate([rho, rho_m], ax_np), np.concatenate([u, u_m], ax_np))
    for _ in range(4):
        a.step(3)
        b.step(3)
        fa = a.f(0)
        fb = np.take(b.f(0), np.arange(n[axis]), axis=ax_np)
        np.testing.assert_allclose(fa, fb, rtol=0, atol=1e-14)
    # the field is not trivial: the walls' neighbourhood carries a normal flow
    _, ua = a.macro(0)
    assert np.abs(np.take(ua, [0], axis=ax_np)[..., axis]).max() > 1e-3


@pytest.mark.parametrize("levels", [2, 3])
def test_refinement_with_zero_rates_is_an_exact_coarse_shift(levels):
    """With every relaxation rate zero the collision is the identity and the
    lattice only streams.  A composite field that is constant over each coarse
    cell (the finer levels hold their coarse parent's populations) is then
    carried by exactly one coarse cell along c_i per coarse step on every
    level: the finer levels stream 2^l times per coarse step (recursive
    sub-cycling), the explode hands a coarse cell's populations to its
    virtual children and the coalesce averages the 8 children that arrived
    (volumetric transfer, Sec. 2.2's octree refinement).  A wrong child
    index, parent index, averaging weight or sub-step count shows up as a
    population from the wrong coarse cell."""
    N = 8
    boxes = [None, [4, 4, 4, 12, 12, 12], [12, 12, 12, 20, 20, 20]][:levels]
    s = O.Sim(N, N, N, levels=levels, boxes=boxes, bc=("periodic",) * 3, nu0=1e30, omega2=0.0,
              omega_hi=(0.0,) * 8, galilean=False, u_in=0.0)
    rng = np.random.default_rng(21 + levels)
    rho0 = 1.0 + 0.02 * rng.standard_normal((N, N, N))
    u0 = 0.05 * rng.standard_normal((N, N, N, 3))

    def parent_slice(l, arr):
        lo, hi = s.box(l)
        idx = [np.arange(lo[a], hi[a]) >> l for a in (2, 1, 0)]
        return arr[np.ix_(*idx)]

    for l in range(levels):
        s.init_field(l, parent_slice(l, rho0), parent_slice(l, u0))
    F0 = np.stack([O.equilibrium(r, v) for r, v in zip(rho0.ravel(), u0.reshape(-1, 3))]).reshape(N, N, N, 27)
    done = 0
    for k in (1, 2, 5):
        s.step(k - done)
        done = k
        want = np.empty_like(F0)
        for i in range(27):
            cx_, cy_, cz_ = C27[i]
            want[..., i] = np.roll(F0[..., i], (k * cz_, k * cy_, k * cx_), axis=(0, 1, 2))
        for l in range(levels):
            ok = s.cell_type(l) == 0
            got = s.f(l)[ok]
            np.testing.assert_allclose(got, parent_slice(l, want)[ok], rtol=0, atol=1e-14)


def test_links_without_a_second_fluid_node_bounce_back_simply():
    """A fluid layer one cell thick between two plates: every cut link's
    second node x_f - c_i is solid, so the interpolated bounce-back has no
    second value and the link bounces back simply, f_ibar = f*_i(x_f),
    whatever its wall fraction q.  Two plate placements with different q on
    both walls give the same populations bit for bit, and mass is conserved
    exactly (a q-dependent formula would break both)."""
    runs = []
    for qa, qb in ((0.3, 0.8), (0.45, 0.15)):
        s = O.Sim(6, 4, 5, bc=("periodic",) * 3, nu0=0.04, u_in=0.0, force=(3e-5, 0.0, 1e-5))
        # cells y = 1 (centre 1.5) are fluid; the plates' surfaces sit qa below and qb above it
        s.set_prims(O.prims([(2, (-1, -1, -1, 7, 1.5 - qa, 6)), (2, (-1, 1.5 + qb, -1, 7, 5, 6))]))
        t = s.cell_type(0)
        assert (t[:, 1, :] == 0).all() and (t[:, [0, 2, 3], :] == 1).all()
        cell, d, q = s.links(0)
        cy = C27[d][:, 1]
        # a link's direction points from the fluid cell into the wall
        np.testing.assert_allclose(q[cy == -1], qa, rtol=1e-12)
        np.testing.assert_allclose(q[cy == 1], qb, rtol=1e-12)
        assert len(q) == 18 * 6 * 5
        rng = np.random.default_rng(3)
        rho = 1.0 + 0.01 * rng.standard_normal((5, 4, 6))
        u = 0.02 * rng.standard_normal((5, 4, 6, 3))
        s.init_field(0, rho, u)
        m0, _ = s.mass()
        s.step(25)
        m1, _ = s.mass()
        assert abs(m1 - m0) / m0 < 1e-14
        runs.append(s.f(0)[:, 1, :])
    np.testing.assert_array_equal(runs[0], runs[1])


def _oracle_tree(t):
    return O.make_tree(t["n"], t["children"], t["s0"], t["w0"], t["r"], t["dfac"], alpha_deg=t["alpha_deg"],
                       azimuth_mode=t["azimuth_mode"], seed=t["seed"])


def test_sampled_one_cell_recursion_reproduces_the_oracle_step():
    """The sampled check used on runs too large for the oracle (each level-l
    interior cell advanced by 2^l one-cell collide-stream updates per coarse
    step) reproduces the oracle's own two-level step on the quarter-scale
    tree case from a non-uniform state, to round-off: the recursion, its
    direction convention and its interior criterion are those of the
    stepping itself."""
    from sampled_cells import check_level
    from paper_2603_27954_gb300 import workloads as W
    c = W.CASES["amr2_quarter"]
    sim, info = O.tree_case(*c["n0"], _oracle_tree(c["tree"]), c["tree"]["trunk_cells"], c["re_h"],
                            u_in=c["u_in"], levels=c["levels"], block=c["block"], bc=c["bc"])
    for l in range(2):
        lo, hi = sim.box(l)
        rho, u = W.tgv_fields(lo, hi, 2 ** l, 16, 0.02, (c["u_in"], 0.0, 0.01))
        sim.init_field(l, rho, u)
    sim.step(2)
    S0 = [sim.f(l) for l in range(2)]
    sim.step(1)
    for l in range(2):
        n, err, moved = check_level(S0[l], sim.f(l), sim.cell_type(l), l, info["nu0"] * 2 ** l, 40, l, 1e-13)
        assert n == 40 and moved > 1e-4


def test_lateral_inflow_faces_pull_the_inflow_equilibrium_and_interior_streams():
    """Sec. 2.3's inflow on the faces other than the outlet: from a random
    non-uniform state, after one step every population a cell pulls from
    outside y or z (x - c_i beyond a lateral face) is the inflow equilibrium
    f^eq(1, U e_x) exactly, whatever the interior holds, and every population
    pulled from inside is the post-collision value at x - c_i (plain
    streaming, one-cell collision pinned separately)."""
    nx, ny, nz, nu, U = 4, 5, 6, 0.03, 0.05
    s = O.Sim(nx, ny, nz, bc=("periodic", "inflow", "inflow"), nu0=nu, u_in=U)
    rng = np.random.default_rng(17)
    s.init_field(0, 1.0 + 0.01 * rng.standard_normal((nz, ny, nx)), 0.03 * rng.standard_normal((nz, ny, nx, 3)))
    A = _post_collision(s, nu)
    s.step(1)
    B = s.f(0)
    feq_in = O.equilibrium(1.0, [U, 0.0, 0.0])
    outside = 0
    for i in range(27):
        cx, cy, cz = C27[i]
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    sy, sz, sx = y - cy, z - cz, (x - cx) % nx
                    if 0 <= sy < ny and 0 <= sz < nz:
                        assert B[z, y, x, i] == A[sz, sy, sx, i]
                    else:
                        assert B[z, y, x, i] == feq_in[i]
                        outside += 1
    assert outside > 0
