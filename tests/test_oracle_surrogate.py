"""Pins for the branch-wise model and network oracle (no GPU): closed forms of
Eq. 2 and Eq. 4 for single cylinders, the cylinder-law value at Re = 1000,
bfloat16 rounding against torch's conversion and hand-worked ties, GELU
identities, backpropagation against central finite differences, Adam's
closed form for a constant gradient, and the library's branch feature table
against the oracle's restatement (host code)."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import surrogate as S
from paper_2603_27954_gb300 import lbm as L
from paper_2603_27954_gb300 import workloads as W


# ---------------------------------------------------------------- branch-wise model

def test_white_law_value():
    # 1000^(-2/3) = 1/100 exactly
    assert S.cylinder_cd_white(1000.0) == pytest.approx(1.1, rel=1e-14)
    assert S.cylinder_cd_white(1e6) == pytest.approx(1.001, rel=1e-14)


def test_cross_flow_cylinder_estimate_equals_cylinder_cd():
    """One branch normal to the stream: A_x = L D, so C_D-est = C_d(Re)."""
    L_, D, u, nu = 40.0, 6.0, 0.05, 0.01
    seg = np.array([[10.0, 20.0, 5.0, 10.0, 20.0, 5.0 + L_, D, 0.0]])
    F = S.branch_forces_model(seg, u, nu, S.cylinder_cd_white)
    cd = S.tree_cd_estimate(F, u, L_ * D)
    assert cd == pytest.approx(float(S.cylinder_cd_white(u * D / nu)), rel=1e-13)


@pytest.mark.parametrize("alpha_deg,factor", [(0.0, 0.0), (30.0, 0.125), (90.0, 1.0), (150.0, 0.125)])
def test_inclination_factor(alpha_deg, factor):
    a = math.radians(alpha_deg)
    d = np.array([math.cos(a), 0.0, math.sin(a)]) * 10.0
    seg = np.array([[0, 0, 0, *d, 2.0, 0.0]])
    F = S.branch_forces_model(seg, 0.1, 0.01, lambda re: np.ones_like(re))
    assert F[0] == pytest.approx(factor * 0.5 * 0.01 * 10.0 * 2.0, abs=1e-15)


def test_shadowed_fraction_and_leaf_flag():
    D = 4.0
    # tandem: the downstream branch lies fully in the upstream one's shadow
    tandem = np.array([[10, 10, 0, 10, 10, 20, D, 0], [30, 10, 0, 30, 10, 20, D, 0]], float)
    assert S.shadowed_fraction(tandem, 1) == 1.0 and S.shadowed_fraction(tandem, 0) == 0.0
    # offset sideways by 0.625 D: the lateral points at -0.4 D and -0.2 D of
    # the downstream branch (2 of 5, y = 10.9 and 11.7) lie behind the
    # upstream cylinder (|y - 10| < 2)
    half = np.array([[10, 10, 0, 10, 10, 20, D, 0], [30, 12.5, 0, 30, 12.5, 20, D, 0]], float)
    assert S.shadowed_fraction(half, 1) == pytest.approx(0.4)
    # an overlapping body whose front face is not ahead of the branch's own
    # front face (x - D/2) casts no shadow on it
    touch = np.array([[10, 10, 0, 10, 10, 20, D, 0], [9.9, 10, 0, 9.9, 10, 20, D, 0]], float)
    assert S.shadowed_fraction(touch, 1) == 0.0
    # a two-generation fork: the trunk carries children, the children are leaves
    fork = np.array([[0, 0, 0, 0, 0, 10, 2, 0], [0, 0, 10, 3, 0, 15, 1, 1], [0, 0, 10, -3, 0, 15, 1, 1]], float)
    assert [S.is_leaf(fork, k) for k in range(3)] == [False, True, True]


def test_shielding_depth_tandem_and_side_by_side():
    D = 4.0
    tandem = np.array([[10, 10, 0, 10, 10, 20, D, 0], [30, 10, 0, 30, 10, 20, D, 0]], float)
    assert S.shielding_depth(tandem, 0) == 0.0
    assert S.shielding_depth(tandem, 1) == 1.0
    side = np.array([[10, 10, 0, 10, 10, 20, D, 0], [30, 20, 0, 30, 20, 20, D, 0]], float)
    assert S.shielding_depth(side, 0) == 0.0 and S.shielding_depth(side, 1) == 0.0
    # a shorter upstream branch covers the lower half of the downstream axis
    half = np.array([[10, 10, 0, 10, 10, 10, D, 0], [30, 10, 0, 30, 10, 20, D, 0]], float)
    assert S.shielding_depth(half, 1) == 0.5


@pytest.mark.parametrize("case", ["tiny", "amr2_small", "amr2", "amr4_quarter"])
def test_library_branch_table_matches_oracle(case):
    c = W.CASES[case]
    d = L.domain_desc(*c["n0"], levels=c["levels"], block=c["block"], bc=c["bc"], u_in=c["u_in"],
                      re_h=c["re_h"])
    h = L.lbm_create_domain(d)
    L.lbm_set_geometry(h, L.tree_desc(**c["tree"]))
    seg = L.lbm_get_segments(h)
    g = L.lbm_geometry_info(h)
    tab = L.lbm_branch_table(h)
    ref = S.branch_features(seg, c["u_in"], g["nu_finest"], g["H"])
    L.lbm_destroy(h)
    assert tab.shape == ref.shape == (len(seg), L.BRANCH_COLS)
    # counts of ray hits and the leaf flag are integer data
    for col in (5, 9, 10):
        np.testing.assert_array_equal(tab[:, col], ref[:, col])
    np.testing.assert_allclose(tab, ref, rtol=1e-12, atol=1e-13)


# ---------------------------------------------------------------- network pieces

def test_bf16_round_ties_and_torch():
    one = 1.0
    e = 2.0 ** -7  # bfloat16 spacing at 1
    assert S.bf16_round(np.float32(one + e / 2))[()] == one  # tie to even (down)
    assert S.bf16_round(np.float32(one + 1.5 * e))[()] == one + 2 * e  # tie to even (up)
    assert S.bf16_round(np.float32(one + 0.75 * e))[()] == one + e
    assert S.bf16_round(np.float32(-3.0))[()] == -3.0
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(3).standard_normal(4096).astype(np.float32) * 10.0 ** np.random.default_rng(
        4).uniform(-6, 6, 4096).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(S.bf16_round(x), ref)


def test_gelu_identities():
    z = np.linspace(-6, 6, 97)
    np.testing.assert_allclose(S.gelu(z) - S.gelu(-z), z, atol=1e-15)
    assert S.gelu(np.array([0.0]))[0] == 0.0
    assert S.gelu(np.array([1.0]))[0] == pytest.approx(0.8413447460685429, rel=1e-15)  # Phi(1)
    h = 1e-6
    np.testing.assert_allclose(S.gelu_grad(z), (S.gelu(z + h) - S.gelu(z - h)) / (2 * h), atol=1e-9)


def small_net(seed=0, n_in=3, width=5, hidden=2, batch=11):
    shapes = S.layer_shapes(n_in, width, hidden)
    p = S.init_params(shapes, seed).astype(np.float64)
    rng = np.random.default_rng(seed + 100)
    x = rng.standard_normal((batch, n_in)) * [1.0, 3.0, 0.2] + [0.5, -1.0, 2.0]
    y = np.sin(x[:, 0]) + 0.3 * x[:, 1]
    return shapes, p, x, y, S.Norm.fit(x, y)


def test_backprop_matches_central_differences():
    shapes, p, x, y, norm = small_net()
    loss, g = S.loss_and_grad(p, shapes, x, y, norm, round_bf16=False)
    h = 1e-6
    fd = np.zeros_like(p)
    for k in range(len(p)):
        e = np.zeros_like(p)
        e[k] = h
        fd[k] = (S.loss_and_grad(p + e, shapes, x, y, norm, False)[0] -
                 S.loss_and_grad(p - e, shapes, x, y, norm, False)[0]) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)
    assert loss > 0


def test_bf16_forward_is_the_exact_network_at_rounded_weights():
    """Rounding is idempotent, so the bfloat16 path equals the exact path at
    pre-rounded weights (biases stay float)."""
    shapes, p, x, y, norm = small_net(seed=1)
    q = p.copy()
    o = 0
    for no, ni in shapes:
        q[o:o + no * ni] = S.bf16_round(p[o:o + no * ni].astype(np.float32))
        o += no * ni + no
    l1, g1 = S.loss_and_grad(p, shapes, x, y, norm, True)
    l2, g2 = S.loss_and_grad(q, shapes, x, y, norm, False)
    assert l1 == l2
    np.testing.assert_array_equal(g1, g2)


def test_adam_constant_gradient_closed_form():
    """With a constant gradient g the bias-corrected moments are g and g^2 at
    every step, so each step moves by lr g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    opt = S.Adam(4, lr=0.01)
    w = np.zeros(4)
    for t in range(1, 6):
        w = opt.step(w, g)
        np.testing.assert_allclose(w, -t * 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-18)


def test_training_reduces_loss():
    shapes, p, x, y, norm = small_net(seed=2, batch=64)
    opt = S.Adam(len(p), lr=1e-2)
    l0 = S.loss_and_grad(p, shapes, x, y, norm)[0]
    for _ in range(200):
        _, g = S.loss_and_grad(p, shapes, x, y, norm)
        p = opt.step(p, g)
    assert S.loss_and_grad(p, shapes, x, y, norm)[0] < 0.1 * l0


def test_oracle_branch_forces_partition_the_total_force():
    """Every cut link belongs to exactly one branch, so the per-branch mean
    forces add up to the mean total force."""
    c = W.CASES["tiny"]
    t = c["tree"]
    tree = O.make_tree(t["n"], t["children"], t["s0"], t["w0"], t["r"], t["dfac"], alpha_deg=t["alpha_deg"],
                       azimuth_mode=t["azimuth_mode"], seed=t["seed"])
    sim, info = O.tree_case(*c["n0"], tree, t["trunk_cells"], c["re_h"], u_in=c["u_in"], levels=c["levels"],
                            block=c["block"], bc=c["bc"])
    sim.step(20)
    _, tot, n = sim.force()
    fb = sim.branch_forces(len(info["segments"]))
    assert np.abs(fb).sum() > 0
    assert (np.abs(fb[:, 0]) > 0).all()  # every branch is hit by the flow
    # summation order differs: bound the difference by round-off of the largest terms
    np.testing.assert_allclose(fb.sum(axis=0), tot / n, rtol=0, atol=1e-12 * np.abs(fb).max())


@pytest.mark.parametrize("case", ["tiny", "amr2"])
def test_library_branch_estimate_matches_oracle(case):
    """Eq. 4 with the cylinder law, and with given sectional coefficients."""
    c = W.CASES[case]
    d = L.domain_desc(*c["n0"], levels=c["levels"], block=c["block"], bc=c["bc"], u_in=c["u_in"],
                      re_h=c["re_h"])
    h = L.lbm_create_domain(d)
    L.lbm_set_geometry(h, L.tree_desc(**c["tree"]))
    seg = L.lbm_get_segments(h)
    g = L.lbm_geometry_info(h)
    rows = L.lbm_branch_table(h)
    L.lbm_destroy(h)
    cd, ck = L.lbm_branch_drag_estimate(rows, g["A_x"])
    F = S.branch_forces_model(seg, c["u_in"], g["nu_finest"], S.cylinder_cd_white)
    assert cd == pytest.approx(S.tree_cd_estimate(F, c["u_in"], g["A_x"]), rel=1e-12)
    given = np.linspace(0.5, 2.0, len(seg))
    cd2, ck2 = L.lbm_branch_drag_estimate(rows, g["A_x"], given)
    np.testing.assert_array_equal(ck2, given)
    Lk, Dk, _ = S.branch_geometry(seg)
    assert cd2 == pytest.approx(np.sum(given * Lk * Dk) / g["A_x"], rel=1e-12)
    with pytest.raises(L.LbmError):
        L.lbm_branch_drag_estimate(rows, 0.0)


def test_oracle_branch_forces_vanish_at_rest():
    """Fluid at rest at the reference density: every population stays w_i,
    so each branch's gauge-form force is zero (a plain momentum exchange
    would leave each open branch surface with a net reference-pressure force)."""
    c = W.CASES["tiny"]
    t = c["tree"]
    tree = O.make_tree(t["n"], t["children"], t["s0"], t["w0"], t["r"], t["dfac"], alpha_deg=t["alpha_deg"],
                       azimuth_mode=t["azimuth_mode"], seed=t["seed"])
    sim, info = O.tree_case(*c["n0"], tree, t["trunk_cells"], c["re_h"], u_in=0.0, levels=1,
                            block=c["block"], bc=("periodic",) * 3)
    sim.init_uniform(1.0, np.zeros(3))
    sim.step(3)
    fb = sim.branch_forces(len(info["segments"]))
    assert np.abs(fb).max() < 1e-15
    _, tot, _ = sim.force()
    assert np.abs(tot).max() < 1e-13
