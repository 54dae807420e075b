"""Pins of the oracle's tree and geometry (Sec. 2.1 Eq. 1, Tables 1-2; Sec. 2.3).

Each test checks the oracle against something other than itself: values the
paper prints, closed-form areas (single, tilted and crossing cylinders) and
ray intersections, a published test vector, or a brute-force entry search
along each cut link's ray (the branch it belongs to and its wall fraction).
"""
import ctypes as C
import math
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLD, name)) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


def _basic_tree(n):
    row = [r for r in _rows("table1_basic.txt") if int(r[-1]) == n][0]
    r1, r2, a1, a2, p1, p2, s0, w0, q, e, mn = map(float, row[1:12])
    return O.make_tree(n, 2, s0, w0, (r1, r2), None, q, e, (a1, a2), (p1, p2), 0, 0, mn)


@pytest.mark.parametrize("row", _rows("table2_geometry.txt"), ids=lambda r: "n=" + r[0])
def test_table2_d0_l0_over_height(row):
    """Table 2: D0/H and L0/H to all printed digits (H = vertical extent of the
    cylinders, envelope included; n rewritings draw generations 0..n-1)."""
    n, d0h, l0h = int(row[0]), float(row[1]), float(row[2])
    t = _basic_tree(n)
    seg = O.lsystem(t)
    H = O.tree_height(seg)
    assert round(t.w0 / H, 3) == pytest.approx(d0h, abs=1e-12)
    assert round(t.s0 / H, 3) == pytest.approx(l0h, abs=1e-12)


@pytest.mark.parametrize("n", [4, 6, 8])
def test_branch_scaling_laws(n):
    """Sec. 2.1: L_k = 0.8 L_{k-1} and D_k = 0.5^0.5 D_{k-1}; 2^n - 1 segments."""
    seg = O.lsystem(_basic_tree(n))
    assert len(seg) == 2 ** n - 1
    for g in range(n):
        rows = seg[seg[:, 7] == g]
        assert len(rows) == 2 ** g
        L = np.linalg.norm(rows[:, 3:6] - rows[:, 0:3], axis=1)
        np.testing.assert_allclose(L, 100.0 * 0.8 ** g, rtol=1e-12)
        np.testing.assert_allclose(rows[:, 6], 30.0 * 0.5 ** (0.5 * g), rtol=1e-12)


def test_children_attach_at_parent_tip_with_branching_angle():
    """Children start at the end of their parent and make angle |alpha| with it."""
    seg = O.lsystem(_basic_tree(4))
    ends = {tuple(np.round(r[3:6], 9)) for r in seg}
    for r in seg[1:]:
        assert tuple(np.round(r[0:3], 9)) in ends
    # the trunk is vertical, its two children tilt by 30 degrees
    trunk = seg[0]
    assert np.allclose(trunk[3:6] - trunk[0:3], [0, 0, 100])
    for r in seg[seg[:, 7] == 1]:
        d = (r[3:6] - r[0:3]) / np.linalg.norm(r[3:6] - r[0:3])
        assert math.degrees(math.acos(d[2])) == pytest.approx(30.0, abs=1e-9)


def test_seeded_azimuths_spread_children_around_the_parent():
    """Azimuth form: three children at the same tilt, distinct azimuths drawn
    from the seed; same seed gives the same tree, another seed another one."""
    t = O.make_tree(2, 3, 64, 19.2, (0.6,), (0.6,), alpha_deg=(35.0,), azimuth_mode=1, seed=2)
    a = O.lsystem(t)
    assert len(a) == 4
    kids = a[1:]
    dirs = (kids[:, 3:6] - kids[:, 0:3]) / np.linalg.norm(kids[:, 3:6] - kids[:, 0:3], axis=1)[:, None]
    np.testing.assert_allclose(np.degrees(np.arccos(dirs[:, 2])), 35.0, atol=1e-9)
    az = np.degrees(np.arctan2(dirs[:, 1], dirs[:, 0]))
    assert len(set(np.round(az, 6))) == 3
    np.testing.assert_array_equal(O.lsystem(t), a)
    t.seed = 3
    assert not np.allclose(O.lsystem(t), a)


def test_splitmix64_published_vector():
    L = O.lib()
    L.orc_splitmix64.restype = C.c_uint64
    L.orc_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
    want = [int(r[0]) for r in _rows("splitmix64_seed1234567.txt")]
    assert [L.orc_splitmix64(1234567, k) for k in range(5)] == want


def test_frontal_area_of_a_cross_flow_cylinder_is_l_times_d():
    """A vertical cylinder seen along x projects to an L x D rectangle."""
    seg = np.array([[10.0, 16.0, 4.0, 10.0, 16.0, 16.0, 2.0, 0.0]])
    assert O.frontal_area(seg, 0.125) == pytest.approx(12.0 * 2.0, abs=1e-12)


@pytest.mark.parametrize("theta_deg", [20.0, 45.0, 70.0])
def test_frontal_area_of_a_tilted_cylinder(theta_deg):
    """Projection of a flat-capped cylinder whose axis makes angle theta with x:
    L D sin(theta) + (pi/4) D^2 |cos(theta)| (rectangle plus two half ellipses)."""
    th = math.radians(theta_deg)
    L, D = 20.0, 4.0
    p0 = np.array([30.0, 30.0, 30.0])
    p1 = p0 + L * np.array([math.cos(th), 0.0, math.sin(th)])
    seg = np.array([list(p0) + list(p1) + [D, 0.0]])
    exact = L * D * math.sin(th) + math.pi / 4 * D * D * abs(math.cos(th))
    assert O.frontal_area(seg, 1.0 / 64) == pytest.approx(exact, rel=3e-3)


def test_link_fraction_against_circle_intersection():
    """q along +x from a fluid point to a vertical cylinder: the chord formula."""
    c = (20.0, 20.0)
    r = 3.0
    pr = O.cylinders_as_prims(np.array([[c[0], c[1], 0.0, c[0], c[1], 40.0, 2 * r, 0]]))
    for y0 in (18.5, 20.0, 21.7):
        xs = c[0] - math.sqrt(r * r - (y0 - c[1]) ** 2)
        x0 = xs - 0.37
        q = O.prim_ray(pr, [x0, y0, 10.0], [1.0, 0.0, 0.0])
        assert q == pytest.approx(0.37, abs=1e-12)
        assert not O.prim_inside(pr, [x0, y0, 10.0])
        assert O.prim_inside(pr, [x0 + 1.0, y0, 10.0])
    # a diagonal ray to a half-space: t = (d - n.x) / (n.dir)
    hs = O.prims([(1, (0.0, 1.0, 0.0, 4.3))])
    assert O.prim_ray(hs, [1.0, 5.0, 1.0], [1.0, -1.0, 1.0]) == pytest.approx(0.7, abs=1e-12)
    # entering a cap: axis along z, ray along -z from above the top disc
    assert O.prim_ray(pr, [20.5, 20.5, 40.25], [0.0, 0.0, -1.0]) == pytest.approx(0.25, abs=1e-12)


def test_centre_of_mass_and_placement():
    """Two equal cylinders mirrored about a point have their COM there; the
    placed tree has its COM at (Lx/4, Ly/2, Lz/2) and a trunk of the asked length."""
    seg = np.array([[0, 0, 0, 0, 0, 10, 2, 0], [4, 0, 0, 4, 0, 10, 2, 0]], float)
    np.testing.assert_allclose(O.tree_com(seg), [2, 0, 5], atol=1e-12)
    t = O.make_tree(2, 2, 12.0, 2.0, (0.6, 0.6), (0.7, 0.7), alpha_deg=(30.0, 30.0),
                    azimuth_mode=1, seed=0)
    s = O.place_tree(t, 12.0, (64, 32, 32))
    np.testing.assert_allclose(O.tree_com(s), [16, 16, 16], atol=1e-12)
    assert np.linalg.norm(s[0, 3:6] - s[0, 0:3]) == pytest.approx(12.0)
    assert s[0, 6] == pytest.approx(2.0)


DIRS = np.array([[i % 3 - 1, (i // 3) % 3 - 1, i // 9 - 1] for i in range(27)])


def _inside_cylinders(seg, pts):
    """Membership of points (m x 3) in each flat-capped cylinder (n x m):
    0 <= (x - p0) . a <= |p1 - p0| and distance from the axis <= D / 2."""
    p0, p1, rad = seg[:, None, 0:3], seg[:, None, 3:6], 0.5 * seg[:, None, 6]
    ax = p1 - p0
    ln = np.linalg.norm(ax, axis=2, keepdims=True)
    a = ax / ln
    w = pts[None, :, :] - p0
    wa = (w * a).sum(axis=2, keepdims=True)
    perp = np.linalg.norm(w - wa * a, axis=2)
    return (wa[..., 0] >= 0) & (wa[..., 0] <= ln[..., 0]) & (perp <= rad)


def _first_entries(seg, x, d, samples=20000):
    """Per cylinder, the first t in [0, 1] with x + t d inside it (inf if
    none), by dense sampling of the inside test and bisection on the first
    bracket - brute force, independent of any ray-quadric formula."""
    out = np.full(len(seg), np.inf)
    # a cylinder farther from x than its radius plus |d| cannot be reached (triangle inequality)
    p0, p1 = seg[:, 0:3], seg[:, 3:6]
    s = np.clip(((x - p0) * (p1 - p0)).sum(axis=1) / ((p1 - p0) ** 2).sum(axis=1), 0.0, 1.0)
    dist = np.linalg.norm(x - (p0 + s[:, None] * (p1 - p0)), axis=1)
    near = np.flatnonzero(dist <= 0.5 * seg[:, 6] + np.linalg.norm(d) + 1e-9)
    t = np.linspace(0.0, 1.0, samples + 1)
    inside = np.zeros((len(seg), len(t)), bool)
    inside[near] = _inside_cylinders(seg[near], x[None, :] + t[:, None] * d[None, :])
    for k in np.flatnonzero(inside.any(axis=1)):
        j = int(np.argmax(inside[k]))
        if j == 0:
            out[k] = 0.0
            continue
        lo, hi = t[j - 1], t[j]
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if _inside_cylinders(seg[k:k + 1], (x + mid * d)[None, :])[0, 0]:
                hi = mid
            else:
                lo = mid
        out[k] = hi
    return out


@pytest.mark.parametrize("case", ["tiny", "amr2_quarter"])
def test_cut_links_belong_to_the_branch_their_ray_enters_first(case):
    """Per-branch forces (Sec. 2.4's branch-by-branch view) rest on the link
    attribution: a cut link belongs to the cylinder its ray x_f + t c_i enters
    first (ties at the junctions: either tied branch), and its wall fraction
    q is that entry point.  Checked on a seeded sample of the finest level's
    links against a brute-force entry search over every branch."""
    from paper_2603_27954_gb300 import workloads as W
    c = W.CASES[case]
    t = c["tree"]
    tree = O.make_tree(t["n"], t["children"], t["s0"], t["w0"], t["r"], t["dfac"], alpha_deg=t["alpha_deg"],
                       azimuth_mode=t["azimuth_mode"], seed=t["seed"])
    sim, info = O.tree_case(*c["n0"], tree, t["trunk_cells"], c["re_h"], u_in=c["u_in"], levels=c["levels"],
                            block=c["block"], bc=c["bc"])
    fin = c["levels"] - 1
    cell, d, q = sim.links(fin)
    segs = sim.link_segments(fin)
    seg = np.asarray(info["segments"], dtype=np.float64)
    lo, hi = sim.box(fin)
    nx, ny = hi[0] - lo[0], hi[1] - lo[1]
    assert len(seg) > 2 and len(np.unique(segs)) == len(seg)  # every branch carries links
    rng = np.random.default_rng(0)
    pick = rng.choice(len(cell), size=min(400, len(cell)), replace=False)
    for k in pick:
        z, rem = divmod(int(cell[k]), nx * ny)
        y, x = divmod(rem, nx)
        xf = np.array([x + lo[0] + 0.5, y + lo[1] + 0.5, z + lo[2] + 0.5])
        ent = _first_entries(seg, xf, DIRS[d[k]].astype(np.float64))
        tmin = ent.min()
        assert np.isfinite(tmin)
        tied = np.flatnonzero(ent <= tmin + 1e-9)
        assert segs[k] in tied, (k, segs[k], ent)
        assert q[k] == pytest.approx(max(tmin, 1e-6), abs=1e-9)


@pytest.mark.parametrize("theta_deg", [90.0, 60.0, 35.0])
def test_frontal_area_counts_overlapping_branches_once(theta_deg):
    """A_x is the area of the union of the projected cylinders (Eq. 7's
    frontal area; overlaps counted once): two long cross-flow cylinders in
    the y-z plane crossing at angle theta project to two strips of width D
    whose overlap is a rhombus of area D^2 / sin(theta), so
    A_x = 2 L D - D^2 / sin(theta) (the flat caps project to nothing)."""
    th = math.radians(theta_deg)
    L, D = 40.0, 3.0
    c = np.array([20.0, 50.0, 50.0])
    a1 = np.array([0.0, 0.0, 1.0])
    a2 = np.array([0.0, math.sin(th), math.cos(th)])
    seg = np.array([list(c - 0.5 * L * a1) + list(c + 0.5 * L * a1) + [D, 0.0],
                    list(c - 0.5 * L * a2) + list(c + 0.5 * L * a2) + [D, 1.0]])
    exact = 2 * L * D - D * D / math.sin(th)
    assert O.frontal_area(seg, 1.0 / 32) == pytest.approx(exact, rel=2e-3)
    # each alone is L x D; the union is less than their sum by the rhombus
    assert O.frontal_area(seg[:1], 1.0 / 32) == pytest.approx(L * D, rel=1e-3)


def test_refinement_boxes_of_a_hand_worked_case():
    """Reading 12's box rule worked by hand for one vertical cylinder, finest
    cells from (128, 128, 100) to (128, 128, 160), D = 8, three levels,
    coarse 64^3 in 8^3 blocks:
    bounding box x, y [124, 132], z [100, 160]; grown by 25 % of the extent
    per side: x, y [122, 134], z [85, 175]; outward to whole finest blocks:
    x, y [120, 136], z [80, 176].  Level 1: that box's footprint [60, 68] x
    [60, 68] x [40, 88], outward to blocks [56, 72] x [56, 72] x [40, 88],
    plus one block per side: [48, 80] x [48, 80] x [32, 96].  The library
    builds the same boxes; a tree whose level-1 box would leave the domain is
    rejected."""
    from paper_2603_27954_gb300 import lbm as L
    seg = np.array([[128.0, 128.0, 100.0, 128.0, 128.0, 160.0, 8.0, 0.0]])
    want = [None, [48, 48, 32, 80, 80, 96], [120, 120, 80, 136, 136, 176]]
    assert O.refine_boxes(seg, 3, (64, 64, 64), 8) == want
    h = L.lbm_create_domain(L.domain_desc(64, 64, 64, levels=3, block=8, bc=("inout", "slip", "slip"),
                                          nu_finest=0.01))
    L.lbm_set_geometry_segments(h, seg)
    for lv in (1, 2):
        info = L.lbm_level_info(h, lv)
        assert list(info["lo"]) + list(info["hi"]) == want[lv]
    L.lbm_destroy(h)
    # near the floor: the level-1 box would start at z = -8
    low = np.array([[40.0, 32.0, 20.0, 40.0, 32.0, 40.0, 4.0, 0.0]])
    assert O.refine_boxes(low, 3, (32, 16, 16), 8)[1][2] < 0
    h = L.lbm_create_domain(L.domain_desc(32, 16, 16, levels=3, block=8, bc=("inout", "slip", "slip"),
                                          nu_finest=0.01))
    with pytest.raises(L.LbmError) as e:
        L.lbm_set_geometry_segments(h, low)
    assert e.value.code == L.LBM_EINVAL
    L.lbm_destroy(h)
