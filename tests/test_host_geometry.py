"""The library's host side (no GPU needed) against the oracle: the L-system,
placement, tree height, frontal area, refinement boxes, cell classification
per level and the cut links with their wall fractions.  Cell types and link
sets are integer data and must agree exactly."""
import functools

import numpy as np
import pytest

import oracle as O
from paper_2603_27954_gb300 import lbm as L
from paper_2603_27954_gb300 import workloads as W


def oracle_tree(t):
    return O.make_tree(t["n"], t["children"], t["s0"], t["w0"], t["r"], t["dfac"], alpha_deg=t["alpha_deg"],
                       phi_deg=t.get("phi_deg", (0.0,)), azimuth_mode=t["azimuth_mode"], seed=t["seed"])


def lib_domain(case):
    c = W.CASES[case]
    d = L.domain_desc(*c["n0"], levels=c["levels"], block=c["block"], bc=c["bc"], u_in=c["u_in"], re_h=c["re_h"])
    h = L.lbm_create_domain(d)
    L.lbm_set_geometry(h, L.tree_desc(**c["tree"]))
    return h


@pytest.fixture(scope="module", autouse=True)
def _release_oracle_cases():
    """The cached oracle geometries (several GB for the four-level case) live
    only as long as this module's tests."""
    yield
    oracle_case.cache_clear()


@functools.lru_cache(maxsize=None)
def oracle_case(case):
    """The oracle's geometry of a workload case (built once per case; the
    tests here only read it)."""
    c = W.CASES[case]
    return O.tree_case(*c["n0"], oracle_tree(c["tree"]), c["tree"]["trunk_cells"], c["re_h"], u_in=c["u_in"],
                       levels=c["levels"], block=c["block"], bc=c["bc"])


@pytest.mark.parametrize("n", [4, 6, 8])
def test_lsystem_matches_oracle_paper_form(n):
    """Table 1 trees (fixed phi = 137 deg): identical segments."""
    h = L.lbm_create_domain(L.domain_desc(64, 64, 64, bc=("periodic",) * 3, nu_finest=0.01))
    t = L.tree_desc(n, trunk_cells=100.0)
    L.lbm_set_geometry(h, t)
    seg = L.lbm_get_segments(h)
    ref = O.place_tree(O.make_tree(n), 100.0, (64, 64, 64))
    np.testing.assert_allclose(seg, ref, rtol=0, atol=1e-9)
    L.lbm_destroy(h)


@pytest.mark.parametrize("case", ["tiny", "amr2_small", "amr2", "amr3_small", "amr4_quarter"])
def test_geometry_scalars_match_oracle(case):
    h = lib_domain(case)
    g = L.lbm_geometry_info(h)
    _, info = oracle_case(case) if case != "amr2" else (None, None)
    if info is None:
        c = W.CASES[case]
        fin = 2 ** (c["levels"] - 1)
        seg = O.place_tree(oracle_tree(c["tree"]), c["tree"]["trunk_cells"], tuple(n * fin for n in c["n0"]))
        info = {"segments": seg, "H": O.tree_height(seg), "A_x": O.frontal_area(seg),
                "boxes": O.refine_boxes(seg, c["levels"], c["n0"], c["block"])}
    np.testing.assert_allclose(L.lbm_get_segments(h), info["segments"], atol=1e-9)
    assert g["H"] == pytest.approx(info["H"], rel=1e-12)
    assert g["A_x"] == pytest.approx(info["A_x"], rel=1e-12)
    for l in range(1, len(info["boxes"])):
        li = L.lbm_level_info(h, l)
        assert list(li["lo"]) + list(li["hi"]) == list(info["boxes"][l])
    if case in ("amr3_small", "amr4_quarter"):
        # fluid cells and cut links per level, and the cell updates of a coarse step (sum n_l 2^l)
        sim, _ = oracle_case(case)
        work = 0
        for l in range(len(info["boxes"])):
            li = L.lbm_level_info(h, l)
            nf = int((sim.cell_type(l) == 0).sum())
            assert li["n_fluid"] == nf and li["n_links"] == len(sim.links(l)[0])
            work += nf << l
        assert L.lbm_work_per_step(h)[0] == work
    L.lbm_destroy(h)


@pytest.mark.parametrize("case", ["tiny", "amr2_small", "amr3_small", "amr4_quarter"])
def test_cell_types_and_links_match_oracle(case):
    h = lib_domain(case)
    sim, info = oracle_case(case)
    levels = W.CASES[case]["levels"]
    total_links = 0
    for l in range(levels):
        lt = L.lbm_get_cell_types(h, l)
        ot = sim.cell_type(l)
        np.testing.assert_array_equal(lt, ot)
        c1, d1, q1 = L.lbm_get_links(h, l)
        c2, d2, q2 = sim.links(l)
        k1 = np.lexsort((d1, c1))
        k2 = np.lexsort((d2, c2))
        np.testing.assert_array_equal(c1[k1], c2[k2])
        np.testing.assert_array_equal(d1[k1], d2[k2])
        # two independent FP64 ray-cylinder computations: they agree to a few
        # 1e-12 at finest coordinates of several hundred cells
        np.testing.assert_allclose(q1[k1], q2[k2], rtol=0, atol=1e-11)
        total_links += len(q1)
        if len(q1):
            assert (q1 > 0).all() and (q1 <= 1).all()
    assert total_links > 0
    L.lbm_destroy(h)


@pytest.mark.parametrize("case", ["tiny", "amr2_small", "amr2_quarter", "amr3_small", "amr4_quarter"])
def test_link_branches_match_oracle(case):
    """The branch each finest-level cut link is attributed to (the cylinder
    its ray enters first; per-branch forces, Sec. 2.4) is the oracle's,
    link for link: integer data, compared exactly."""
    h = lib_domain(case)
    sim, _ = oracle_case(case)
    fin = W.CASES[case]["levels"] - 1
    c1, d1, _ = L.lbm_get_links(h, fin)
    b1 = L.lbm_get_link_branches(h, fin)
    c2, d2, _ = sim.links(fin)
    b2 = sim.link_segments(fin)
    k1, k2 = np.lexsort((d1, c1)), np.lexsort((d2, c2))
    np.testing.assert_array_equal(c1[k1], c2[k2])
    np.testing.assert_array_equal(d1[k1], d2[k2])
    np.testing.assert_array_equal(b1[k1], b2[k2])
    assert len(np.unique(b1)) == L.lbm_geometry_info(h)["n_segments"]
    L.lbm_destroy(h)


def test_planar_walls_links_match_oracle():
    """General primitives (two half-spaces) classify and link identically."""
    kinds = [1, 1]
    params = np.zeros((2, 8))
    params[0, :4] = (0, 1, 0, 2.3)
    params[1, :4] = (0, -1, 0, -17.8)
    h = L.lbm_create_domain(L.domain_desc(16, 20, 16, bc=("periodic", "periodic", "periodic"), nu_finest=0.1))
    with pytest.raises(L.LbmError):
        L.lbm_set_geometry_prims(h, kinds, params)  # y = 20 is not a multiple of the block
    L.lbm_destroy(h)
    h = L.lbm_create_domain(L.domain_desc(16, 32, 16, block=16, bc=("periodic",) * 3, nu_finest=0.1))
    params[1, :4] = (0, -1, 0, -29.6)
    L.lbm_set_geometry_prims(h, kinds, params)
    s = O.Sim(16, 32, 16, bc=("periodic",) * 3, nu0=0.1, u_in=0.0)
    s.set_prims(O.prims([(1, params[0, :4]), (1, params[1, :4])]))
    np.testing.assert_array_equal(L.lbm_get_cell_types(h, 0), s.cell_type(0))
    c1, d1, q1 = L.lbm_get_links(h, 0)
    c2, d2, q2 = s.links(0)
    k1, k2 = np.lexsort((d1, c1)), np.lexsort((d2, c2))
    np.testing.assert_array_equal(c1[k1], c2[k2])
    np.testing.assert_allclose(q1[k1], q2[k2], atol=1e-12)
    L.lbm_destroy(h)


def test_degenerate_wall_fractions_clamp_alike():
    """Walls that graze the cell centres: a plane 1e-9 below a row of fluid
    centres gives q = 1e-9, clamped to 1e-6, and a plane through a row of
    centres makes that row solid (inclusive test) and gives q = 1 from the
    next row.  Library and oracle classify, link and clamp identically."""
    kinds = [1, 1]
    params = np.zeros((2, 8))
    params[0, :4] = (0, 1, 0, 10.5 - 1e-9)   # n.x <= d: rows y <= 9 solid, row 10 fluid at 1e-9
    params[1, :4] = (0, -1, 0, -20.5)        # -y <= -20.5: rows y >= 20 solid (centre 20.5 on the plane)
    h = L.lbm_create_domain(L.domain_desc(16, 32, 16, block=16, bc=("periodic",) * 3, nu_finest=0.1))
    L.lbm_set_geometry_prims(h, kinds, params)
    s = O.Sim(16, 32, 16, bc=("periodic",) * 3, nu0=0.1, u_in=0.0)
    s.set_prims(O.prims([(1, params[0, :4]), (1, params[1, :4])]))
    t = L.lbm_get_cell_types(h, 0)
    np.testing.assert_array_equal(t, s.cell_type(0))
    assert (t[:, 10, :] == 0).all() and (t[:, 9, :] == 1).all() and (t[:, 20, :] == 1).all()
    c1, d1, q1 = L.lbm_get_links(h, 0)
    c2, d2, q2 = s.links(0)
    k1, k2 = np.lexsort((d1, c1)), np.lexsort((d2, c2))
    np.testing.assert_array_equal(c1[k1], c2[k2])
    np.testing.assert_array_equal(d1[k1], d2[k2])
    np.testing.assert_allclose(q1[k1], q2[k2], rtol=0, atol=1e-15)
    y = (c1 // 16) % 32
    cy = (d1 // 3) % 3 - 1
    assert np.all(q1[(y == 10) & (cy == -1)] == 1e-6)
    assert np.all(q1[(y == 19) & (cy == 1)] == 1.0)
    L.lbm_destroy(h)


def test_invalid_descriptors_are_rejected():
    bad = [
        dict(levels=0), dict(levels=7), dict(block=12), dict(u_in=0.5),
    ]
    for kw in bad:
        args = dict(nx=32, ny=32, nz=32, bc=("inout", "slip", "slip"), nu_finest=0.01)
        args.update(kw)
        nx, ny, nz = args.pop("nx"), args.pop("ny"), args.pop("nz")
        with pytest.raises(L.LbmError) as e:
            L.lbm_create_domain(L.domain_desc(nx, ny, nz, **args))
        assert e.value.code == L.LBM_EINVAL
    h = L.lbm_create_domain(L.domain_desc(32, 32, 32, bc=("inout", "slip", "slip"), nu_finest=0.01))
    with pytest.raises(L.LbmError) as e:
        L.lbm_memory_requirements(h)
    assert e.value.code == L.LBM_ESTATE
    with pytest.raises(L.LbmError) as e:
        L.lbm_step(h, 1)
    assert e.value.code == L.LBM_ESTATE
    L.lbm_destroy(h)


def test_ragged_domain_keeps_every_cell():
    """A domain that is not a multiple of the block size: partial blocks hold
    the extra cells, the rest of those blocks is outside."""
    h = L.lbm_create_domain(L.domain_desc(40, 20, 24, bc=("inout", "slip", "slip"), nu_finest=0.02))
    L.lbm_set_geometry_prims(h, [], np.zeros((0, 8)))
    info = L.lbm_level_info(h, 0)
    assert info["n_fluid"] == 40 * 20 * 24
    assert info["n_active_blocks"] == 3 * 2 * 2
    assert (L.lbm_get_cell_types(h, 0) == 0).all()
    L.lbm_destroy(h)


@pytest.mark.parametrize("mode", [0, 1])
def test_lsystem_with_four_distinct_children_matches_oracle(mode):
    """Rule p1 with the most children the boundary allows (4), each with its
    own length and diameter factor, branching angle and turn, in both child
    orientation forms: the library's string rewriting and turtle give the
    oracle's recursive turtle's segments."""
    kw = dict(children=4, s0=40.0, w0=8.0, r=(0.7, 0.6, 0.5, 0.65), dfac=(0.7, 0.6, 0.55, 0.5),
              alpha_deg=(25.0, -40.0, 55.0, -15.0), phi_deg=(0.0, 90.0, 200.0, 300.0), azimuth_mode=mode, seed=9)
    h = L.lbm_create_domain(L.domain_desc(64, 64, 64, bc=("periodic",) * 3, nu_finest=0.01))
    L.lbm_set_geometry(h, L.tree_desc(4, trunk_cells=20.0, **kw))
    seg = L.lbm_get_segments(h)
    L.lbm_destroy(h)
    ref = O.place_tree(O.make_tree(4, **kw), 20.0, (64, 64, 64))
    assert len(seg) == 1 + 4 + 16 + 64
    np.testing.assert_allclose(seg, ref, rtol=0, atol=1e-9)
