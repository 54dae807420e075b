"""Batched form: several domains of different sizes, level counts and inflow
kinds stepped in lockstep by one persistent collide launch per level depth
and sub-step and one CUDA graph per coarse step.  The batch must give the
populations and forces of stepping each domain alone, bit for bit, under
every schedule (persistent grid size, odd-step variant)."""
import numpy as np
import pytest

import oracle as O
from paper_2603_27954_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_27954_gb300 import lbm
    return lbm


@pytest.fixture(scope="module")
def stream():
    import torch
    return torch.cuda.Stream()


def records():
    """Four 8^3-block cases: one, two and three levels, uniform and turbulent inflow."""
    tiny8 = dict(W.CASES["tiny"], block=8)
    turb = dict(W.CASES["amr2_small"], i_u=0.08, seed=5)
    return [tiny8, W.CASES["amr2_small"], turb, W.CASES["amr3_small"]]


def make(L, stream, c):
    desc = L.domain_desc(*c["n0"], levels=c["levels"], block=c["block"], bc=c["bc"], u_in=c["u_in"],
                         re_h=c["re_h"], i_u=c.get("i_u", 0.0), seed=c.get("seed", 0))
    dom = L.Domain(desc, tree=L.tree_desc(**c["tree"]), stream=stream)
    dom.set_branch_forces(True)
    return dom


def state(dom, levels):
    return [dom.get_populations(l) for l in range(levels)], dom.drag()[1], dom.get_branch_forces(
        dom.geometry_info()["n_segments"])[0]


@pytest.mark.parametrize("ctas,odd,ze,zo,even", [(0, 0, 1, 1, 0), (2, 0, 0, 0, 0), (3, 2, 2, 8, 0), (1, 2, 4, 1, 0),
                                                 (0, 2, 8, 4, 0), (0, 3, 1, 1, 2), (2, 3, 2, 4, 2), (0, 3, 0, 0, 0)])
def test_batch_equals_domains_stepped_alone(L, stream, ctas, odd, ze, zo, even):
    """Every schedule, including the paired (two cells per thread) kernels in
    the batch, equals the domains stepped alone with the same kernels."""
    recs = records()
    alone = [make(L, stream, c) for c in recs]
    for d in alone:
        d.set_schedule(0, odd, even)
        d.step(5)
    doms = [make(L, stream, c) for c in recs]
    batch = L.Batch(doms, stream=stream)
    batch.set_schedule(ctas, odd, ze, zo, even)
    batch.step(5)
    for a, b, c in zip(alone, doms, recs):
        sa, sb = state(a, c["levels"]), state(b, c["levels"])
        for pa, pb in zip(sa[0], sb[0]):
            np.testing.assert_array_equal(pa, pb)
        np.testing.assert_array_equal(sa[1], sb[1])
        np.testing.assert_array_equal(sa[2], sb[2])
    batch.close()
    for d in alone + doms:
        d.close()


def test_batch_autotune_picks_a_candidate_and_graphs_match_direct(L, stream):
    recs = records()
    d1 = [make(L, stream, c) for c in recs]
    d2 = [make(L, stream, c) for c in recs]
    b1, b2 = L.Batch(d1, stream=stream), L.Batch(d2, stream=stream)
    best, ms = b1.autotune(steps=2)
    assert best.ctas_per_sm in (0, 1, 2, 3, 4, 6, 8) and best.odd_variant in (0, 2, 3) and ms > 0
    # both batches continue from the same state: re-initialise, then step with and without graphs
    for d in d1 + d2:
        d.init_uniform(1.0, np.array([0.05, 0.0, 0.0]))
    b2.set_schedule(best.ctas_per_sm, best.odd_variant, even_variant=best.even_variant)
    b2.use_graphs(False)
    b1.step(4)
    b2.step(4)
    for a, b, c in zip(d1, d2, recs):
        for l in range(c["levels"]):
            np.testing.assert_array_equal(a.get_populations(l), b.get_populations(l))
    for x in (b1, b2):
        x.close()
    for d in d1 + d2:
        d.close()


def test_batch_rejects_mixed_domains(L, stream):
    a = make(L, stream, records()[0])
    b = make(L, stream, W.CASES["tiny"])  # 16^3 blocks
    with pytest.raises(L.LbmError):
        L.Batch([a, b], stream=stream)
    with pytest.raises(L.LbmError):
        L.Batch([a, a], stream=stream)
    a.step(1)
    c = make(L, stream, records()[1])
    with pytest.raises(L.LbmError):
        L.Batch([a, c], stream=stream)  # different step parity
    for d in (a, b, c):
        d.close()


def test_domain_autotune_keeps_results(L, stream):
    """Every collide variant of a single domain gives the same populations."""
    c = W.CASES["amr2_small"]
    ref = make(L, stream, c)
    ref.step(3)
    want = [ref.get_populations(l) for l in range(2)]
    ref.close()
    tuned = make(L, stream, c)
    best, ms = tuned.autotune(2)
    assert ms > 0
    for odd in (0, 2):
        d = make(L, stream, c)
        d.set_schedule(0, odd, 0)
        d.step(3)
        for l in range(2):
            np.testing.assert_array_equal(d.get_populations(l), want[l])
        d.close()
    tuned.close()


def test_three_level_small_case_matches_oracle(L, stream):
    c = W.CASES["amr3_small"]
    t = c["tree"]
    dom = make(L, stream, c)
    tree = O.make_tree(t["n"], t["children"], t["s0"], t["w0"], t["r"], t["dfac"], alpha_deg=t["alpha_deg"],
                       azimuth_mode=t["azimuth_mode"], seed=t["seed"])
    sim, _ = O.tree_case(*c["n0"], tree, t["trunk_cells"], c["re_h"], u_in=c["u_in"], levels=c["levels"],
                         block=c["block"], bc=c["bc"])
    done = 0
    for s in (1, 3):
        dom.step(s - done)
        sim.step(s - done)
        done = s
        for l in range(3):
            f, ref = dom.get_populations(l), sim.f(l)
            ok = ~np.isnan(ref)
            assert np.array_equal(ok, ~np.isnan(f))
            assert np.abs(f[ok] - ref[ok]).max() < 2e-6
        np.testing.assert_allclose(dom.drag()[0], sim.force()[0], rtol=1e-4, atol=1e-7)
    dom.close()


@pytest.mark.parametrize("case,precision", [("amr2_small", "fp32"), ("amr2_small", "fp16"), ("tiny8", "fp32"),
                                            ("tiny8", "fp16")])
def test_z_splits_give_identical_results(L, stream, case, precision):
    """Any split of the blocks' z walks over several CTAs gives the same
    populations and forces bit for bit (every cell update touches only its
    own locations)."""
    c = dict(W.CASES["tiny"], block=8) if case == "tiny8" else W.CASES[case]
    prec = L.LBM_FP16_DEV if precision == "fp16" else L.LBM_FP32
    even = 2 if precision == "fp16" else 0

    def run(ze, zo):
        desc = L.domain_desc(*c["n0"], levels=c["levels"], block=c["block"], bc=c["bc"], u_in=c["u_in"],
                             re_h=c["re_h"], precision=prec)
        dom = L.Domain(desc, tree=L.tree_desc(**c["tree"]), stream=stream)
        dom.set_schedule(0, 0, even, ze, zo)
        dom.step(3)
        out = [dom.get_populations(l) for l in range(c["levels"])], dom.drag()[1]
        dom.close()
        return out

    ref = run(1, 1)
    for ze, zo in ((2, 2), (4, 4), (c["block"], c["block"]), (1, 8), (8, 1)):
        got = run(ze, zo)
        for a, b in zip(ref[0], got[0]):
            np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(ref[1], got[1])


def test_batch_matches_the_oracle(L, stream):
    """A three-domain batch (one, two and three levels in 8^3 blocks; the
    two-level one with 8 % random-Fourier-mode inflow) against the FP64
    oracle element by element, each domain compared with its own oracle
    simulation: the batched kernels and the batch's per-domain branching
    reach the method's result, not only the single-domain path's."""
    from oracle import turbulence as T
    recs = [dict(W.CASES["tiny"], block=8), dict(W.CASES["amr2_small"], i_u=0.08, seed=7), W.CASES["amr3_small"]]
    doms = [make(L, stream, c) for c in recs]
    l_int = 10.0
    doms[1].set_inflow_turbulence(256, l_int)
    sims = []
    for c in recs:
        t = c["tree"]
        tree = O.make_tree(t["n"], t["children"], t["s0"], t["w0"], t["r"], t["dfac"], alpha_deg=t["alpha_deg"],
                           azimuth_mode=t["azimuth_mode"], seed=t["seed"])
        sim, _ = O.tree_case(*c["n0"], tree, t["trunk_cells"], c["re_h"], u_in=c["u_in"], levels=c["levels"],
                             block=c["block"], bc=c["bc"])
        if c.get("i_u", 0.0) > 0:
            sim.set_turbulence(T.rfm_modes(c["seed"], 256, c["i_u"], c["u_in"], l_int), c["u_in"])
        sims.append(sim)
    batch = L.Batch(doms, stream=stream)
    batch.set_schedule(2, 0, 2, 4)
    done = 0
    for n in (1, 3):
        batch.step(n - done)
        for s in sims:
            s.step(n - done)
        done = n
        for d, s, c in zip(doms, sims, recs):
            for l in range(c["levels"]):
                f, ref = d.get_populations(l), s.f(l)
                ok = ~np.isnan(ref)
                assert np.array_equal(ok, ~np.isnan(f))
                err = np.abs(f[ok] - ref[ok]).max()
                assert err < 2e-6, (c["n0"], l, n, err)
            np.testing.assert_allclose(d.drag()[0], s.force()[0], rtol=1e-4, atol=1e-7)
    batch.close()
    for d in doms:
        d.close()
