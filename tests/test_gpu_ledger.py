"""FP64 ledger of the refinement interface (lbm_interface_ledger): the mass
and momentum the volumetric coarse/fine transfer moves every coarse step -
In (coarse values handed to the fine level), OutF (fine values taken back),
RecvC (what the coarse cells receive) - against what the mathematics fixes.

1. Closed form.  In a uniform flow every fine step moves, across the surface
   of an a x b x c fine box and along c_i, the populations of the
   N_i = abc - (a - |c_x|)(b - |c_y|)(c - |c_z|) lattice links that cross it,
   each carrying f_i^eq; a coarse step is two fine steps.  So In = OutF =
   RecvC = 2 sum_i N_i f_i^eq (1, c_i) in fine-cell volumes, to the ledger's
   resolution: every recorded population deviation is rounded to a multiple
   of 2^-40, at most 2^-41 per entry (systematic in a uniform state, where
   all entries of a direction carry the same value), plus the storage
   rounding of f_i^eq in the reduced forms.
2. Conservation.  In a closed periodic box the only exchange between the
   levels is the interface, so over every coarse step the FP64 mass change of
   the fine level equals In - OutF and that of the coarse level RecvC - In,
   up to the rounding of the collisions in the storage precision: to 1e-12
   of the level's mass in the FP64 storage form (and for the three-level
   box), to the FP32 rounding of the stored deviations in FP32.
3. The ledger observes, it does not change the flow: populations with the
   ledger on and off are identical bit for bit.
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_27954_gb300 import workloads as W

pytestmark = pytest.mark.gpu

C27 = np.array([[i % 3 - 1, (i // 3) % 3 - 1, i // 9 - 1] for i in range(27)])


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


PREC = {"fp64": 0, "fp32": 1, "fp16": 2}


def periodic_box(L, stream, precision, levels=2, u_in=0.0):
    boxes = [None, (16, 16, 16, 48, 48, 48)]
    if levels == 3:
        boxes = [None, (16, 16, 16, 48, 48, 48), (48, 48, 48, 80, 80, 80)]
    desc = L.domain_desc(32, 32, 32, levels=levels, block=8, bc=("periodic",) * 3, u_in=u_in, nu_finest=0.04,
                         boxes=boxes, precision=PREC[precision])
    return L.Domain(desc, prims=([], np.zeros((0, 8))), stream=stream)


def crossing_flows(a, b, c, f):
    """2 sum_i N_i f_i (1, c_i): mass and momentum crossing an a x b x c box
    in two lattice steps of a uniform state f (per fine-cell volume), and the
    number of crossings 2 sum_i N_i."""
    out, links = np.zeros(4), 0
    for i in range(27):
        n = a * b * c - (a - abs(C27[i, 0])) * (b - abs(C27[i, 1])) * (c - abs(C27[i, 2]))
        out += 2 * n * f[i] * np.array([1.0, *C27[i]])
        links += 2 * n
    return out, links


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-13), ("fp32", 1e-7), ("fp16", 1e-3)])
def test_uniform_flow_ledger_equals_the_crossing_count(L, stream, precision, rtol):
    u = np.array([0.05, 0.02, -0.01])
    dom = periodic_box(L, stream, precision, u_in=0.05)
    dom.init_uniform(1.0, u)
    dom.step(3)
    last, total, steps = dom.interface_ledger(0)
    assert steps == 3
    want, links = crossing_flows(32, 32, 32, O.equilibrium(1.0, u))
    want /= 8.0  # level-1 cells weigh 1/8
    quantum = links * 2.0 ** -41 / 8.0  # the ledger's resolution, per component and coarse step
    print(precision, "ledger In", last[:4], "closed form", want, "resolution", quantum)
    for k in range(3):  # In, OutF, RecvC
        np.testing.assert_allclose(last[4 * k:4 * k + 4], want, rtol=rtol, atol=quantum + rtol * want[0])
        np.testing.assert_allclose(total[4 * k:4 * k + 4], 3 * want, rtol=rtol, atol=3 * (quantum + rtol * want[0]))
    dom.close()


def level_masses(dom, levels):
    return [dom.level_mass(l) for l in range(levels)]


def tgv_init(L, dom, levels):
    for lv in range(levels):
        info = L.lbm_level_info(dom.h, lv)
        rho, u = W.tgv_fields(info["lo"], info["hi"], 2 ** lv, 32, 0.03, (0.03, 0.01, -0.02))
        dom.init_field(lv, rho, u)


# Bounds: the FP64 form rounds at ~1e-16 per operation (the identity holds to
# ~1e-13 of the level mass); FP32 storage rounds every collision's 27
# outputs at 2^-24 of deviations ~1e-2, ~1e-8 per cell update, a random walk
# of ~2e-6 over the ~3e4 updates of a level and step (~1e-10 of its mass;
# measured 1.3e-9 over six steps; bound 5e-9, still 10x below the 6e-8 a
# single missing entry of ~1e-2 / 8 would leave); binary16 storage rounds at
# 2^-12 of the stored deviation (measured 3.2e-7; bound 2e-6).
@pytest.mark.parametrize("precision,levels,rtol", [("fp64", 2, 1e-12), ("fp64", 3, 1e-12), ("fp32", 2, 5e-9),
                                                   ("fp16", 2, 2e-6)])
def test_level_mass_changes_equal_the_ledger(L, stream, precision, levels, rtol):
    """Per coarse step and level: the FP64 mass / momentum change equals the
    ledger's flows across the level's interfaces (totals, so that an inner
    interface's two folds per coarse step - one per step of its coarser
    level - are both counted)."""
    dom = periodic_box(L, stream, precision, levels)
    tgv_init(L, dom, levels)
    before = level_masses(dom, levels)
    tot0 = [dom.interface_ledger(l)[1] for l in range(levels - 1)]
    worst = 0.0
    for step in range(6):
        dom.step(1)
        after = level_masses(dom, levels)
        tot1 = [dom.interface_ledger(l)[1] for l in range(levels - 1)]
        led = [t1 - t0 for t0, t1 in zip(tot0, tot1)]
        for lv in range(levels):
            flux = np.zeros(4)
            if lv + 1 < levels:  # coarse side of the interface below
                flux += led[lv][8:12] - led[lv][0:4]
            if lv > 0:  # fine side of the interface above
                flux += led[lv - 1][0:4] - led[lv - 1][4:8]
            dm = np.array([after[lv][0] - before[lv][0], *(after[lv][1] - before[lv][1])])
            err = np.abs(dm - flux).max() / after[lv][0]
            worst = max(worst, err)
            assert err < rtol, (precision, levels, step, lv, dm, flux)
        before, tot0 = after, tot1
    for l in range(levels - 1):
        assert dom.interface_ledger(l)[2] == 6 * 2 ** l  # folds: one per step of the coarser level
    print("%s, %d levels: worst |dM - ledger| / M = %.3g" % (precision, levels, worst))
    dom.close()


def test_ledger_leaves_the_flow_unchanged(L, stream):
    c = W.CASES["amr2_small"]
    out = []
    for on in (True, False):
        desc = L.domain_desc(*c["n0"], levels=c["levels"], block=c["block"], bc=c["bc"], u_in=c["u_in"],
                             re_h=c["re_h"])
        d = L.Domain(desc, tree=L.tree_desc(**c["tree"]), stream=stream)
        d.set_interface_ledger(on)
        d.step(4)
        out.append([d.get_populations(l) for l in range(2)] + [d.drag()[1]])
        if on:
            assert d.interface_ledger(0)[2] == 4
        else:
            assert d.interface_ledger(0)[2] == 0
        d.close()
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)
