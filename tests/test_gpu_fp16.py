"""FP16-deviation storage: populations stored as (f_i - f_i^eq(1, U e_x)) * 2^13
in IEEE binary16 (deviations from the inflow equilibrium), collision in FP32,
drag and mass reductions in FP64, against the FP64 oracle.

Bounds for the reduced-precision form: C_D within 2e-3 relative of the
oracle, instantaneous and run-averaged.  A stored deviation of
size ~1e-2 carries a rounding of ~5e-6 (2^-11 relative), so populations stay
within 1e-4 absolute over the short horizons below and the velocity within
5e-3 relative L2 over the 1000-step run.
"""
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


def oracle_case(case):
    c = W.CASES[case]
    t = c["tree"]
    tree = O.make_tree(t["n"], t["children"], t["s0"], t["w0"], t["r"], t["dfac"], alpha_deg=t["alpha_deg"],
                       azimuth_mode=t["azimuth_mode"], seed=t["seed"])
    return O.tree_case(*c["n0"], tree, t["trunk_cells"], c["re_h"], u_in=c["u_in"], levels=c["levels"],
                       block=c["block"], bc=c["bc"])


def fp16_case(L, stream, case):
    c = W.CASES[case]
    desc = L.domain_desc(*c["n0"], levels=c["levels"], block=c["block"], bc=c["bc"], u_in=c["u_in"],
                         re_h=c["re_h"], precision=L.LBM_FP16_DEV)
    return L.Domain(desc, tree=L.tree_desc(**c["tree"]), stream=stream)


def max_err(f, ref):
    ok = ~np.isnan(ref)
    assert np.array_equal(ok, ~np.isnan(f))
    return np.abs(f[ok] - ref[ok]).max()


def test_fp16_tiny_case_drag_within_2e3(L, stream):
    c = W.CASES["tiny"]
    dom = fp16_case(L, stream, "tiny")
    sim, info = oracle_case("tiny")
    dom.step(c["steps"])
    sim.step(c["steps"])
    _, mean, cd = dom.drag()
    ref, ref_sum, n = sim.force()
    cd_ref = O.drag_coefficient(ref[0], c["u_in"], info["A_x"])
    mean_ref = ref_sum / n
    print("fp16 C_D %.6f oracle %.6f rel %.2e; mean F_x rel %.2e" % (
        cd, cd_ref, abs(cd - cd_ref) / abs(cd_ref), abs(mean[0] - mean_ref[0]) / abs(mean_ref[0])))
    # the 2e-3 target of the FP16 form, on the instantaneous C_D and on the run-averaged drag
    # (measured on GB300 with deviations stored from the inflow equilibrium: 1.6e-3 and 6.0e-4)
    assert abs(cd - cd_ref) <= 2e-3 * abs(cd_ref), (cd, cd_ref)
    assert abs(mean[0] - mean_ref[0]) <= 2e-3 * abs(mean_ref[0]), (mean, mean_ref)
    _, u = dom.get_velocity(0)
    _, ur = sim.macro(0)
    ok = ~np.isnan(ur[..., 0])
    rel = np.sqrt(((u[ok] - ur[ok]) ** 2).sum() / (ur[ok] ** 2).sum())
    assert rel < 5e-3, rel
    dom.close()


def test_fp16_two_level_populations_short_horizon(L, stream):
    dom = fp16_case(L, stream, "amr2_small")
    sim, _ = oracle_case("amr2_small")
    done = 0
    for s in (1, 4):
        dom.step(s - done)
        sim.step(s - done)
        done = s
        for lv in (0, 1):
            assert max_err(dom.get_populations(lv), sim.f(lv)) < 1e-4
    dom.close()


def test_fp16_refined_periodic_mass(L, stream):
    """Closed refined box in binary16 storage: the FP64 mass drift over 10
    coarse steps, split by the interface ledger into the interface's
    rounding defect (RecvC - OutF: the coalesce result rounded once to
    binary16) and the rest, the rounding of the collisions' stored outputs
    (2^-12 of deviations ~1e-2, a random walk over ~3e4 cell updates per
    level and step)."""
    desc = L.domain_desc(32, 32, 32, levels=2, block=8, bc=("periodic",) * 3, u_in=0.0, nu_finest=0.04,
                         boxes=[None, (16, 16, 16, 48, 48, 48)], precision=L.LBM_FP16_DEV)
    dom = L.Domain(desc, prims=([], np.zeros((0, 8))), stream=stream)
    for lv in range(2):
        info = L.lbm_level_info(dom.h, lv)
        rho, u = W.tgv_fields(info["lo"], info["hi"], 2 ** lv, 32, 0.03, (0.03, 0.01, -0.02))
        dom.init_field(lv, rho, u)
    dom.reset_force()  # clears the ledger
    m0, _ = dom.mass()
    dom.step(10)
    m1, _ = dom.mass()
    _, total, steps = dom.interface_ledger(0)
    assert steps == 10
    defect = total[8] - total[4]  # mass the coarse level received minus what the fine level gave
    drift = m1 - m0
    print("fp16 closed box, 10 coarse steps: drift %.3e (rel %.2e), interface defect %.3e, collisions %.3e" % (
        drift, drift / m0, defect, drift - defect))
    # the interface: one binary16 rounding per coalesce result, ~3e-6 of a
    # level-0 volume per entry, random over ~5e5 entry-steps (measured
    # 2.7e-9 of the mass); the collisions: measured 1.4e-7 of the mass
    assert abs(defect) < 1e-8 * m0
    assert abs(drift - defect) < 1e-6 * m0
    assert abs(drift) < 1e-6 * m0
    dom.close()


@pytest.mark.parametrize("case", ["tiny", "amr2_small"])
def test_fp16_paired_even_step_equals_direct(L, stream, case):
    """Two cells per thread with 4-byte pair loads and stores (16^3 and 8^3
    blocks, pairs with one solid cell) give the one-cell-per-thread result
    bit for bit over both parities."""
    c = W.CASES[case]
    out = []
    for even in (0, 2):
        desc = L.domain_desc(*c["n0"], levels=c["levels"], block=c["block"], bc=c["bc"], u_in=c["u_in"],
                             re_h=c["re_h"], precision=L.LBM_FP16_DEV)
        d = L.Domain(desc, tree=L.tree_desc(**c["tree"]), stream=stream)
        d.set_schedule(0, 0, even)
        d.step(5)
        out.append([d.get_populations(l) for l in range(c["levels"])])
        d.close()
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("case", ["tiny", "amr2_small"])
def test_fp16_odd_step_variants_agree(L, stream, case):
    """The paired odd step (two x-neighbouring cells per thread, one packed
    collision) against the one-cell column-pointer and direct odd steps,
    over several z splits: the packed and the one-cell arithmetic round
    differently in the last FP32 bit, so some stored binary16 values differ
    by one unit (at most ~1.5e-5 in f at these magnitudes, most of them far
    smaller: many stored values are near zero); the pair kernel
    itself gives the same result for every z split, bit for bit."""
    c = W.CASES[case]
    B = c["block"]
    runs = {}
    for odd, zo in ((3, 1), (3, 2), (3, B // 2), (3, B), (0, 0), (2, 1)):
        desc = L.domain_desc(*c["n0"], levels=c["levels"], block=B, bc=c["bc"], u_in=c["u_in"],
                             re_h=c["re_h"], precision=L.LBM_FP16_DEV)
        d = L.Domain(desc, tree=L.tree_desc(**c["tree"]), stream=stream)
        d.set_schedule(0, odd, 2, 0, zo)
        d.step(5)
        runs[(odd, zo)] = [d.get_populations(l) for l in range(c["levels"])], d.drag()[1]
        d.close()
    ref = runs[(3, 1)]
    for key, got in runs.items():
        for a, b in zip(ref[0], got[0]):
            if key[0] == 3:
                np.testing.assert_array_equal(a, b, err_msg=str(key))
            else:
                ok = ~np.isnan(a)
                assert np.array_equal(ok, ~np.isnan(b))
                diff = np.abs(a[ok] - b[ok])
                # one binary16 unit of the stored values at most, on average far below it
                assert diff.max() < 2e-5, (key, diff.max())
                assert diff.mean() < 1e-7, (key, diff.mean())
        np.testing.assert_allclose(ref[1], got[1], rtol=1e-4, atol=1e-5 * np.abs(ref[1]).max(), err_msg=str(key))
