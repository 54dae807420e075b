"""The FP64 storage form (LBM_FP64): populations stored as FP64 deviations
f - w, collision and bounce-back in FP64 with FP64 wall fractions - the method
in the precision the paper's smallest workload states, on the GPU - against
the FP64 oracle on the same seeded inputs.

Both sides compute the same FP64 arithmetic in different orders (the
kernel's closed-form rates-1 collision against the oracle's set-partition
cumulant transform), so they differ by rounding alone: ~1e-16 per operation,
a few hundred operations per cell update, accumulated over the run.
Tolerances: populations within 1e-13 absolute over short horizons; after the
1000-step tiny case (laminar, Re_H = 100) C_D within 1e-9 relative and the
velocity within 1e-10 relative L2.  A closed refined box conserves mass and
momentum to 1e-13 relative.
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


def gpu_case(L, stream, case):
    c = W.CASES[case]
    desc = L.domain_desc(*c["n0"], levels=c["levels"], block=c["block"], bc=c["bc"], u_in=c["u_in"],
                         re_h=c["re_h"], precision=L.LBM_FP64)
    return L.Domain(desc, tree=L.tree_desc(**c["tree"]), stream=stream)


def oracle_case(case):
    c = W.CASES[case]
    t = c["tree"]
    tree = O.make_tree(t["n"], t["children"], t["s0"], t["w0"], t["r"], t["dfac"], alpha_deg=t["alpha_deg"],
                       azimuth_mode=t["azimuth_mode"], seed=t["seed"])
    return O.tree_case(*c["n0"], tree, t["trunk_cells"], c["re_h"], u_in=c["u_in"], levels=c["levels"],
                       block=c["block"], bc=c["bc"])


def max_err(f, ref):
    ok = ~np.isnan(ref)
    assert np.array_equal(ok, ~np.isnan(f)), "fluid masks differ"
    return float(np.abs(f[ok] - ref[ok]).max())


@pytest.mark.parametrize("case,checkpoints", [("tiny", (1, 5, 20)), ("amr2_small", (1, 4)), ("amr3_small", (1, 2))])
def test_fp64_populations_match_the_oracle(L, stream, case, checkpoints):
    dom = gpu_case(L, stream, case)
    sim, _ = oracle_case(case)
    done = 0
    for n in checkpoints:
        dom.step(n - done)
        sim.step(n - done)
        done = n
        for lv in range(W.CASES[case]["levels"]):
            err = max_err(dom.get_populations(lv), sim.f(lv))
            assert err < 1e-13, (case, n, lv, err)
        last, _, _ = dom.drag()
        ref, _, _ = sim.force()
        np.testing.assert_allclose(last, ref, rtol=1e-11, atol=1e-14)
    dom.close()


def test_fp64_tiny_case_drag_and_velocity_after_1000_steps(L, stream):
    """The paper-sized smallest workload (64x32x32, Re_H = 100, 1000 steps) in
    FP64 on both sides."""
    c = W.CASES["tiny"]
    dom = gpu_case(L, stream, "tiny")
    sim, info = oracle_case("tiny")
    dom.step(c["steps"])
    sim.step(c["steps"])
    last, mean, cd = dom.drag()
    ref, ref_sum, n = sim.force()
    cd_ref = O.drag_coefficient(ref[0], c["u_in"], info["A_x"])
    print("FP64 C_D %.15f oracle %.15f rel %.2e" % (cd, cd_ref, abs(cd - cd_ref) / abs(cd_ref)))
    assert abs(cd - cd_ref) <= 1e-9 * abs(cd_ref)
    np.testing.assert_allclose(mean, ref_sum / n, rtol=1e-9, atol=1e-13)
    _, u = dom.get_velocity(0)
    _, ur = sim.macro(0)
    ok = ~np.isnan(ur[..., 0])
    rel = np.sqrt(((u[ok] - ur[ok]) ** 2).sum() / (ur[ok] ** 2).sum())
    assert rel < 1e-10, rel
    dom.close()


def test_fp64_refined_periodic_box_conserves_mass(L, stream):
    desc = L.domain_desc(32, 32, 32, levels=2, block=8, bc=("periodic",) * 3, u_in=0.0, nu_finest=0.04,
                         boxes=[None, (16, 16, 16, 48, 48, 48)], precision=L.LBM_FP64)
    dom = L.Domain(desc, prims=([], np.zeros((0, 8))), stream=stream)
    for lv in range(2):
        info = L.lbm_level_info(dom.h, lv)
        rho, u = W.tgv_fields(info["lo"], info["hi"], 2 ** lv, 32, 0.03, (0.03, 0.01, -0.02))
        dom.init_field(lv, rho, u)
    m0, p0 = dom.mass()
    dom.step(10)
    m1, p1 = dom.mass()
    assert abs(m1 - m0) / m0 < 1e-13
    np.testing.assert_allclose(p1, p0, atol=1e-13 * m0)
    dom.close()


def test_fp64_rejects_turbulent_inflow_and_batches(L, stream):
    c = W.CASES["tiny"]
    desc = L.domain_desc(*c["n0"], levels=1, block=16, bc=c["bc"], u_in=0.05, re_h=100.0, i_u=0.08,
                         precision=L.LBM_FP64)
    with pytest.raises(L.LbmError):
        L.lbm_create_domain(desc)
    d = gpu_case(L, stream, "tiny")
    with pytest.raises(L.LbmError):
        L.Batch([d], stream=stream)
    d.close()
