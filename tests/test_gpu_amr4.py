"""Four-level block AMR (the precision-form workload, Re_H = 1.2e5).

Quarter scale (coarse 128x64x64, 8^3 blocks, 1.07e7 active cells): every
population of all four levels against the FP64 oracle after one coarse step
(eight finest steps through three nested interfaces), the drag after two;
the FP16-deviation form against the same oracle.  Full scale (coarse
512x256x256, 6.1e8 active cells, 87 GB in FP32): properties that hold at any
size - finite drag that the two storage forms agree on, per-branch forces
adding up to the total, mass bookkeeping in FP64.

Tolerances: FP32 deviations round at ~1e-9 per update, so populations stay
within 2e-6 of the oracle over these few updates; FP16 deviations carry an
11-bit significand on values up to ~0.05, ~3e-5 per rounding, held to 2e-4
after eight updates.
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


def gpu_case(L, stream, case, precision=None):
    c = W.CASES[case]
    desc = L.domain_desc(*c["n0"], levels=c["levels"], block=c["block"], bc=c["bc"], u_in=c["u_in"],
                         re_h=c["re_h"], precision=precision or L.LBM_FP32)
    return L.Domain(desc, tree=L.tree_desc(**c["tree"]), stream=stream)


@pytest.fixture(scope="module")
def quarter_oracle():
    """Oracle states of the quarter-scale case after one and two coarse steps."""
    c = W.CASES["amr4_quarter"]
    t = c["tree"]
    tree = O.make_tree(t["n"], t["children"], t["s0"], t["w0"], t["r"], t["dfac"], alpha_deg=t["alpha_deg"],
                       azimuth_mode=t["azimuth_mode"], seed=t["seed"])
    sim, info = O.tree_case(*c["n0"], tree, t["trunk_cells"], c["re_h"], u_in=c["u_in"], levels=c["levels"],
                            block=c["block"], bc=c["bc"])
    sim.step(1)
    pops = [sim.f(l) for l in range(c["levels"])]
    f1 = sim.force()[0]
    sim.step(1)
    f2 = sim.force()[0]
    return dict(pops=pops, force1=f1, force2=f2, info=info)


def max_pop_error(f, ref):
    ok = ~np.isnan(ref)
    assert np.array_equal(ok, ~np.isnan(f)), "fluid masks differ"
    return float(np.abs(f[ok] - ref[ok]).max())


def test_quarter_scale_fp32_matches_oracle(L, stream, quarter_oracle):
    dom = gpu_case(L, stream, "amr4_quarter")
    for l in range(4):
        info = L.lbm_level_info(dom.h, l)
        assert list(info["lo"]) + list(info["hi"]) == (
            [0, 0, 0] + list(W.CASES["amr4_quarter"]["n0"]) if l == 0 else list(quarter_oracle["info"]["boxes"][l]))
    dom.step(1)
    for l in range(4):
        err = max_pop_error(dom.get_populations(l), quarter_oracle["pops"][l])
        assert err < 2e-6, (l, err)
    np.testing.assert_allclose(dom.drag()[0], quarter_oracle["force1"], rtol=1e-4)
    dom.step(1)
    np.testing.assert_allclose(dom.drag()[0], quarter_oracle["force2"], rtol=1e-4)
    dom.close()


def test_quarter_scale_fp16_matches_oracle(L, stream, quarter_oracle):
    dom = gpu_case(L, stream, "amr4_quarter", L.LBM_FP16_DEV)
    dom.step(1)
    for l in range(4):
        err = max_pop_error(dom.get_populations(l), quarter_oracle["pops"][l])
        assert err < 2e-4, (l, err)
    np.testing.assert_allclose(dom.drag()[0][0], quarter_oracle["force1"][0], rtol=5e-3)
    dom.step(1)
    np.testing.assert_allclose(dom.drag()[0][0], quarter_oracle["force2"][0], rtol=5e-3)
    dom.close()


@pytest.mark.slow
def test_full_scale_properties(L, stream):
    """The 6.1e8-cell case in both storage forms: finite drag within 1e-2 of
    each other after two coarse steps, branch forces that add up to the
    total, and an FP64 mass in line with the fluid volume."""
    c = W.CASES["amr4"]
    res = {}
    for name, prec in (("fp32", L.LBM_FP32), ("fp16", L.LBM_FP16_DEV)):
        dom = gpu_case(L, stream, "amr4", prec)
        dom.set_branch_forces(True)
        m0, _ = dom.mass()
        dom.step(2)
        last, mean, cd = dom.drag()
        nb = dom.geometry_info()["n_segments"]
        fb, cnt = dom.get_branch_forces(nb)
        assert cnt == 2 * 2 ** (c["levels"] - 1)
        np.testing.assert_allclose(fb.sum(axis=0), mean, rtol=0, atol=1e-9 * np.abs(fb).max())
        m1, _ = dom.mass()
        assert np.isfinite(cd) and np.isfinite(m1)
        # the inflow adds mass at most at the inflow faces' rate over two steps
        assert abs(m1 - m0) / m0 < 1e-3
        res[name] = cd
        dom.close()
    assert abs(res["fp16"] - res["fp32"]) <= 1e-2 * abs(res["fp32"]), res
