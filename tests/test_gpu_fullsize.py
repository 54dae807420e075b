"""The benchmark workloads at full size, checked where the oracle cannot run them whole.

Two levels, coarse 256 x 128 x 128 in 16^3 blocks, the n = 4 x 3-children
tree with a trunk of 64 finest cells, Re_H = 2.5e3 (1.27e7 cell updates per
coarse step), in FP32 and in the FP16 deviation form, in the launch
configuration the benchmark times: the schedule the library's autotuner
picks and graph replay.  From a non-uniform state, one coarse step of the
GPU is compared on sampled interior cells of both levels with the FP64
oracle's one-cell collision applied 2^l times (`sampled_cells`), within the
element-wise tolerances of the smaller parity cases (2e-6 absolute on the
populations in FP32, 2e-4 in binary16 storage).
"""
import numpy as np
import pytest

from paper_2603_27954_gb300 import workloads as W
from sampled_cells import C27, Recursion, check_level, window_all_fluid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_27954_gb300 import lbm
    return lbm


@pytest.mark.parametrize("precision,atol", [("fp32", 2e-6), ("fp16", 2e-4)])
def test_benchmark_workload_sampled_cells_match_the_oracle(L, precision, atol):
    import torch
    stream = torch.cuda.Stream()
    c = W.CASES["amr2"]
    prec = L.LBM_FP16_DEV if precision == "fp16" else L.LBM_FP32
    desc = L.domain_desc(*c["n0"], levels=c["levels"], block=c["block"], bc=c["bc"], u_in=c["u_in"],
                         re_h=c["re_h"], precision=prec)
    dom = L.Domain(desc, tree=L.tree_desc(**c["tree"]), stream=stream)
    schedule, _ = dom.autotune(8)
    for lv in range(2):
        info = dom.level_info(lv)
        rho, u = W.tgv_fields(info["lo"], info["hi"], 2 ** lv, 32, 0.02, (c["u_in"], 0.0, 0.01))
        dom.init_field(lv, rho, u)
    dom.reset_force()
    dom.step(2)
    before = [dom.get_populations(lv) for lv in range(2)]
    dom.step(1)
    nu_finest = dom.geometry_info()["nu_finest"]
    for lv in range(2):
        after = dom.get_populations(lv)
        n, err, moved = check_level(before[lv], after, dom.get_cell_types(lv), lv, nu_finest / 2 ** (1 - lv),
                                    150, 10 + lv, atol)
        print("%s level %d: %d sampled cells, max |f - f_oracle| = %.3g (populations moved up to %.3g); schedule %s"
              % (precision, lv, n, err, moved, schedule.as_dict()))
        assert n == 150 and moved > 1e-5  # the state changes by far more than the error
    assert np.isfinite(dom.drag()[2])
    dom.close()


def test_population_window_equals_the_whole_level_readback(L):
    """lbm_get_populations_window (a gather of only the window's stored
    elements) returns exactly the window of the whole-level readback, in both
    AA parities and in both storage forms."""
    import torch
    stream = torch.cuda.Stream()
    c = W.CASES["amr2_small"]
    for prec in (L.LBM_FP32, L.LBM_FP16_DEV):
        desc = L.domain_desc(*c["n0"], levels=c["levels"], block=c["block"], bc=c["bc"], u_in=c["u_in"],
                             re_h=c["re_h"], precision=prec)
        dom = L.Domain(desc, tree=L.tree_desc(**c["tree"]), stream=stream)
        for steps in (3, 1):
            dom.step(steps)
            for lv in range(2):
                whole = dom.get_populations(lv)
                nz, ny, nx, _ = whole.shape
                for lo, hi in (((0, 0, 0), (nx, ny, nz)), ((3, 5, 2), (nx - 1, 9, nz - 4)), ((7, 7, 7), (8, 8, 8))):
                    win = dom.get_populations_window(lv, lo, hi)
                    np.testing.assert_array_equal(win, whole[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]])
        with pytest.raises(L.LbmError):
            dom.get_populations_window(0, (0, 0, 0), (c["n0"][0] + 1, 1, 1))
        dom.close()


@pytest.mark.parametrize("precision,atol", [("fp32", 2e-6), ("fp16", 2e-4)])
def test_four_level_workload_sampled_finest_cells_match_the_oracle(L, precision, atol):
    """The four-level workload (coarse 512 x 256 x 256, n = 5 x 3-children
    tree, trunk 360 finest cells, Re_H = 1.2e5, 6.1e8 active cells; its finest
    level holds more than 2^31 stored elements, so every kernel addresses it
    with 64-bit offsets) under the autotuned schedule, from the impulsive
    start: after 12 coarse steps, one more coarse step (8 finest sub-steps) of
    seeded finest-level cells 9-24 cells off the tree's surface - where the
    flow has moved - against the oracle's one-cell collision applied eight
    times over the cell's 17^3 neighbourhood.  The coarser levels run the
    kernels the two-level workload checks on sampled cells; from the
    impulsive start their flow here is still the uniform inflow."""
    import torch
    stream = torch.cuda.Stream()
    c = W.CASES["amr4"]
    prec = L.LBM_FP16_DEV if precision == "fp16" else L.LBM_FP32
    desc = L.domain_desc(*c["n0"], levels=c["levels"], block=c["block"], bc=c["bc"], u_in=c["u_in"],
                         re_h=c["re_h"], precision=prec)
    dom = L.Domain(desc, tree=L.tree_desc(**c["tree"]), stream=stream)
    fin = c["levels"] - 1
    k = 2 ** fin
    schedule, _ = dom.autotune(3)
    dom.init_uniform(1.0, (c["u_in"], 0.0, 0.0))
    dom.reset_force()
    dom.step(12)
    types = dom.get_cell_types(fin)
    cell, d, _ = dom.get_links(fin)
    nz, ny, nx = types.shape
    rng = np.random.default_rng(5)
    samples = []
    for t in rng.permutation(len(cell))[:4000]:
        z, rem = divmod(int(cell[t]), nx * ny)
        y, x = divmod(rem, nx)
        cx, cy, cz = C27[d[t]]
        m = int(rng.integers(k + 1, k + 17))  # away from the wall, against the link's direction
        cand = (z - m * cz, y - m * cy, x - m * cx)
        if window_all_fluid(types, cand, k):
            samples.append(cand)
        if len(samples) == 16:
            break
    assert len(samples) == 16
    before = []
    for (z, y, x) in samples:
        before.append(dom.get_populations_window(fin, (x - k, y - k, z - k), (x + k + 1, y + k + 1, z + k + 1)))
    dom.step(1)
    nu = dom.geometry_info()["nu_finest"]
    err = moved = 0.0
    for (z, y, x), S0 in zip(samples, before):
        got = dom.get_populations_window(fin, (x, y, z), (x + 1, y + 1, z + 1))[0, 0, 0]
        want = Recursion(S0, nu).after((k, k, k), k)
        e = float(np.abs(got - want).max())
        assert e < atol, "finest cell (z,y,x) = %s: max |f - f_oracle| = %g" % ((z, y, x), e)
        err, moved = max(err, e), max(moved, float(np.abs(got - S0[k, k, k]).max()))
    print("%s four-level finest level: 16 sampled cells, max |f - f_oracle| = %.3g (moved up to %.3g); "
          "schedule %s" % (precision, err, moved, schedule.as_dict()))
    assert moved > 1e-5  # the state changes by far more than the error
    dom.close()
    torch.cuda.empty_cache()  # return the 46-87 GB buffer to the device for the tests after this one
