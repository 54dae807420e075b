"""The benchmark workload itself, checked where the oracle cannot run it whole.

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
from sampled_cells import check_level

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
