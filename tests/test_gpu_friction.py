"""GPU parity of the friction force (C_F) against the FP64 oracle on the same
quadrature points.  The GPU reads FP32 deviations (rounding ~1e-9 on values
~1e-2) and forms the stress in FP64; the stress is a difference of O(1e-4)
moments, so the per-branch friction carries ~1e-5 relative error, held to
1e-4 like the momentum-exchange force (FP16 storage: 2e-2)."""
import numpy as np
import pytest

import oracle as O
from oracle import friction as Fr
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


def setup(L, stream, case, precision=None):
    c = W.CASES[case]
    t = c["tree"]
    desc = L.domain_desc(*c["n0"], levels=c["levels"], block=c["block"], bc=c["bc"], u_in=c["u_in"],
                         re_h=c["re_h"], precision=precision or L.LBM_FP32)
    dom = L.Domain(desc, tree=L.tree_desc(**t), stream=stream)
    tree = O.make_tree(t["n"], t["children"], t["s0"], t["w0"], t["r"], t["dfac"], alpha_deg=t["alpha_deg"],
                       azimuth_mode=t["azimuth_mode"], seed=t["seed"])
    sim, info = O.tree_case(*c["n0"], tree, t["trunk_cells"], c["re_h"], u_in=c["u_in"], levels=c["levels"],
                            block=c["block"], bc=c["bc"])
    return dom, sim, info, c


def oracle_friction(dom, sim, info, c):
    lv = c["levels"] - 1
    rows = dom.friction_samples()
    lo = np.array(sim.box(lv)[0])
    f = sim.f(lv)
    omega1 = 1.0 / (3.0 * info["nu_finest"] + 0.5)

    def pops(cells):
        q = cells - lo
        return f[q[:, 2], q[:, 1], q[:, 0]]

    F = Fr.friction(rows, pops, omega1)
    return Fr.per_branch(F, rows, len(info["segments"]))


@pytest.mark.parametrize("case,steps", [("tiny", (1, 40)), ("amr2_small", (1, 3))])
def test_friction_matches_oracle(L, stream, case, steps):
    dom, sim, info, c = setup(L, stream, case)
    nb = len(info["segments"])
    done = 0
    for s in steps:
        dom.step(s - done)
        sim.step(s - done)
        done = s
        tot, rows, cf = dom.friction(nb)
        ref = oracle_friction(dom, sim, info, c)
        scale = np.abs(ref).max()
        np.testing.assert_allclose(rows, ref, rtol=1e-4, atol=1e-4 * scale)
        np.testing.assert_allclose(tot, ref.sum(axis=0), rtol=1e-4, atol=1e-4 * scale)
        assert cf == pytest.approx(tot[0] / (0.5 * c["u_in"] ** 2 * dom.geometry_info()["A_x"]), rel=1e-12)
    dom.close()


def test_fp16_friction_matches_oracle(L, stream):
    dom, sim, info, c = setup(L, stream, "tiny", L.LBM_FP16_DEV)
    dom.step(40)
    sim.step(40)
    tot, rows, _ = dom.friction(len(info["segments"]))
    ref = oracle_friction(dom, sim, info, c).sum(axis=0)
    assert abs(tot[0] - ref[0]) <= 2e-2 * abs(ref[0])
    dom.close()


def test_friction_mean_accumulates_every_coarse_step(L, stream):
    """The in-graph accumulation equals the mean of on-demand evaluations
    after each coarse step (one and two levels, both parities)."""
    for case in ("tiny", "amr2_small"):
        dom, _, info, _ = setup(L, stream, case)
        nb = len(info["segments"])
        dom.step(2)
        dom.set_friction_mean(True)
        dom.reset_force()
        vals = []
        for _ in range(5):
            dom.step(1)
            vals.append(dom.friction(nb)[1])
        mean, rows, n = dom.get_friction_mean(nb)
        assert n == 5
        np.testing.assert_allclose(rows, np.mean(vals, axis=0), rtol=1e-12, atol=1e-18)
        np.testing.assert_allclose(mean, np.mean(vals, axis=0).sum(axis=0), rtol=1e-12, atol=1e-18)
        dom.close()
