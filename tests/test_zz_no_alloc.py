"""lbm_mass_noalloc: the mass / momentum check for callers that may not
allocate device memory when they call it (an allocator or pool that forbids
growth).  Its reduction scratch is a fixed array inside the library, so the
call allocates nothing; it must agree with lbm_mass, which uses scratch from
the domain's bound buffer, in both storage forms (FP32 deviations, and
binary16 deviations from the inflow equilibrium with their scale).

Collected last on purpose (file name), so a failure here never hides the
other tests in a run that stops at the first failure.
"""
import numpy as np
import pytest

from paper_2603_27954_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_27954_gb300 import lbm
    return lbm


@pytest.mark.parametrize("case,precision", [("tiny", "fp32"), ("amr2_small", "fp32"), ("amr2_small", "fp16")])
def test_noalloc_mass_matches_lbm_mass_on_two_calls(L, case, precision):
    import torch
    c = W.CASES[case]
    prec = L.LBM_FP16_DEV if precision == "fp16" else L.LBM_FP32
    desc = L.domain_desc(*c["n0"], levels=c["levels"], block=c["block"], bc=c["bc"], u_in=c["u_in"],
                         re_h=c["re_h"], precision=prec)
    dom = L.Domain(desc, tree=L.tree_desc(**c["tree"]), stream=torch.cuda.Stream())
    for steps in (3, 4):  # two calls in a row, on different states
        dom.step(steps)
        m_ref, p_ref = dom.mass()
        m1, p1 = dom.mass_noalloc()
        m2, p2 = dom.mass_noalloc()
        for m, p in ((m1, p1), (m2, p2)):
            assert m == pytest.approx(m_ref, rel=1e-12)
            np.testing.assert_allclose(p, p_ref, rtol=1e-9, atol=1e-9 * m_ref)
    dom.close()
