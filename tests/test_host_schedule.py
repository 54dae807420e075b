"""Schedule validation on the host (no GPU): every collide-variant pair a
domain accepts, and the ones it must refuse (staged and TMA kernels only
for FP32 in 16^3 blocks, the 7- and 8-CTA budgets of the paired odd step
only in 16^3 blocks)."""
import numpy as np
import pytest

from paper_2603_27954_gb300 import lbm as L


def domain(precision, block=16):
    h = L.lbm_create_domain(L.domain_desc(32, 32, 32, block=block, bc=("periodic",) * 3, nu_finest=0.02,
                                          precision=precision))
    L.lbm_set_geometry_prims(h, [], np.zeros((0, 8)))
    return h


@pytest.mark.parametrize("precision,block,odd,even,ok", [
    (L.LBM_FP32, 16, 0, 0, True), (L.LBM_FP32, 16, 1, 1, True), (L.LBM_FP32, 16, 2, 0, True),
    (L.LBM_FP32, 16, 0, 2, True), (L.LBM_FP32, 8, 1, 0, False), (L.LBM_FP32, 8, 0, 1, False),
    (L.LBM_FP16_DEV, 16, 0, 2, True), (L.LBM_FP16_DEV, 8, 2, 2, True), (L.LBM_FP16_DEV, 16, 1, 0, False),
    (L.LBM_FP16_DEV, 16, 0, 1, False), (L.LBM_FP32, 16, 3, 0, True), (L.LBM_FP32, 16, 0, 3, False),
    (L.LBM_FP32, 8, 3, 2, True), (L.LBM_FP32, 16, 6, 0, False),
    (L.LBM_FP16_DEV, 16, 3, 2, True), (L.LBM_FP16_DEV, 8, 3, 0, True), (L.LBM_FP16_DEV, 16, 6, 2, False),
    # the pair kernel budgeted for 7 or 8 resident CTAs: 16^3 blocks only
    (L.LBM_FP32, 16, 4, 0, True), (L.LBM_FP16_DEV, 16, 5, 2, True), (L.LBM_FP32, 8, 4, 0, False),
    (L.LBM_FP16_DEV, 8, 5, 2, False),
])
def test_schedule_validation(precision, block, odd, even, ok):
    h = domain(precision, block)
    if ok:
        L.lbm_set_schedule(h, 0, odd, even)
        s = L.lbm_get_schedule(h)
        assert (s.odd_variant, s.even_variant) == (odd, even)
    else:
        with pytest.raises(L.LbmError) as e:
            L.lbm_set_schedule(h, 0, odd, even)
        assert e.value.code == L.LBM_EINVAL
    L.lbm_destroy(h)


def test_default_schedules():
    for precision, odd, even in ((L.LBM_FP32, 0, 0), (L.LBM_FP16_DEV, 3, 2)):
        h = domain(precision)
        s = L.lbm_get_schedule(h)
        assert (s.odd_variant, s.even_variant) == (odd, even)
        L.lbm_destroy(h)


@pytest.mark.parametrize("block,split,ok", [
    (16, 1, True), (16, 2, True), (16, 4, True), (16, 8, True), (16, 16, True), (16, 3, False), (16, 32, False),
    (16, -2, False), (8, 8, True), (8, 16, False),
])
def test_z_split_validation(block, split, ok):
    for precision in (L.LBM_FP32, L.LBM_FP16_DEV):
        h = domain(precision, block)
        even = 2 if precision == L.LBM_FP16_DEV else 0
        if ok:
            L.lbm_set_schedule(h, 0, 0, even, split, split)
            s = L.lbm_get_schedule(h)
            assert (s.z_split_even, s.z_split_odd) == (split, split)
        else:
            with pytest.raises(L.LbmError) as e:
                L.lbm_set_schedule(h, 0, 0, even, split, 1)
            assert e.value.code == L.LBM_EINVAL
            with pytest.raises(L.LbmError):
                L.lbm_set_schedule(h, 0, 0, even, 1, split)
        L.lbm_destroy(h)


def test_z_split_defaults_to_automatic():
    for precision, even in ((L.LBM_FP32, 0), (L.LBM_FP16_DEV, 2)):
        for block in (8, 16):
            h = domain(precision, block)
            d = L.lbm_get_schedule(h)
            assert (d.z_split_even, d.z_split_odd) == (0, 0)
            L.lbm_set_schedule(h, 0, 0, even, 2, 4)
            s = L.lbm_get_schedule(h)
            assert (s.z_split_even, s.z_split_odd) == (2, 4)
            L.lbm_set_schedule(h, 0, 0, even, 0, 0)
            s = L.lbm_get_schedule(h)
            assert (s.z_split_even, s.z_split_odd) == (0, 0)
            L.lbm_destroy(h)


def test_overlap_check_finds_independent_and_conflicting_kernels():
    """The host check behind the parallel branches: a cylinder clear of the
    domain faces leaves the faces free to overlap the walls; one that crosses
    the slip walls puts cut links next to face entries and keeps them serial;
    refined trees let the finest walls overlap the interface transfer."""
    from paper_2603_27954_gb300 import workloads as W

    def single(seg):
        h = L.lbm_create_domain(L.domain_desc(32, 32, 32, block=16, bc=("inout", "slip", "slip"), u_in=0.05,
                                              nu_finest=0.02))
        L.lbm_set_geometry_prims(h, [0], np.array([seg]))
        r = L.lbm_get_overlap(h)
        L.lbm_destroy(h)
        return r

    assert single([16.0, 16.0, 6.0, 16.0, 16.0, 26.0, 6.0, 0.0]) == (True, 0)
    assert single([16.0, -2.0, 16.0, 16.0, 34.0, 16.0, 6.0, 0.0]) == (False, 0)
    for case, bits in (("amr2_small", 2), ("amr3_small", 4)):
        c = W.CASES[case]
        h = L.lbm_create_domain(L.domain_desc(*c["n0"], levels=c["levels"], block=c["block"], bc=c["bc"],
                                              u_in=c["u_in"], re_h=c["re_h"]))
        L.lbm_set_geometry(h, L.tree_desc(**c["tree"]))
        assert L.lbm_get_overlap(h) == (True, bits)
        L.lbm_destroy(h)


def test_fp64_form_descriptor_rules():
    """The FP64 storage form: twice the FP32 population bytes, one collide
    kernel per parity (only the direct / column-pointer variant names are
    accepted), no turbulent inflow."""
    from paper_2603_27954_gb300 import lbm as L
    from paper_2603_27954_gb300 import workloads as W
    c = W.CASES["tiny"]
    sizes = {}
    for prec in (L.LBM_FP64, L.LBM_FP32):
        d = L.domain_desc(*c["n0"], levels=1, block=16, bc=c["bc"], u_in=0.05, re_h=100.0, precision=prec)
        h = L.lbm_create_domain(d)
        L.lbm_set_geometry(h, L.tree_desc(**c["tree"]))
        sizes[prec] = L.lbm_memory_breakdown(h)[0]
        if prec == L.LBM_FP64:
            L.lbm_set_schedule(h, 0, 2, 0)
            for odd, even in ((3, 0), (0, 2), (6, 0)):
                with pytest.raises(L.LbmError):
                    L.lbm_set_schedule(h, 0, odd, even)
        L.lbm_destroy(h)
    assert sizes[L.LBM_FP64] == 2 * sizes[L.LBM_FP32]
    d = L.domain_desc(*c["n0"], levels=1, block=16, bc=c["bc"], u_in=0.05, re_h=100.0, i_u=0.08,
                      precision=L.LBM_FP64)
    with pytest.raises(L.LbmError):
        L.lbm_create_domain(d)


def test_overlap_features_mask():
    """The reorderings switch on and off one by one (default: branches,
    levels and transfers); unknown bits are refused."""
    h = domain(L.LBM_FP32)
    assert L.lbm_get_overlap_features(h) == L.LBM_OVL_BRANCHES | L.LBM_OVL_LEVELS | L.LBM_OVL_TRANSFERS
    for m in (0, L.LBM_OVL_BRANCHES, L.LBM_OVL_DEFER | L.LBM_OVL_LEVELS, L.LBM_OVL_ALL):
        L.lbm_set_overlap_features(h, m)
        assert L.lbm_get_overlap_features(h) == m
    for bad in (32, -1, 64 | 1):
        with pytest.raises(L.LbmError) as e:
            L.lbm_set_overlap_features(h, bad)
        assert e.value.code == L.LBM_EINVAL
    L.lbm_destroy(h)


def test_learned_form_branch_weights():
    """Each branch's training weight is its share of Eq. 4's sum, L_k D_k /
    A_x of its own tree, normalised over all branches."""
    from paper_2603_27954_gb300 import surrogate as SG
    rows = np.zeros((3, 12))
    rows[:, 6] = [10.0, 5.0, 2.0]
    rows[:, 7] = [3.0, 2.0, 1.0]
    a = SG.Sample(rows, np.ones(3), 100.0, 1.0, {})
    b = SG.Sample(rows[:2], np.ones(2), 50.0, 1.0, {})
    w = SG.sample_weights([a, b])
    raw = np.array([30 / 100, 10 / 100, 2 / 100, 30 / 50, 10 / 50])
    np.testing.assert_allclose(w, raw / raw.sum(), rtol=1e-15)


def test_drag_decode_on_the_host():
    """lbm_drag_decode turns the 8 force accumulators into lbm_drag's
    outputs: the last force, the mean over the counted steps, C_D by Eq. 7
    with the tree's frontal area; a nonzero status word is LBM_ETIMEOUT."""
    from paper_2603_27954_gb300 import workloads as W
    c = W.CASES["tiny"]
    h = L.lbm_create_domain(L.domain_desc(*c["n0"], levels=1, block=16, bc=c["bc"], u_in=c["u_in"],
                                          re_h=c["re_h"]))
    L.lbm_set_geometry(h, L.tree_desc(**c["tree"]))
    area = L.lbm_geometry_info(h)["A_x"]
    acc = np.array([0.5, -0.1, 0.2, 3.0, 0.6, -0.9, 3.0, 0.0])
    last, mean, cd = L.lbm_drag_decode(h, acc)
    np.testing.assert_array_equal(last, acc[:3])
    np.testing.assert_allclose(mean, acc[3:6] / 3.0, rtol=1e-15)
    assert cd == pytest.approx(0.5 / (0.5 * c["u_in"] ** 2 * area), rel=1e-15)
    acc[7] = 1.0
    with pytest.raises(L.LbmError) as e:
        L.lbm_drag_decode(h, acc)
    assert e.value.code == L.LBM_ETIMEOUT
    L.lbm_destroy(h)


def test_host_allocation_failure_returns_a_status():
    """A host allocation that fails inside the library - here the mesh build
    of a 2048^3 domain in a process whose address space is capped at 8 GB -
    comes back as LBM_ENOMEM with a message, and the caller carries on: no
    C++ exception crosses the C-ABI (one would end the calling process with
    std::terminate)."""
    import os
    import subprocess
    import sys
    import textwrap
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = textwrap.dedent("""
        import resource, sys
        resource.setrlimit(resource.RLIMIT_AS, (8 << 30, 8 << 30))
        sys.path.insert(0, %r)
        import numpy as np
        from paper_2603_27954_gb300 import lbm as L
        h = L.lbm_create_domain(L.domain_desc(2048, 2048, 2048, bc=("inout", "slip", "slip"), nu_finest=0.01))
        try:
            L.lbm_set_geometry_prims(h, [], np.zeros((0, 8)))
        except L.LbmError as e:
            print("status", e.code)
        L.lbm_destroy(h)
        h = L.lbm_create_domain(L.domain_desc(32, 32, 32, bc=("inout", "slip", "slip"), nu_finest=0.01))
        L.lbm_set_geometry_prims(h, [], np.zeros((0, 8)))
        L.lbm_destroy(h)
        print("alive")
    """ % root)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "status %d" % L.LBM_ENOMEM in r.stdout and "alive" in r.stdout, r.stdout
