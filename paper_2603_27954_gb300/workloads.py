"""Seeded synthetic workloads shaped like the paper's tree-drag runs.

Plain parameter records (no method arithmetic); the test-suite hands the same
records to the CUDA library and to the oracle.  The paper's own runs (Sec.
2.3: a 32H x 16H x 16H box, Re_H from 2.5e3 to 1.2e5, finest cells of H/1024
to H/2048) are far larger; these stand in for them with trees from the
parametric L-system of Eq. (1), seeded branch azimuths and lattice inflow
speed 0.05.
"""

# tree of Eq. (1) in the "azimuth" form: each child tilted by alpha from its
# parent and turned about the parent's axis by a seeded azimuth
TINY_TREE = dict(n=2, children=2, s0=12.0, w0=2.0, r=(0.6,), dfac=(0.7,), alpha_deg=(30.0,),
                 azimuth_mode=1, seed=0, trunk_cells=12.0)

CASES = {
    # single-level 64x32x32, trunk 12 cells / diameter 2, two children, Re_H = 100
    "tiny": dict(n0=(64, 32, 32), levels=1, block=16, bc=("inout", "slip", "slip"), u_in=0.05, re_h=100.0,
                 steps=1000, tree=TINY_TREE),
    # two levels, coarse 256x128x128 in 16^3 blocks, 3 generations of 3 children,
    # trunk 64 finest cells (diameter 0.3 of its length, as w0/s0 of Table 1), Re_H = 2.5e3
    "amr2": dict(n0=(256, 128, 128), levels=2, block=16, bc=("inout", "inflow", "inflow"), u_in=0.05,
                 re_h=2500.0, steps=10000,
                 tree=dict(n=4, children=3, s0=64.0, w0=19.2, r=(0.6,), dfac=(0.6,), alpha_deg=(35.0,),
                           azimuth_mode=1, seed=1, trunk_cells=64.0)),
    # four levels, coarse 512x256x256 in 16^3 blocks, 4 generations of 3 children,
    # trunk 360 finest cells (diameter 0.3 of its length), Re_H = 1.2e5: about
    # 6e8 active cells summed over the levels
    "amr4": dict(n0=(512, 256, 256), levels=4, block=16, bc=("inout", "inflow", "inflow"), u_in=0.05,
                 re_h=1.2e5, steps=20,
                 tree=dict(n=5, children=3, s0=360.0, w0=108.0, r=(0.6,), dfac=(0.6,), alpha_deg=(35.0,),
                           azimuth_mode=1, seed=2, trunk_cells=360.0)),
    # the four-level case scaled down by 4 per axis (coarse 128x64x64, 8^3 blocks), sized for the oracle
    "amr4_quarter": dict(n0=(128, 64, 64), levels=4, block=8, bc=("inout", "inflow", "inflow"), u_in=0.05,
                         re_h=1.2e5, steps=2,
                         tree=dict(n=5, children=3, s0=90.0, w0=27.0, r=(0.6,), dfac=(0.6,), alpha_deg=(35.0,),
                                   azimuth_mode=1, seed=2, trunk_cells=90.0)),
    # three levels, coarse 48x32x32 in 8^3 blocks, 2 generations of 3 children,
    # trunk 16 finest cells: the smallest case with two nested interfaces
    "amr3_small": dict(n0=(48, 32, 32), levels=3, block=8, bc=("inout", "inflow", "inflow"), u_in=0.05,
                       re_h=800.0, steps=20,
                       tree=dict(n=3, children=3, s0=16.0, w0=4.8, r=(0.6,), dfac=(0.6,), alpha_deg=(35.0,),
                                 azimuth_mode=1, seed=4, trunk_cells=16.0)),
    # the two-level case scaled down by 4 per axis for the oracle: the same tree (n = 4 rewritings,
    # 3 children, 40 branches, seed 1) with a trunk of 16 finest cells, Re_H = 2.5e3, 8^3 blocks;
    # coarse 64x32x36: at 64x32x32 the tree's box with its 25 % margin, rounded out to whole
    # 8^3 finest blocks, leaves no room for the two parent cells the interface needs in z
    "amr2_quarter": dict(n0=(64, 32, 36), levels=2, block=8, bc=("inout", "inflow", "inflow"), u_in=0.05,
                         re_h=2500.0, steps=300,
                         tree=dict(n=4, children=3, s0=16.0, w0=4.8, r=(0.6,), dfac=(0.6,), alpha_deg=(35.0,),
                                   azimuth_mode=1, seed=1, trunk_cells=16.0)),
    # a small two-level tree case for element-wise oracle tests: coarse 64x48x48 in 8^3 blocks,
    # n = 3 rewritings (13 branches), trunk 16 finest cells, Re_H = 400
    "amr2_small": dict(n0=(64, 48, 48), levels=2, block=8, bc=("inout", "inflow", "inflow"), u_in=0.05,
                       re_h=400.0, steps=100,
                       tree=dict(n=3, children=3, s0=16.0, w0=4.8, r=(0.6,), dfac=(0.6,), alpha_deg=(35.0,),
                                 azimuth_mode=1, seed=1, trunk_cells=16.0)),
}


def tgv_fields(lo, hi, scale, n, amplitude, mean=(0.0, 0.0, 0.0)):
    """Taylor-Green initial field (rho, u) on cells [lo, hi) of a level whose
    cells are 1/scale of a level-0 cell, wavelength n level-0 cells."""
    import numpy as np
    k = 2 * np.pi / n
    z, y, x = np.meshgrid(*(np.arange(lo[a], hi[a]) + 0.5 for a in (2, 1, 0)), indexing="ij")
    x = x / scale - 0.5
    y = y / scale - 0.5
    ux = mean[0] + amplitude * np.sin(k * x) * np.cos(k * y)
    uy = mean[1] - amplitude * np.cos(k * x) * np.sin(k * y)
    uz = mean[2] + 0 * x
    rho = 1 - 0.75 * amplitude ** 2 * (np.cos(2 * k * x) + np.cos(2 * k * y))
    return rho, np.stack([ux, uy, uz], -1)


# ---------------------------------------------------------------- batched form
# 16 independent cases: trees of 1-4 child generations (3 children, ratios
# 0.6 / 0.6, 35 deg, seeded azimuths) x Re_H in {2.5e3, 1e4, 4e4, 1.2e5}; the
# tree size sets the domain (64 to 4096 coarse blocks of 16^3) and the levels
# (2 or 3); the cases with Re_H = 1e4 and 1.2e5 have turbulent inflow with
# I_u = 8 % (256 random Fourier modes, integral length = the tree height).
BATCH_DOMAINS = {
    1: dict(n0=(64, 64, 64), levels=2, trunk=16.0),
    2: dict(n0=(192, 96, 96), levels=2, trunk=48.0),
    3: dict(n0=(256, 128, 128), levels=3, trunk=64.0),
    4: dict(n0=(512, 256, 128), levels=3, trunk=96.0),
}
BATCH_RE = (2.5e3, 1e4, 4e4, 1.2e5)


def batch_cases():
    """The 16 case records of the batched form, in (generations, Re_H) order."""
    out = []
    for g, dom in BATCH_DOMAINS.items():
        for k, re in enumerate(BATCH_RE):
            t = dom["trunk"]
            out.append(dict(n0=dom["n0"], levels=dom["levels"], block=16, bc=("inout", "inflow", "inflow"),
                            u_in=0.05, re_h=re, i_u=0.08 if k % 2 else 0.0, seed=100 + 4 * g + k,
                            tree=dict(n=g + 1, children=3, s0=t, w0=0.3 * t, r=(0.6,), dfac=(0.6,),
                                      alpha_deg=(35.0,), azimuth_mode=1, seed=4 + g, trunk_cells=t)))
    return out


# ---------------------------------------------------------------- learned form
# Trees shaped like the three tree workloads - family 1: n = 2 rewritings x 2
# children, length / diameter ratios 0.6 / 0.7, 30 deg (the tiny case's tree);
# family 2: n = 4 x 3 children, 0.6 / 0.6, 35 deg (the two-level case's tree at
# quarter scale); family 3: n = 5 x 3 children, 0.6 / 0.6, 35 deg (the
# four-level case's tree, trunk 32 finest cells) - with seeded azimuths,
# Re_H log-uniform in [2.5e3, 1.2e5] and every second case with 8 %
# random-Fourier-mode inflow.  Domains keep the smallest twig at about one
# finest cell or more.  Every case runs `transient` flow-through times H / U
# from the impulsive start, then averages its forces over `average` more.
LEARNED_FAMILIES = {
    1: dict(n0=(64, 32, 32), levels=1, block=16, bc=("inout", "slip", "slip"), u_in=0.05,
            tree=dict(n=2, children=2, s0=12.0, w0=2.0, r=(0.6,), dfac=(0.7,), alpha_deg=(30.0,), azimuth_mode=1,
                      trunk_cells=12.0)),
    2: dict(n0=(64, 32, 36), levels=2, block=8, bc=("inout", "inflow", "inflow"), u_in=0.05,
            tree=dict(n=4, children=3, s0=16.0, w0=4.8, r=(0.6,), dfac=(0.6,), alpha_deg=(35.0,), azimuth_mode=1,
                      trunk_cells=16.0)),
    3: dict(n0=(128, 64, 72), levels=2, block=8, bc=("inout", "inflow", "inflow"), u_in=0.05,
            tree=dict(n=5, children=3, s0=32.0, w0=9.6, r=(0.6,), dfac=(0.6,), alpha_deg=(35.0,), azimuth_mode=1,
                      trunk_cells=32.0)),
}
LEARNED_RE = (2.5e3, 1.2e5)
LEARNED_PROTOCOL = dict(transient=2, average=3)
LEARNED_I_U = 0.08
# training cases per family of the full data set (about 1.9e5 branch samples)
LEARNED_COUNTS = {1: 2048, 2: 3072, 3: 512}


def learned_cases(family, count, seed):
    """`count` seeded training records of one family: tree azimuth seed,
    Re_H (log-uniform over LEARNED_RE), inflow turbulence and its seed."""
    import numpy as np
    rng = np.random.default_rng(seed * 1000 + family)
    lo, hi = np.log(LEARNED_RE[0]), np.log(LEARNED_RE[1])
    out = []
    for k in range(count):
        out.append(dict(family=family, tree_seed=int(rng.integers(0, 1 << 30)), re_h=float(np.exp(rng.uniform(lo, hi))),
                        i_u=LEARNED_I_U if k % 2 else 0.0, inflow_seed=int(rng.integers(0, 1 << 30))))
    return out


# the evaluation: 8 held-out (geometry, Re_H) points across the range, tree seeds
# outside the training draws' range, uniform inflow (with 8 % turbulent inflow
# the C_D of one averaging window scatters by 7-13 % from window to window -
# eddies as large as the tree - so such a point cannot test an estimate at
# the per-cent level; turbulent held-out trees are reported apart)
LEARNED_JUDGES = [
    dict(family=1, tree_seed=(1 << 30) + 1, re_h=3.0e3, i_u=0.0, inflow_seed=11),
    dict(family=1, tree_seed=(1 << 30) + 2, re_h=6.0e4, i_u=0.0, inflow_seed=12),
    dict(family=2, tree_seed=(1 << 30) + 3, re_h=2.5e3, i_u=0.0, inflow_seed=13),
    dict(family=2, tree_seed=(1 << 30) + 4, re_h=1.5e4, i_u=0.0, inflow_seed=14),
    dict(family=2, tree_seed=(1 << 30) + 5, re_h=1.2e5, i_u=0.0, inflow_seed=15),
    dict(family=3, tree_seed=(1 << 30) + 6, re_h=5.0e3, i_u=0.0, inflow_seed=16),
    dict(family=3, tree_seed=(1 << 30) + 7, re_h=4.0e4, i_u=0.0, inflow_seed=17),
    dict(family=3, tree_seed=(1 << 30) + 8, re_h=1.0e5, i_u=0.0, inflow_seed=18),
]
