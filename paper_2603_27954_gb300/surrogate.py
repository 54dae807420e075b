"""Learned sectional drag for the branch-wise model (Sec. 2.4).

The paper estimates a tree's drag by summing Eq. 3 over its branches with a
cylinder law C_d(Re) fitted to measurements (Eq. 5).  Here the per-branch
law is learned from the LBM itself: every simulated tree yields, per branch,
the features of lbm_branch_table and the measured sectional coefficient
c_k = F_x,k / (rho U^2 L_k D_k / 2) (per-branch momentum-exchange forces,
lbm_get_branch_forces).  A 6-input network (log10 Re_d, D/H, cos alpha,
shielding depth, shadowed fraction, leaf flag) trained by the library's
kernels predicts c_k, and Eq. 5 turns the predictions into C_D-est.  The same
pipeline learns the sectional friction coefficient from the per-branch wall
shear (lbm_get_friction_mean) for Eq. 4 and C_F-est; C_P-est = C_D-est -
C_F-est (Eq. 6).

Everything numeric runs in liblbm (simulation, feature table, network
kernels, Eq. 5); this module only sequences the calls.
"""
import numpy as np

from . import lbm as L
from . import workloads as W

# branch-table columns used as network inputs: log10 Re_d, D/H, cos alpha,
# shielding depth, shadowed fraction, leaf flag
FEATURES = (0, 2, 3, 5, 9, 10)
# the six inputs the learned-form workload names: log10 Re_d, generation,
# D/H, cos alpha, I_u, shielding depth
FEATURES_NAMED = (0, 1, 2, 3, 4, 5)


class Sample:
    """One simulated tree: its branch table, measured sectional drag and
    friction coefficients, frontal area, measured C_D and C_F."""

    def __init__(self, rows, c, area, cd, cf=None, c_f=None):
        self.rows, self.c, self.area, self.cd = rows, c, area, cd
        self.cf, self.c_f = cf, c_f


def simulate(case, stream=None, domain=None, steps=None, average=None):
    """Run one (tree, Re_H) record to a time-averaged state and return its
    Sample.  Forces are averaged over the last `average` of `steps` updates."""
    dom_kw = dict(W.SURROGATE_DOMAIN, **(domain or {}))
    steps = steps or W.SURROGATE_STEPS["steps"]
    average = average or W.SURROGATE_STEPS["average"]
    desc = L.domain_desc(*dom_kw["n0"], levels=dom_kw["levels"], block=dom_kw["block"], bc=dom_kw["bc"],
                         u_in=dom_kw["u_in"], re_h=case["re_h"])
    dom = L.Domain(desc, tree=L.tree_desc(**case["tree"]), stream=stream)
    try:
        dom.set_branch_forces(True)
        dom.set_friction_mean(True)
        dom.step(steps - average)
        dom.reset_force()
        dom.step(average)
        g = dom.geometry_info()
        rows = L.lbm_branch_table(dom.h)
        fb, _ = dom.get_branch_forces(len(rows))
        _, mean, _ = dom.drag()
        fmean, frows, _ = dom.get_friction_mean(len(rows))
    finally:
        dom.close()
    u = dom_kw["u_in"]
    q = 0.5 * u * u
    ld = q * rows[:, 6] * rows[:, 7]
    return Sample(rows, fb[:, 0] / ld, g["A_x"], mean[0] / (q * g["A_x"]), fmean[0] / (q * g["A_x"]), frows[:, 0] / ld)


def dataset(samples, features=FEATURES, target="c"):
    """Stack the branch rows of several samples: inputs (float32, n x 6) and
    targets (float32, n): sectional drag "c" or sectional friction "c_f"."""
    x = np.concatenate([s.rows[:, list(features)] for s in samples]).astype(np.float32)
    y = np.concatenate([getattr(s, target) for s in samples]).astype(np.float32)
    return x, y


def standardisation(x, y):
    """Means and spreads of inputs and target (a constant input gets spread 1)."""
    sd = x.std(axis=0).astype(np.float64)
    sd[sd == 0] = 1.0
    return x.mean(axis=0), sd, float(y.mean()), float(y.std()) or 1.0


def train(x, y, width=128, hidden=3, steps=2000, batch=256, lr=3e-4, seed=0, stream=None):
    """Fit the network to (x, y) with mini-batch Adam; returns the Mlp."""
    import torch
    n = len(y)
    rng = np.random.default_rng(seed)
    net = L.Mlp(x.shape[1], width, hidden, max_batch=max(n, batch), stream=stream)
    shapes = [(width, x.shape[1])] + [(width, width)] * (hidden - 1) + [(1, width)]
    params = []
    for no, ni in shapes:
        s = 1.0 / np.sqrt(ni)
        params += [rng.uniform(-s, s, no * ni), rng.uniform(-s, s, no)]
    net.set_params(np.concatenate(params).astype(np.float32))
    net.set_normalization(*standardisation(x, y))
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = torch.from_numpy(np.ascontiguousarray(y)).cuda()
    b = min(batch, n)
    per_epoch = max(1, n // b)
    done = 0
    while done < steps:
        perm = torch.from_numpy(rng.permutation(n).astype(np.int32)).cuda()
        for k in range(per_epoch):
            if done == steps:
                break
            net.train_step(xd, yd, perm[k * b:(k + 1) * b], lr=lr)
            done += 1
    return net


def train_ensemble(x, y, members=4, seed=0, **kw):
    """`members` networks trained from different seeded initialisations and
    mini-batch orders; predict() averages them."""
    return [train(x, y, seed=seed + k, **kw) for k in range(members)]


def predict(net, rows, features=FEATURES):
    """Sectional coefficients predicted for the branches of a branch table
    (the mean over the members when `net` is a list)."""
    import torch
    x = torch.from_numpy(np.ascontiguousarray(rows[:, list(features)], dtype=np.float32)).cuda()
    nets = net if isinstance(net, (list, tuple)) else [net]
    return np.mean([m.forward(x).cpu().numpy().astype(np.float64) for m in nets], axis=0)


def estimate(rows, area, c=None):
    """Eq. 5: C_D-est from sectional coefficients c (None: the cylinder law)."""
    return L.lbm_branch_drag_estimate(rows, area, c)[0]
