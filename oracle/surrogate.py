"""Oracle for the branch-wise drag model and its learned sectional drag law.

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the CPU
baseline of the benchmark, never by the product path.

Branch-wise model (Sec. 2.4): every branch is a cylinder of length L and
diameter D whose axis makes the angle alpha with the free stream; its drag is
F_d = C_d (rho U^2 / 2) L D sin^3(alpha) (Eq. 2) and the tree estimate is
C_D-est = sum_k F_d,k / (rho U^2 A_x / 2) (Eq. 4), A_x the frontal area.  The
local Reynolds number of a branch is U D / nu.  The paper fits C_d(Re) to
cylinder measurements that are not available here; `cylinder_cd_white` is
the textbook fit C_d = 1 + 10 Re^(-2/3) (F. M. White, Fluid Mechanics, the
cross-flow cylinder correlation for 1 < Re < 2e5), used as the analytic
baseline the learned law is compared with.

Learned law: a fully connected network, standardised inputs, hidden GELU
layers, one linear output, mean-squared-error loss on the standardised
target, Adam (Kingma & Ba 2015).  The forward pass uses the weights rounded
to bfloat16 (round to nearest even), as the GPU does; everything else is
float64 here.  The branch feature table is restated from its definition:
log10 Re_d, generation, D/H, cos alpha (signed), I_u, shielding depth (the
mean number of other branches met upstream along stream-wise lines through
16 axis points), L, D, sin^3 alpha, the shadowed fraction of the branch's
silhouette and a leaf flag.
"""
import math

import numpy as np

from . import cylinders_as_prims, prim_ray


# ---------------------------------------------------------------- branch-wise model

def cylinder_cd_white(re):
    """C_d = 1 + 10 Re^(-2/3) for a circular cylinder in cross-flow."""
    re = np.asarray(re, dtype=np.float64)
    return 1.0 + 10.0 * re ** (-2.0 / 3.0)


def branch_geometry(seg):
    """L, D and cos(alpha) per branch (segments: x0 y0 z0 x1 y1 z1 D gen),
    alpha in [0, pi] measured from the stream-wise x axis to the axis drawn
    from the branch's base to its tip."""
    seg = np.asarray(seg, dtype=np.float64)
    d = seg[:, 3:6] - seg[:, 0:3]
    L = np.linalg.norm(d, axis=1)
    cosa = d[:, 0] / L
    return L, seg[:, 6], cosa


def branch_forces_model(seg, u, nu, cd_of_re, rho=1.0):
    """Eq. 2 for every branch: F_d,k = C_d(Re_k) (rho u^2 / 2) L_k D_k sin^3 alpha_k."""
    L, D, cosa = branch_geometry(seg)
    sin3 = np.sqrt(np.maximum(0.0, 1.0 - cosa * cosa)) ** 3
    return cd_of_re(u * D / nu) * 0.5 * rho * u * u * L * D * sin3


def tree_cd_estimate(forces, u, area, rho=1.0):
    """Eq. 4: C_D-est = sum_k F_d,k / (rho u^2 A_x / 2)."""
    return float(np.sum(forces)) / (0.5 * rho * u * u * area)


def shielding_depth(seg, k, samples=16):
    """Mean over `samples` evenly spaced points of branch k's axis of the number
    of other branches that a stream-wise line through the point enters
    upstream of it (entry x below the point's x)."""
    seg = np.asarray(seg, dtype=np.float64)
    pr = [cylinders_as_prims(seg[m:m + 1]) for m in range(len(seg))]
    a, b = seg[k, 0:3], seg[k, 3:6]
    hits = 0
    for j in range(samples):
        p = a + (j + 0.5) / samples * (b - a)
        start = np.array([0.0, p[1], p[2]])
        for m in range(len(seg)):
            if m == k:
                continue
            t = prim_ray(pr[m], start, (1.0, 0.0, 0.0))
            if np.isfinite(t) and t < p[0]:
                hits += 1
    return hits / samples


def shadowed_fraction(seg, k, axial=16, lateral=(-0.4, -0.2, 0.0, 0.2, 0.4)):
    """Fraction of points spread over branch k's projected silhouette
    (`axial` stations along the axis, `lateral` offsets in diameters along
    the direction normal to the axis and the stream) whose stream-wise line
    enters another branch more than D/2 upstream of the point."""
    seg = np.asarray(seg, dtype=np.float64)
    pr = [cylinders_as_prims(seg[m:m + 1]) for m in range(len(seg))]
    a, b = seg[k, 0:3], seg[k, 3:6]
    ax = (b - a) / np.linalg.norm(b - a)
    w = np.cross(ax, [1.0, 0.0, 0.0])
    w = w / np.linalg.norm(w) if np.linalg.norm(w) > 1e-9 else np.array([0.0, 1.0, 0.0])
    D = seg[k, 6]
    hit = 0
    for j in range(axial):
        for s in lateral:
            p = a + (j + 0.5) / axial * (b - a) + s * D * w
            start = np.array([0.0, p[1], p[2]])
            if any(np.isfinite(t) and t < p[0] - 0.5 * D
                   for t in (prim_ray(pr[m], start, (1.0, 0.0, 0.0)) for m in range(len(seg)) if m != k)):
                hit += 1
    return hit / (axial * len(lateral))


def is_leaf(seg, k):
    """No other branch starts at branch k's tip."""
    seg = np.asarray(seg, dtype=np.float64)
    tip = seg[k, 3:6]
    others = np.delete(seg[:, 0:3], k, axis=0)
    return not np.any(np.abs(others - tip).sum(axis=1) < 1e-9 * (1.0 + np.linalg.norm(seg[k, 3:6] - seg[k, 0:3])))


def branch_features(seg, u, nu, height, i_u=0.0):
    """Rows of 11 per branch: log10 Re_d, generation, D/H, cos alpha, I_u,
    shielding depth, L, D, sin^3 alpha, shadowed fraction, leaf flag."""
    L, D, cosa = branch_geometry(seg)
    sin3 = np.sqrt(np.maximum(0.0, 1.0 - cosa * cosa)) ** 3
    n = len(L)
    rows = np.zeros((n, 11))
    rows[:, 0] = np.log10(u * D / nu)
    rows[:, 1] = np.asarray(seg)[:, 7]
    rows[:, 2] = D / height
    rows[:, 3] = cosa
    rows[:, 4] = i_u
    rows[:, 5] = [shielding_depth(seg, k) for k in range(n)]
    rows[:, 6] = L
    rows[:, 7] = D
    rows[:, 8] = sin3
    rows[:, 9] = [shadowed_fraction(seg, k) for k in range(n)]
    rows[:, 10] = [1.0 if is_leaf(seg, k) else 0.0 for k in range(n)]
    return rows


# ---------------------------------------------------------------- network

def bf16_round(x):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as
    float64.  Works on the float32 bit pattern: add 0x7fff plus the lowest kept
    bit, then clear the 16 dropped bits (finite inputs)."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def _erf(z):
    return np.vectorize(math.erf, otypes=[np.float64])(z)


def layer_shapes(n_in, width, hidden):
    """(out, in) of every layer, input layer first."""
    dims = [n_in] + [width] * hidden + [1]
    return [(dims[l + 1], dims[l]) for l in range(hidden + 1)]


def unpack(p, shapes):
    """Flat vector -> [(W, b)] with W (out x in, row-major) then b per layer."""
    out, o = [], 0
    for no, ni in shapes:
        W = np.asarray(p[o:o + no * ni], dtype=np.float64).reshape(no, ni)
        o += no * ni
        b = np.asarray(p[o:o + no], dtype=np.float64)
        o += no
        out.append((W, b))
    assert o == len(p)
    return out


def init_params(shapes, seed):
    """Uniform(-1/sqrt(in), 1/sqrt(in)) weights and biases (float32 values)."""
    rng = np.random.default_rng(seed)
    parts = []
    for no, ni in shapes:
        s = 1.0 / math.sqrt(ni)
        parts.append(rng.uniform(-s, s, no * ni))
        parts.append(rng.uniform(-s, s, no))
    return np.concatenate(parts).astype(np.float32)


class Norm:
    """Standardisation of inputs and target: (x - mu) / sd."""

    def __init__(self, mu_x, sd_x, mu_y=0.0, sd_y=1.0):
        self.mu_x = np.asarray(mu_x, np.float64)
        self.sd_x = np.asarray(sd_x, np.float64)
        self.mu_y, self.sd_y = float(mu_y), float(sd_y)

    @staticmethod
    def fit(x, y):
        x = np.asarray(x, np.float64)
        sd = x.std(axis=0)
        sd[sd == 0] = 1.0
        return Norm(x.mean(axis=0), sd, float(np.mean(y)), float(np.std(y)) or 1.0)


def forward(p, shapes, x, norm, round_bf16=True):
    """Prediction y (de-standardised) and the per-layer caches (input, Z)."""
    a = (np.asarray(x, np.float64) - norm.mu_x) / norm.sd_x
    caches = []
    layers = unpack(p, shapes)
    for l, (W, b) in enumerate(layers):
        Wq = bf16_round(W) if round_bf16 else W
        z = a @ Wq.T + b
        caches.append((a, z, Wq))
        a = z if l == len(layers) - 1 else gelu(z)
    return a[:, 0] * norm.sd_y + norm.mu_y, caches


def loss_and_grad(p, shapes, x, y, norm, round_bf16=True):
    """Mean squared error of the standardised output and its gradient with
    respect to the flat parameter vector (backpropagation through the
    bfloat16-rounded weights, which a straight-through copy applies to the
    float32 master weights)."""
    yp, caches = forward(p, shapes, x, norm, round_bf16)
    n = len(y)
    d = (yp - norm.mu_y) / norm.sd_y - (np.asarray(y, np.float64) - norm.mu_y) / norm.sd_y
    loss = float(np.mean(d * d))
    dz = (2.0 * d / n)[:, None]
    grads = []
    for l in range(len(caches) - 1, -1, -1):
        a_in, z, Wq = caches[l]
        grads.append((dz.T @ a_in, dz.sum(axis=0)))
        if l == 0:
            break
        da = dz @ Wq
        dz = da * gelu_grad(caches[l - 1][1])
    flat = []
    for gW, gb in reversed(grads):
        flat += [gW.ravel(), gb]
    return loss, np.concatenate(flat)


class Adam:
    """Adam with bias correction: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
    w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)."""

    def __init__(self, n, lr, b1=0.9, b2=0.999, eps=1e-8):
        self.m, self.v = np.zeros(n), np.zeros(n)
        self.t, self.lr, self.b1, self.b2, self.eps = 0, lr, b1, b2, eps

    def step(self, w, g):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return w - self.lr * mh / (np.sqrt(vh) + self.eps)
