"""Oracle of the friction force (C_F) and the pressure drag (C_P = C_D - C_F).

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the CPU
baseline of the benchmark, never by the product path.

Sec. 3 integrates the wall shear stress over the tree surface to get the
friction force F_F and takes C_F = F_F / (rho U^2 A_x / 2), C_P = C_D - C_F.
The paper does not say how the shear is read from the lattice; the reading
restated here:

* quadrature points over every primitive's surface, spacing h = 1/2 finest
  cell: cylinder lateral points on N_s x N_t lines (N_s = ceil(L/h), N_t =
  max(8, ceil(2 pi r / h)), at s = (i + 1/2) L / N_s, theta = 2 pi (j + 1/2) /
  N_t, radial direction cos(theta) e1 + sin(theta) e2, e1 = a x z / |a x z| or
  a x x / |a x x| when |a x z| < 0.1, e2 = a x e1); each end cap on N_r =
  ceil(r / h) rings of equal width, ring m with max(4, ceil(2 pi rho_m / h))
  points at rho_m = (m + 1/2) r / N_r; half-spaces n . x <= d: a grid of
  spacing h over the two axes other than n's largest component across the
  finest level's box, projected onto the plane along that axis, area h^2 /
  |n_max|.  Points inside another primitive are dropped;
* the stress of a fluid cell from its populations: sigma' = -(1 - omega1/2)
  dev(sum_i c_i c_i (f_i - f_i^eq)), where the equilibrium's second moment
  is rho u u + rho I / 3;
* at a point, the stress extrapolated linearly to the wall from cell A (the
  cell containing x + delta n for the first delta in {1, 1.5, 2} that is
  fluid) and cell B (containing x + (delta + 1) n, if fluid and at least 1/4
  cell farther along n; else A's stress);
* friction force = sum over points of the tangential traction (sigma' n
  minus (n . sigma' n) n) times the area.
"""
import math

import numpy as np

C27 = np.array([[i % 3 - 1, (i // 3) % 3 - 1, i // 9 - 1] for i in range(27)], dtype=np.float64)
H = 0.5


def _unit(v):
    return v / np.linalg.norm(v)


def cylinder_points(p):
    p0, p1, D = np.asarray(p[0:3], float), np.asarray(p[3:6], float), float(p[6])
    axis = p1 - p0
    L = np.linalg.norm(axis)
    a = axis / L
    r = 0.5 * D
    e1 = np.cross(a, [0.0, 0.0, 1.0])
    if np.linalg.norm(e1) < 0.1:
        e1 = np.cross(a, [1.0, 0.0, 0.0])
    e1 = _unit(e1)
    e2 = np.cross(a, e1)
    pts = []
    ns = max(1, math.ceil(L / H))
    nt = max(8, math.ceil(2 * math.pi * r / H))
    dA = (2 * math.pi * r / nt) * (L / ns)
    for i in range(ns):
        for j in range(nt):
            s, th = (i + 0.5) * L / ns, 2 * math.pi * (j + 0.5) / nt
            n = math.cos(th) * e1 + math.sin(th) * e2
            pts.append((p0 + s * a + r * n, n, dA))
    nr = max(1, math.ceil(r / H))
    for c, sgn in ((p0, -1.0), (p1, 1.0)):
        for m in range(nr):
            rho = (m + 0.5) * r / nr
            nphi = max(4, math.ceil(2 * math.pi * rho / H))
            ring = math.pi * r * r * (2 * m + 1) / (nr * nr)
            for j in range(nphi):
                ph = 2 * math.pi * (j + 0.5) / nphi
                pts.append((c + rho * (math.cos(ph) * e1 + math.sin(ph) * e2), sgn * a, ring / nphi))
    return pts


def plane_points(p, lo, hi):
    n = np.asarray(p[0:3], float)
    nn = np.linalg.norm(n)
    n, dist = n / nn, p[3] / nn
    ax = int(np.argmax(np.abs(n)))
    u, w = (ax + 1) % 3, (ax + 2) % 3
    nu, nw = math.ceil((hi[u] - lo[u]) / H), math.ceil((hi[w] - lo[w]) / H)
    dA = H * H / abs(n[ax])
    pts = []
    for i in range(nu):
        for j in range(nw):
            x = np.zeros(3)
            x[u] = lo[u] + (i + 0.5) * H
            x[w] = lo[w] + (j + 0.5) * H
            x[ax] = (dist - n[u] * x[u] - n[w] * x[w]) / n[ax]
            pts.append((x, n.copy(), dA))
    return pts


def inside(kind, p, x):
    """Closed solid test of one primitive (cylinder with flat caps, half-space)."""
    if kind == 0:
        p0, p1 = np.asarray(p[0:3], float), np.asarray(p[3:6], float)
        L = np.linalg.norm(p1 - p0)
        a = (p1 - p0) / L
        rel = x - p0
        along = rel @ a
        if along < 0 or along > L:
            return False
        perp = rel - along * a
        return perp @ perp <= 0.25 * p[6] * p[6]
    if kind == 1:
        return np.asarray(p[0:3], float) @ x <= p[3]
    lo, hi = np.asarray(p[0:3], float), np.asarray(p[3:6], float)
    return bool(np.all(x >= lo) and np.all(x <= hi))


def samples(items, lo, hi, fluid):
    """Quadrature rows (n x 13): cell A (3), cell B (3, -1e9 if absent),
    normal (3), area, distances of A and B along n, primitive index.
    items: [(kind, params)]; fluid(c): is integer cell c a fluid cell of the
    finest level; lo, hi: that level's box."""
    rows = []
    for k, (kind, p) in enumerate(items):
        pts = cylinder_points(p) if kind == 0 else plane_points(p, lo, hi) if kind == 1 else []
        for x, n, dA in pts:
            if any(inside(kk, pp, x) for o, (kk, pp) in enumerate(items) if o != k):
                continue
            for delta in (1.0, 1.5, 2.0):
                ca = np.floor(x + delta * n).astype(int)
                if not fluid(ca):
                    continue
                da = float((ca + 0.5 - x) @ n)
                cb = np.floor(x + (delta + 1.0) * n).astype(int)
                row = [*ca, -1e9, -1e9, -1e9, *n, dA, da, 0.0, k]
                if fluid(cb) and float((cb + 0.5 - x) @ n) > da + 0.25:
                    row[3:6] = cb
                    row[11] = float((cb + 0.5 - x) @ n)
                rows.append(row)
                break
    return np.array(rows, dtype=np.float64).reshape(-1, 13)


def cell_stress(f, omega1):
    """sigma' for populations f (..., 27)."""
    rho = f.sum(axis=-1)
    j = f @ C27
    Pi = np.einsum("...i,ia,ib->...ab", f, C27, C27)
    neq = Pi - rho[..., None, None] * np.eye(3) / 3.0 - j[..., :, None] * j[..., None, :] / rho[..., None, None]
    dev = neq - np.trace(neq, axis1=-2, axis2=-1)[..., None, None] * np.eye(3) / 3.0
    return -(1.0 - 0.5 * omega1) * dev


def friction(rows, pops, omega1):
    """Per-point friction forces (n x 3).  pops(c) -> the 27 populations of
    integer cell c (rows of c)."""
    fa = pops(rows[:, 0:3].astype(int))
    sa = cell_stress(fa, omega1)
    has_b = rows[:, 3] > -1e8
    sw = sa.copy()
    if has_b.any():
        fb = pops(rows[has_b, 3:6].astype(int))
        sb = cell_stress(fb, omega1)
        w = rows[has_b, 10] / (rows[has_b, 11] - rows[has_b, 10])
        sw[has_b] = sa[has_b] + (sa[has_b] - sb) * w[:, None, None]
    n = rows[:, 6:9]
    t = np.einsum("kab,kb->ka", sw, n)
    tt = t - (t * n).sum(axis=1, keepdims=True) * n
    return tt * rows[:, 9:10]


def per_branch(forces, rows, nprim):
    out = np.zeros((nprim, 3))
    np.add.at(out, rows[:, 12].astype(int), forces)
    return out
