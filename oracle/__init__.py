"""Plain FP64 CPU oracle of the cumulant-LBM / refinement / drag path.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library: its own L-system, geometry,
collision, streaming, bounce-back, force and refinement, written plainly in
C (``lsys.c``, ``collide.c``, ``lbm.c``) and driven from here through ctypes.

Paper references (Tokiwa, Yin & Onishi, "Drag Crisis in Fractal Trees
Revealed by Simulation and Theory"): Sec. 2.1 Eq. (1) and Tables 1-2 for the
tree, Sec. 2.2 for the D3Q27 cumulant LBM with octree refinement,
interpolated bounce-back and momentum-exchange force, Sec. 2.3 for the set-up
and Sec. 3 Eq. (7) for C_D.
"""
import ctypes as C
import math
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(path)
        _declare(_lib)
    return _lib


class Tree(C.Structure):
    _fields_ = [("n", C.c_int), ("children", C.c_int), ("s0", C.c_double), ("w0", C.c_double),
                ("min_len", C.c_double), ("r", C.c_double * 4), ("dfac", C.c_double * 4),
                ("alpha_deg", C.c_double * 4), ("phi_deg", C.c_double * 4),
                ("azimuth_mode", C.c_int), ("seed", C.c_uint64)]


class Prim(C.Structure):
    _fields_ = [("kind", C.c_int), ("p", C.c_double * 8)]


class Rates(C.Structure):
    _fields_ = [("omega1", C.c_double), ("omega2", C.c_double), ("omega_hi", C.c_double * 8),
                ("galilean", C.c_int)]


class Desc(C.Structure):
    _fields_ = [("levels", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("box", (C.c_int * 6) * 6), ("bc", C.c_int * 3), ("u_in", C.c_double),
                ("nu0", C.c_double), ("omega2", C.c_double), ("omega_hi", C.c_double * 8),
                ("galilean", C.c_int), ("force", C.c_double * 3)]


BC_PERIODIC, BC_INOUT, BC_SLIP, BC_INFLOW = 0, 1, 2, 3
_BC_NAMES = {"periodic": 0, "inout": 1, "slip": 2, "inflow": 3}

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_bp = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def _declare(L):
    L.orc_lsystem.argtypes = [C.POINTER(Tree), _dp, C.c_int]
    L.orc_lsystem.restype = C.c_int
    L.orc_tree_bbox.argtypes = [_dp, C.c_int, _dp, _dp]
    L.orc_tree_height.argtypes = [_dp, C.c_int]
    L.orc_tree_height.restype = C.c_double
    L.orc_tree_com.argtypes = [_dp, C.c_int, _dp]
    L.orc_transform.argtypes = [_dp, C.c_int, C.c_double, _dp]
    L.orc_prim_inside.argtypes = [C.POINTER(Prim), C.c_int, _dp]
    L.orc_prim_inside.restype = C.c_int
    L.orc_prim_ray.argtypes = [C.POINTER(Prim), C.c_int, _dp, _dp]
    L.orc_prim_ray.restype = C.c_double
    L.orc_frontal_area.argtypes = [_dp, C.c_int, C.c_double]
    L.orc_frontal_area.restype = C.c_double
    L.orc_equilibrium.argtypes = [C.c_double, _dp, _dp]
    L.orc_cumulants.argtypes = [_dp, _dp]
    L.orc_collide.argtypes = [_dp, _dp, C.POINTER(Rates), C.c_void_p]
    L.orc_create.argtypes = [C.POINTER(Desc)]
    L.orc_create.restype = C.c_void_p
    L.orc_destroy.argtypes = [C.c_void_p]
    L.orc_set_prims.argtypes = [C.c_void_p, C.POINTER(Prim), C.c_int]
    L.orc_set_prims.restype = C.c_int
    L.orc_init_uniform.argtypes = [C.c_void_p, C.c_double, _dp]
    L.orc_init_field.argtypes = [C.c_void_p, C.c_int, _dp, _dp]
    L.orc_init_field.restype = C.c_int
    L.orc_step.argtypes = [C.c_void_p, C.c_int]
    L.orc_level_box.argtypes = [C.c_void_p, C.c_int, _ip, _ip]
    L.orc_get_f.argtypes = [C.c_void_p, C.c_int, _dp]
    L.orc_get_macro.argtypes = [C.c_void_p, C.c_int, _dp, _dp]
    L.orc_level_links.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
    L.orc_level_links.restype = C.c_int
    L.orc_level_link_segs.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int]
    L.orc_level_link_segs.restype = C.c_int
    L.orc_force.argtypes = [C.c_void_p, _dp, _dp, C.POINTER(C.c_long)]
    L.orc_mass.argtypes = [C.c_void_p, C.POINTER(C.c_double), _dp]
    L.orc_cell_type.argtypes = [C.c_void_p, C.c_int, _bp]
    L.orc_cell_type.restype = C.c_int
    L.orc_branch_forces.argtypes = [C.c_void_p, _dp, C.c_int]
    L.orc_branch_forces.restype = C.c_int
    L.orc_set_turbulence.argtypes = [C.c_void_p, _dp, C.c_int, C.c_double]
    L.orc_set_turbulence.restype = C.c_int
    L.orc_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
    L.orc_splitmix64.restype = C.c_uint64
    L.orc_set_threads.argtypes = [C.c_int]
    L.orc_set_threads.restype = C.c_int


# ---------------------------------------------------------------- tree (Sec. 2.1)

def make_tree(n, children=2, s0=100.0, w0=30.0, r=(0.8, 0.8), dfac=None, q=0.5, e=0.5,
              alpha_deg=(30.0, -30.0), phi_deg=(137.0, 137.0), azimuth_mode=0, seed=0,
              min_len=0.02):
    """Parameters of rule p1 (Eq. 1).  ``dfac`` defaults to (q^e, (1-q)^e)."""
    t = Tree()
    t.n, t.children, t.s0, t.w0, t.min_len = n, children, s0, w0, min_len
    if dfac is None:
        dfac = (q ** e, (1.0 - q) ** e)
    for k in range(children):
        t.r[k] = r[k % len(r)]
        t.dfac[k] = dfac[k % len(dfac)]
        t.alpha_deg[k] = alpha_deg[k % len(alpha_deg)]
        t.phi_deg[k] = phi_deg[k % len(phi_deg)]
    t.azimuth_mode, t.seed = azimuth_mode, seed
    return t


def lsystem(tree):
    """Segments (rows x0 y0 z0 x1 y1 z1 D gen) of the tree in turtle units."""
    cap = 1
    for g in range(tree.n):
        cap += tree.children ** (g + 1)
    seg = np.zeros((cap, 8))
    n = lib().orc_lsystem(C.byref(tree), seg, cap)
    if n < 0:
        raise ValueError("bad tree")
    return seg[:n].copy()


def tree_bbox(seg):
    lo, hi = np.zeros(3), np.zeros(3)
    lib().orc_tree_bbox(np.ascontiguousarray(seg), len(seg), lo, hi)
    return lo, hi


def tree_height(seg):
    return lib().orc_tree_height(np.ascontiguousarray(seg), len(seg))


def tree_com(seg):
    c = np.zeros(3)
    lib().orc_tree_com(np.ascontiguousarray(seg), len(seg), c)
    return c


def transform(seg, scale, shift):
    s = np.ascontiguousarray(seg, dtype=np.float64).copy()
    lib().orc_transform(s, len(s), float(scale), np.asarray(shift, dtype=np.float64))
    return s


def frontal_area(seg, pitch=0.125):
    return lib().orc_frontal_area(np.ascontiguousarray(seg), len(seg), float(pitch))


def place_tree(tree, trunk_cells, domain_finest):
    """Scale so the trunk is ``trunk_cells`` finest cells long and move the
    centre of mass to (Lx/4, Ly/2, Lz/2) of the domain (Sec. 2.3: the tree's
    centre of mass at (8H, 8H, 8H) of a 32H x 16H x 16H box)."""
    seg = lsystem(tree)
    s = transform(seg, trunk_cells / tree.s0, np.zeros(3))
    com = tree_com(s)
    Lx, Ly, Lz = domain_finest
    target = np.array([Lx / 4.0, Ly / 2.0, Lz / 2.0])
    return transform(s, 1.0, target - com)


def refine_boxes(seg, levels, n0, block, margin=0.25):
    """Refinement boxes R_l (l >= 1) in level-l cells, [lo, hi).

    Finest level: the tree's bounding box grown by ``margin`` of its extent on
    every side, rounded outward to whole blocks of finest cells.  Each coarser
    level: the footprint of the next finer box on it, rounded outward to whole
    blocks of its own cells and grown by one block on every side."""
    boxes = [None] * levels
    if levels == 1:
        return boxes
    lo, hi = tree_bbox(seg)
    ext = hi - lo
    lo_f = np.floor((lo - margin * ext) / block) * block
    hi_f = np.ceil((hi + margin * ext) / block) * block
    boxes[levels - 1] = lo_f.astype(int).tolist() + hi_f.astype(int).tolist()
    for l in range(levels - 2, 0, -1):
        f = np.array(boxes[l + 1], dtype=float)
        lo_l = np.floor(f[:3] / 2.0 / block) * block - block
        hi_l = np.ceil(f[3:] / 2.0 / block) * block + block
        boxes[l] = lo_l.astype(int).tolist() + hi_l.astype(int).tolist()
    return boxes


def cylinders_as_prims(seg):
    arr = (Prim * max(1, len(seg)))()
    for k, row in enumerate(seg):
        arr[k].kind = 0
        for q in range(8):
            arr[k].p[q] = float(row[q])
    return arr, len(seg)


def prims(items):
    """items: list of (kind, params)."""
    arr = (Prim * max(1, len(items)))()
    for k, (kind, p) in enumerate(items):
        arr[k].kind = kind
        for q, v in enumerate(p):
            arr[k].p[q] = float(v)
    return arr, len(items)


def prim_inside(pr, x):
    arr, n = pr
    return bool(lib().orc_prim_inside(arr, n, np.asarray(x, dtype=np.float64)))


def prim_ray(pr, x, d):
    arr, n = pr
    return lib().orc_prim_ray(arr, n, np.asarray(x, dtype=np.float64), np.asarray(d, dtype=np.float64))


# ---------------------------------------------------------------- collision (Sec. 2.2)

def rates(omega1, omega2=1.0, omega_hi=(1.0,) * 8, galilean=True):
    r = Rates()
    r.omega1, r.omega2, r.galilean = omega1, omega2, int(galilean)
    for q in range(8):
        r.omega_hi[q] = omega_hi[q]
    return r


def equilibrium(rho, u):
    f = np.zeros(27)
    lib().orc_equilibrium(float(rho), np.asarray(u, dtype=np.float64), f)
    return f


def cumulants(f):
    k = np.zeros(27)
    lib().orc_cumulants(np.ascontiguousarray(f, dtype=np.float64), k)
    return k


def collide(f, r, force=None):
    out = np.zeros(27)
    fp = None
    if force is not None:
        fa = (C.c_double * 3)(*force)
        fp = C.cast(fa, C.c_void_p)
    lib().orc_collide(np.ascontiguousarray(f, dtype=np.float64), out, C.byref(r), fp)
    return out


# ---------------------------------------------------------------- simulation

class Sim:
    """Multi-level FP64 simulation; levels indexed 0 (coarsest) .. L-1."""

    def __init__(self, nx, ny, nz, levels=1, boxes=None, bc=("inout", "slip", "slip"), u_in=0.05,
                 nu0=0.01, omega2=1.0, omega_hi=(1.0,) * 8, galilean=True, force=(0.0, 0.0, 0.0)):
        d = Desc()
        d.levels, d.nx, d.ny, d.nz = levels, nx, ny, nz
        boxes = boxes or [None] * levels
        for l in range(1, levels):
            for q in range(6):
                d.box[l][q] = int(boxes[l][q])
        for a in range(3):
            d.bc[a] = _BC_NAMES[bc[a]] if isinstance(bc[a], str) else int(bc[a])
            d.force[a] = force[a]
        d.u_in, d.nu0, d.omega2, d.galilean = u_in, nu0, omega2, int(galilean)
        for q in range(8):
            d.omega_hi[q] = omega_hi[q]
        self.levels = levels
        self._h = lib().orc_create(C.byref(d))
        if not self._h:
            raise ValueError("oracle rejected the domain description")

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def set_prims(self, pr):
        arr, n = pr
        rc = lib().orc_set_prims(self._h, arr, n)
        if rc != 0:
            raise ValueError("oracle rejected the geometry (%d)" % rc)

    def init_uniform(self, rho, u):
        lib().orc_init_uniform(self._h, float(rho), np.asarray(u, dtype=np.float64))

    def init_field(self, level, rho, u):
        rho = np.ascontiguousarray(rho, dtype=np.float64).ravel()
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        if lib().orc_init_field(self._h, level, rho, u) != 0:
            raise ValueError("bad level")

    def step(self, n=1):
        lib().orc_step(self._h, int(n))

    def box(self, level):
        lo = np.zeros(3, np.int32)
        hi = np.zeros(3, np.int32)
        lib().orc_level_box(self._h, level, lo, hi)
        return lo, hi

    def shape(self, level):
        lo, hi = self.box(level)
        return tuple(int(v) for v in (hi - lo))

    def f(self, level=0):
        nx, ny, nz = self.shape(level)
        out = np.zeros(nx * ny * nz * 27)
        lib().orc_get_f(self._h, level, out)
        return out.reshape(nz, ny, nx, 27)

    def macro(self, level=0):
        nx, ny, nz = self.shape(level)
        rho = np.zeros(nx * ny * nz)
        u = np.zeros(nx * ny * nz * 3)
        lib().orc_get_macro(self._h, level, rho, u)
        return rho.reshape(nz, ny, nx), u.reshape(nz, ny, nx, 3)

    def links(self, level):
        n = lib().orc_level_links(self._h, level, None, None, None, 0)
        cell = np.zeros(n, np.int64)
        d = np.zeros(n, np.int32)
        q = np.zeros(n)
        lib().orc_level_links(self._h, level, cell.ctypes.data, d.ctypes.data, q.ctypes.data, n)
        return cell, d, q

    def link_segments(self, level):
        """The primitive (branch) each cut link of the level belongs to, in the order of links()."""
        n = lib().orc_level_links(self._h, level, None, None, None, 0)
        seg = np.zeros(n, np.int32)
        lib().orc_level_link_segs(self._h, level, seg.ctypes.data, n)
        return seg

    def force(self):
        last, tot = np.zeros(3), np.zeros(3)
        n = C.c_long()
        lib().orc_force(self._h, last, tot, C.byref(n))
        return last, tot, n.value

    def mass(self):
        m = C.c_double()
        p = np.zeros(3)
        lib().orc_mass(self._h, C.byref(m), p)
        return m.value, p

    def set_turbulence(self, modes, u_in):
        """Turbulent inflow from a mode table (n x 7: k, a, psi)."""
        m = np.ascontiguousarray(modes, dtype=np.float64).reshape(-1, 7)
        lib().orc_set_turbulence(self._h, m.ravel() if len(m) else np.zeros(7), len(m), float(u_in))

    def branch_forces(self, n):
        out = np.zeros((max(1, n), 3))
        lib().orc_branch_forces(self._h, out, max(1, n))
        return out[:n]

    def cell_type(self, level):
        nx, ny, nz = self.shape(level)
        out = np.zeros(nx * ny * nz, np.uint8)
        lib().orc_cell_type(self._h, level, out)
        return out.reshape(nz, ny, nx)


def set_threads(n):
    """Host threads of the oracle's OpenMP loops; returns the previous count."""
    return lib().orc_set_threads(int(n))


def drag_coefficient(fx, u, area):
    """Eq. (7): C_D = F_D / (1/2 rho U^2 A_x) with rho = 1 (lattice units)."""
    return fx / (0.5 * 1.0 * u * u * area)


def tree_case(nx, ny, nz, tree, trunk_cells, re_h, u_in=0.05, levels=1, block=16, margin=0.25,
              bc=("inout", "slip", "slip"), pitch=0.125, galilean=True):
    """Oracle simulation of a tree in a channel: geometry placed and scaled,
    refinement boxes from the bounding-box rule, nu from Re_H = U H / nu on the
    finest level, solids and links classified.  Returns (sim, info)."""
    fin = 2 ** (levels - 1)
    seg = place_tree(tree, trunk_cells, (nx * fin, ny * fin, nz * fin))
    H = tree_height(seg)
    nu_f = u_in * H / re_h
    nu0 = nu_f / fin
    boxes = refine_boxes(seg, levels, (nx, ny, nz), block, margin)
    sim = Sim(nx, ny, nz, levels=levels, boxes=boxes, bc=bc, u_in=u_in, nu0=nu0, galilean=galilean)
    sim.set_prims(cylinders_as_prims(seg))
    area = frontal_area(seg, pitch)
    return sim, {"segments": seg, "H": H, "nu_finest": nu_f, "nu0": nu0, "boxes": boxes, "A_x": area}
