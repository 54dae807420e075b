"""Python binding of liblbm (include/lbm.h): ctypes argument marshalling only.

Every function named ``lbm_*`` here calls the C function of the same name;
all computation runs in the library's CUDA kernels.  Device memory and the
stream come from PyTorch (``Domain`` allocates the bound buffer with
``torch.empty`` on the current device).  Importing this module fails loudly
when the compiled library is missing: there is no other code path.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ESTATE, LBM_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
BC = {"periodic": 0, "inout": 1, "slip": 2, "inflow": 3}
LBM_FP64 = 0
LBM_FP32 = 1
LBM_FP16_DEV = 2
BRANCH_COLS = 11  # columns of lbm_branch_table


class DomainDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("levels", C.c_int), ("block", C.c_int),
                ("bc", C.c_int * 3), ("u_in", C.c_double), ("re_h", C.c_double), ("nu_finest", C.c_double),
                ("i_u", C.c_double), ("seed", C.c_ulonglong), ("refine_margin", C.c_double),
                ("precision", C.c_int), ("galilean", C.c_int), ("omega2", C.c_double),
                ("boxes", (C.c_int * 6) * 6)]


class TreeDesc(C.Structure):
    _fields_ = [("n", C.c_int), ("children", C.c_int), ("s0", C.c_double), ("w0", C.c_double),
                ("min_len", C.c_double), ("r", C.c_double * 4), ("dfac", C.c_double * 4),
                ("alpha_deg", C.c_double * 4), ("phi_deg", C.c_double * 4), ("azimuth_mode", C.c_int),
                ("seed", C.c_ulonglong), ("trunk_cells", C.c_double)]


class Schedule(C.Structure):
    _fields_ = [("ctas_per_sm", C.c_int), ("odd_variant", C.c_int), ("even_variant", C.c_int),
                ("z_split_even", C.c_int), ("z_split_odd", C.c_int)]

    def as_dict(self):
        return {"ctas_per_sm": self.ctas_per_sm, "odd_variant": ODD_VARIANTS[self.odd_variant],
                "even_variant": EVEN_VARIANTS[self.even_variant], "z_split_even": self.z_split_even,
                "z_split_odd": self.z_split_odd}


ODD_VARIANTS = {0: "columns", 1: "staged", 2: "direct", 3: "pairs", 4: "pairs_7", 5: "pairs_8"}
EVEN_VARIANTS = {0: "direct", 1: "tma", 2: "pairs"}


class LbmError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = "%s failed: %s (%d): %s" % (where, _lib.lbm_status_string(code).decode(), code,
                                          _lib.lbm_last_error().decode())
        super().__init__(msg)


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("liblbm.so is not built (run __graft_entry__.build()); there is no fallback path")
    L = C.CDLL(LIB_PATH)
    vp, i, d, sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    dp, ip, llp, ubp = C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_longlong), C.POINTER(C.c_ubyte)
    sig = {
        "lbm_create_domain": ([C.POINTER(DomainDesc), vp, C.POINTER(vp)], i),
        "lbm_set_geometry": ([vp, C.POINTER(TreeDesc)], i),
        "lbm_set_geometry_segments": ([vp, dp, i], i),
        "lbm_set_geometry_prims": ([vp, ip, dp, i], i),
        "lbm_memory_requirements": ([vp, C.POINTER(sz)], i),
        "lbm_bind_memory": ([vp, vp, sz], i),
        "lbm_memory_breakdown": ([vp, C.POINTER(sz), C.POINTER(sz)], i),
        "lbm_init_uniform": ([vp, d, dp], i),
        "lbm_init_field": ([vp, i, dp, dp, sz], i),
        "lbm_step": ([vp, i], i),
        "lbm_drag": ([vp, dp, dp, dp], i),
        "lbm_drag_enqueue": ([vp, vp], i),
        "lbm_drag_decode": ([vp, dp, dp, dp, dp], i),
        "lbm_reset_force": ([vp], i),
        "lbm_get_populations": ([vp, i, dp, sz], i),
        "lbm_get_populations_window": ([vp, i, ip, ip, dp, sz], i),
        "lbm_get_velocity": ([vp, i, dp, dp, sz], i),
        "lbm_mass": ([vp, dp, dp], i),
        "lbm_mass_noalloc": ([vp, dp, dp], i),
        "lbm_level_mass": ([vp, i, dp, dp], i),
        "lbm_set_interface_ledger": ([vp, i], i),
        "lbm_interface_ledger": ([vp, i, dp, dp, llp], i),
        "lbm_level_info": ([vp, i, ip, ip, llp, llp, llp], i),
        "lbm_geometry_info": ([vp, dp, dp, ip, dp], i),
        "lbm_get_cell_types": ([vp, i, ubp, sz], i),
        "lbm_get_links": ([vp, i, llp, ip, dp, sz, llp], i),
        "lbm_get_link_branches": ([vp, i, ip, sz, llp], i),
        "lbm_get_segments": ([vp, dp, i, ip], i),
        "lbm_set_watchdog": ([vp, i], i),
        "lbm_branch_table": ([vp, dp, i, ip], i),
        "lbm_branch_drag_estimate": ([dp, i, dp, C.c_double, dp, dp], i),
        "lbm_branch_coefficients": ([vp, dp, dp, i, dp, dp], i),
        "lbm_mlp_ensemble_forward": ([C.POINTER(vp), i, vp, i, vp], i),
        "lbm_set_branch_forces": ([vp, i], i),
        "lbm_set_wide_offsets": ([vp, i], i),
        "lbm_set_overlap": ([vp, i], i),
        "lbm_get_overlap": ([vp, ip, ip], i),
        "lbm_set_overlap_features": ([vp, i], i),
        "lbm_get_overlap_features": ([vp, ip], i),
        "lbm_set_inflow_turbulence": ([vp, i, C.c_double], i),
        "lbm_friction": ([vp, dp, dp, i, dp], i),
        "lbm_set_friction_mean": ([vp, i], i),
        "lbm_get_friction_mean": ([vp, dp, dp, i, llp], i),
        "lbm_friction_samples": ([vp, dp, i, ip], i),
        "lbm_set_schedule": ([vp, C.POINTER(Schedule)], i),
        "lbm_get_schedule": ([vp, C.POINTER(Schedule)], i),
        "lbm_autotune": ([vp, i, C.POINTER(Schedule), dp], i),
        "lbm_batch_create": ([C.POINTER(vp), i, vp, C.POINTER(vp)], i),
        "lbm_batch_memory_requirements": ([vp, C.POINTER(sz)], i),
        "lbm_batch_bind_memory": ([vp, vp, sz], i),
        "lbm_batch_set_schedule": ([vp, C.POINTER(Schedule)], i),
        "lbm_batch_get_schedule": ([vp, C.POINTER(Schedule)], i),
        "lbm_batch_step": ([vp, i], i),
        "lbm_batch_use_graphs": ([vp, i], i),
        "lbm_batch_autotune": ([vp, i, C.POINTER(Schedule), dp], i),
        "lbm_batch_destroy": ([vp], None),
        "lbm_inflow_modes": ([vp, dp, i, ip], i),
        "lbm_get_branch_forces": ([vp, dp, i, llp], i),
        "lbm_use_graphs": ([vp, i], i),
        "lbm_set_timing": ([vp, i], i),
        "lbm_get_timing": ([vp, dp, llp, llp], i),
        "lbm_work_per_step": ([vp, llp, ip], i),
        "lbm_save": ([vp, C.c_char_p], i),
        "lbm_load": ([vp, C.c_char_p], i),
        "lbm_destroy": ([vp], None),
        "lbm_status_string": ([i], C.c_char_p),
        "lbm_mlp_create": ([i, i, i, vp, C.POINTER(vp)], i),
        "lbm_mlp_memory_requirements": ([vp, i, C.POINTER(sz)], i),
        "lbm_mlp_bind_memory": ([vp, vp, sz, i], i),
        "lbm_mlp_param_count": ([vp, llp], i),
        "lbm_mlp_set_params": ([vp, C.POINTER(C.c_float), C.c_longlong], i),
        "lbm_mlp_get_params": ([vp, C.POINTER(C.c_float), C.c_longlong], i),
        "lbm_mlp_set_normalization": ([vp, C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_float, C.c_float], i),
        "lbm_mlp_forward": ([vp, vp, i, vp], i),
        "lbm_mlp_gradients": ([vp, vp, vp, vp, i, C.POINTER(C.c_float), dp], i),
        "lbm_mlp_train_step": ([vp, vp, vp, vp, i, C.c_float, dp], i),
        "lbm_mlp_last_error": ([], C.c_char_p),
        "lbm_mlp_destroy": ([vp], None),
        "lbm_last_error": ([], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    return L


_lib = _load()


def _ck(rc, where):
    if rc != LBM_OK:
        raise LbmError(rc, where)
    return rc


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# ---------------------------------------------------------------- thin wrappers, C names

def lbm_create_domain(desc, stream_ptr=0):
    h = C.c_void_p()
    _ck(_lib.lbm_create_domain(C.byref(desc), C.c_void_p(stream_ptr), C.byref(h)), "lbm_create_domain")
    return h


def lbm_set_geometry(h, tree):
    return _ck(_lib.lbm_set_geometry(h, C.byref(tree)), "lbm_set_geometry")


def lbm_set_geometry_segments(h, seg):
    seg = np.ascontiguousarray(seg, dtype=np.float64).reshape(-1, 8)
    return _ck(_lib.lbm_set_geometry_segments(h, _dp(seg), len(seg)), "lbm_set_geometry_segments")


def lbm_set_geometry_prims(h, kinds, params):
    kinds = np.ascontiguousarray(kinds, dtype=np.int32)
    params = np.ascontiguousarray(params, dtype=np.float64).reshape(-1, 8)
    return _ck(_lib.lbm_set_geometry_prims(h, kinds.ctypes.data_as(C.POINTER(C.c_int)), _dp(params),
                                           len(kinds)), "lbm_set_geometry_prims")


def lbm_memory_requirements(h):
    n = C.c_size_t()
    _ck(_lib.lbm_memory_requirements(h, C.byref(n)), "lbm_memory_requirements")
    return n.value


def lbm_memory_breakdown(h):
    """(population bytes, host-to-device bytes of one binding)"""
    p, u = C.c_size_t(), C.c_size_t()
    _ck(_lib.lbm_memory_breakdown(h, C.byref(p), C.byref(u)), "lbm_memory_breakdown")
    return p.value, u.value


def lbm_bind_memory(h, ptr, nbytes):
    return _ck(_lib.lbm_bind_memory(h, C.c_void_p(ptr), nbytes), "lbm_bind_memory")


def lbm_init_uniform(h, rho, u):
    u = np.asarray(u, dtype=np.float64)
    return _ck(_lib.lbm_init_uniform(h, float(rho), _dp(u)), "lbm_init_uniform")


def lbm_init_field(h, level, rho, u):
    rho = np.ascontiguousarray(rho, dtype=np.float64).ravel()
    u = np.ascontiguousarray(u, dtype=np.float64).ravel()
    return _ck(_lib.lbm_init_field(h, level, _dp(rho), _dp(u), len(rho)), "lbm_init_field")


def lbm_step(h, n):
    return _ck(_lib.lbm_step(h, int(n)), "lbm_step")


def lbm_drag(h):
    last, mean, cd = np.zeros(3), np.zeros(3), C.c_double()
    _ck(_lib.lbm_drag(h, _dp(last), _dp(mean), C.byref(cd)), "lbm_drag")
    return last, mean, cd.value


def lbm_drag_enqueue(h, host_ptr):
    """Enqueue the copy of the 8 force accumulators to host memory at
    host_ptr (an address, page-locked for the copy to be asynchronous)."""
    return _ck(_lib.lbm_drag_enqueue(h, C.c_void_p(host_ptr)), "lbm_drag_enqueue")


def lbm_drag_decode(h, acc):
    """lbm_drag's (force_last, force_mean, c_d) from 8 accumulators."""
    a = np.ascontiguousarray(acc, dtype=np.float64)
    last, mean, cd = np.zeros(3), np.zeros(3), C.c_double()
    _ck(_lib.lbm_drag_decode(h, _dp(a), _dp(last), _dp(mean), C.byref(cd)), "lbm_drag_decode")
    return last, mean, cd.value


def lbm_reset_force(h):
    return _ck(_lib.lbm_reset_force(h), "lbm_reset_force")


def lbm_level_info(h, level):
    lo, hi = (C.c_int * 3)(), (C.c_int * 3)()
    nf, nl, nb = C.c_longlong(), C.c_longlong(), C.c_longlong()
    _ck(_lib.lbm_level_info(h, level, lo, hi, C.byref(nf), C.byref(nl), C.byref(nb)), "lbm_level_info")
    return {"lo": tuple(lo), "hi": tuple(hi), "n_fluid": nf.value, "n_links": nl.value, "n_active_blocks": nb.value}


def _box_shape(h, level):
    info = lbm_level_info(h, level)
    return tuple(info["hi"][a] - info["lo"][a] for a in range(3))


def lbm_get_populations(h, level):
    nx, ny, nz = _box_shape(h, level)
    out = np.zeros(nx * ny * nz * 27)
    _ck(_lib.lbm_get_populations(h, level, _dp(out), nx * ny * nz), "lbm_get_populations")
    return out.reshape(nz, ny, nx, 27)


def lbm_get_populations_window(h, level, lo, hi):
    """Populations of the cells [lo, hi) (x, y, z; counted from the level's
    box) as an array (z, y, x, 27)."""
    lo_c, hi_c = (C.c_int * 3)(*[int(v) for v in lo]), (C.c_int * 3)(*[int(v) for v in hi])
    nx, ny, nz = (int(hi[a]) - int(lo[a]) for a in range(3))
    out = np.zeros(max(nx * ny * nz, 0) * 27)
    _ck(_lib.lbm_get_populations_window(h, level, lo_c, hi_c, _dp(out), max(nx * ny * nz, 0)),
        "lbm_get_populations_window")
    return out.reshape(nz, ny, nx, 27)


def lbm_get_velocity(h, level):
    nx, ny, nz = _box_shape(h, level)
    rho, u = np.zeros(nx * ny * nz), np.zeros(nx * ny * nz * 3)
    _ck(_lib.lbm_get_velocity(h, level, _dp(rho), _dp(u), nx * ny * nz), "lbm_get_velocity")
    return rho.reshape(nz, ny, nx), u.reshape(nz, ny, nx, 3)


def lbm_mass(h):
    m, p = C.c_double(), np.zeros(3)
    _ck(_lib.lbm_mass(h, C.byref(m), _dp(p)), "lbm_mass")
    return m.value, p


def lbm_mass_noalloc(h):
    m, p = C.c_double(), np.zeros(3)
    _ck(_lib.lbm_mass_noalloc(h, C.byref(m), _dp(p)), "lbm_mass_noalloc")
    return m.value, p


def lbm_level_mass(h, level):
    m, p = C.c_double(), np.zeros(3)
    _ck(_lib.lbm_level_mass(h, level, C.byref(m), _dp(p)), "lbm_level_mass")
    return m.value, p


def lbm_set_interface_ledger(h, on):
    return _ck(_lib.lbm_set_interface_ledger(h, int(bool(on))), "lbm_set_interface_ledger")


def lbm_interface_ledger(h, level):
    """(last coarse step's 12 values, totals, steps): In, OutF, RecvC x (mass, jx, jy, jz)."""
    last, total, n = np.zeros(12), np.zeros(12), C.c_longlong()
    _ck(_lib.lbm_interface_ledger(h, level, _dp(last), _dp(total), C.byref(n)), "lbm_interface_ledger")
    return last, total, n.value


def lbm_geometry_info(h):
    H, A, nu = C.c_double(), C.c_double(), C.c_double()
    ns = C.c_int()
    _ck(_lib.lbm_geometry_info(h, C.byref(H), C.byref(A), C.byref(ns), C.byref(nu)), "lbm_geometry_info")
    return {"H": H.value, "A_x": A.value, "n_segments": ns.value, "nu_finest": nu.value}


def lbm_get_cell_types(h, level):
    nx, ny, nz = _box_shape(h, level)
    out = np.zeros(nx * ny * nz, np.uint8)
    _ck(_lib.lbm_get_cell_types(h, level, out.ctypes.data_as(C.POINTER(C.c_ubyte)), nx * ny * nz),
        "lbm_get_cell_types")
    return out.reshape(nz, ny, nx)


def lbm_get_links(h, level):
    n = C.c_longlong()
    _ck(_lib.lbm_get_links(h, level, None, None, None, 0, C.byref(n)), "lbm_get_links")
    cell = np.zeros(n.value, np.int64)
    d = np.zeros(n.value, np.int32)
    q = np.zeros(n.value)
    _ck(_lib.lbm_get_links(h, level, cell.ctypes.data_as(C.POINTER(C.c_longlong)),
                           d.ctypes.data_as(C.POINTER(C.c_int)), _dp(q), n.value, C.byref(n)), "lbm_get_links")
    return cell, d, q


def lbm_get_link_branches(h, level):
    """The branch of each cut link of a level, in the order of lbm_get_links."""
    n = C.c_longlong()
    _ck(_lib.lbm_get_link_branches(h, level, None, 0, C.byref(n)), "lbm_get_link_branches")
    out = np.zeros(n.value, np.int32)
    _ck(_lib.lbm_get_link_branches(h, level, out.ctypes.data_as(C.POINTER(C.c_int)), n.value, C.byref(n)),
        "lbm_get_link_branches")
    return out


def lbm_get_segments(h):
    n = C.c_int()
    _ck(_lib.lbm_get_segments(h, None, 0, C.byref(n)), "lbm_get_segments")
    seg = np.zeros((n.value, 8))
    _ck(_lib.lbm_get_segments(h, _dp(seg), n.value, C.byref(n)), "lbm_get_segments")
    return seg


def lbm_set_branch_forces(h, on):
    return _ck(_lib.lbm_set_branch_forces(h, int(bool(on))), "lbm_set_branch_forces")


def lbm_set_inflow_turbulence(h, n_modes=256, integral_length=0.0):
    return _ck(_lib.lbm_set_inflow_turbulence(h, int(n_modes), float(integral_length)), "lbm_set_inflow_turbulence")


def lbm_inflow_modes(h):
    """Mode table (n x 7: k, a, psi) of a turbulent-inflow domain."""
    n = C.c_int()
    _ck(_lib.lbm_inflow_modes(h, None, 0, C.byref(n)), "lbm_inflow_modes")
    out = np.zeros((max(1, n.value), 7))
    _ck(_lib.lbm_inflow_modes(h, _dp(out), max(1, n.value), C.byref(n)), "lbm_inflow_modes")
    return out[:n.value]


def _n_prims(h):
    n = C.c_int()
    _ck(_lib.lbm_friction_samples(h, None, 0, C.byref(n)), "lbm_friction_samples")
    return n.value


def lbm_friction(h, n_branches=0):
    """Friction force of the current state, per-branch rows (n_branches x 3) and C_F."""
    f = np.zeros(3)
    rows = np.zeros((max(1, n_branches), 3))
    cf = C.c_double()
    _ck(_lib.lbm_friction(h, _dp(f), _dp(rows) if n_branches else None, n_branches, C.byref(cf)), "lbm_friction")
    return f, rows[:n_branches], cf.value


def lbm_set_friction_mean(h, on):
    return _ck(_lib.lbm_set_friction_mean(h, int(bool(on))), "lbm_set_friction_mean")


def lbm_get_friction_mean(h, n_branches=0):
    f = np.zeros(3)
    rows = np.zeros((max(1, n_branches), 3))
    steps = C.c_longlong()
    _ck(_lib.lbm_get_friction_mean(h, _dp(f), _dp(rows) if n_branches else None, n_branches, C.byref(steps)),
        "lbm_get_friction_mean")
    return f, rows[:n_branches], steps.value


def lbm_friction_samples(h):
    """Quadrature points, n x 13: cell A (3), cell B (3), normal (3), area, distances (2), branch."""
    n = _n_prims(h)
    out = np.zeros((max(1, n), 13))
    c = C.c_int()
    _ck(_lib.lbm_friction_samples(h, _dp(out), max(1, n), C.byref(c)), "lbm_friction_samples")
    return out[:c.value]


def lbm_set_schedule(h, ctas_per_sm=0, odd_variant=0, even_variant=0, z_split_even=0, z_split_odd=0):
    s = Schedule(ctas_per_sm, odd_variant, even_variant, z_split_even, z_split_odd)
    return _ck(_lib.lbm_set_schedule(h, C.byref(s)), "lbm_set_schedule")


def lbm_get_schedule(h):
    s = Schedule()
    _ck(_lib.lbm_get_schedule(h, C.byref(s)), "lbm_get_schedule")
    return s


def lbm_autotune(h, steps=3):
    """Time the collide-variant pairs, then the z splits, keep the fastest: (Schedule, ms per coarse step)."""
    s, ms = Schedule(), C.c_double()
    _ck(_lib.lbm_autotune(h, steps, C.byref(s), C.byref(ms)), "lbm_autotune")
    return s, ms.value


def lbm_set_wide_offsets(h, on):
    return _ck(_lib.lbm_set_wide_offsets(h, int(bool(on))), "lbm_set_wide_offsets")


def lbm_set_overlap(h, on):
    return _ck(_lib.lbm_set_overlap(h, int(bool(on))), "lbm_set_overlap")


LBM_OVL_BRANCHES, LBM_OVL_LEVELS, LBM_OVL_TRANSFERS, LBM_OVL_DEFER, LBM_OVL_WALL_SPLIT = 1, 2, 4, 8, 16
LBM_OVL_ALL = 31


def lbm_set_overlap_features(h, mask):
    return _ck(_lib.lbm_set_overlap_features(h, int(mask)), "lbm_set_overlap_features")


def lbm_get_overlap_features(h):
    m = C.c_int()
    _ck(_lib.lbm_get_overlap_features(h, C.byref(m)), "lbm_get_overlap_features")
    return m.value


def lbm_get_overlap(h):
    """(faces may branch, bit mask of levels whose walls may branch)"""
    f, w = C.c_int(), C.c_int()
    _ck(_lib.lbm_get_overlap(h, C.byref(f), C.byref(w)), "lbm_get_overlap")
    return bool(f.value), w.value


def lbm_get_branch_forces(h, n_branches):
    out = np.zeros((max(1, n_branches), 3))
    steps = C.c_longlong()
    _ck(_lib.lbm_get_branch_forces(h, _dp(out), max(1, n_branches), C.byref(steps)), "lbm_get_branch_forces")
    return out[:n_branches], steps.value


def lbm_branch_drag_estimate(rows, area, c_sect=None):
    """Eq. 4 over the branches of a branch table; returns (C_D-est, c_k)."""
    rows = np.ascontiguousarray(rows, dtype=np.float64)
    n = rows.shape[0]
    c_out = np.zeros(max(1, n))
    cs = None if c_sect is None else np.ascontiguousarray(c_sect, dtype=np.float64)
    cd = C.c_double()
    _ck(_lib.lbm_branch_drag_estimate(_dp(rows) if n else _dp(np.zeros(BRANCH_COLS)), n, _dp(cs) if cs is not None else None,
                                      float(area), C.byref(cd), _dp(c_out)), "lbm_branch_drag_estimate")
    return cd.value, c_out[:n]


def lbm_branch_coefficients(h, n_branches):
    """Eq. 2's measured sectional coefficients: (c_drag, c_fric, C_D, C_F) over the averaging window."""
    cd_, cf_ = np.zeros(max(1, n_branches)), np.zeros(max(1, n_branches))
    cd, cf = C.c_double(), C.c_double()
    _ck(_lib.lbm_branch_coefficients(h, _dp(cd_), _dp(cf_), n_branches, C.byref(cd), C.byref(cf)),
        "lbm_branch_coefficients")
    return cd_[:n_branches], cf_[:n_branches], cd.value, cf.value


def lbm_branch_table(h):
    n = C.c_int()
    _ck(_lib.lbm_branch_table(h, None, 0, C.byref(n)), "lbm_branch_table")
    out = np.zeros((max(1, n.value), BRANCH_COLS))
    _ck(_lib.lbm_branch_table(h, _dp(out), max(1, n.value), C.byref(n)), "lbm_branch_table")
    return out[:n.value]


def lbm_set_watchdog(h, every):
    return _ck(_lib.lbm_set_watchdog(h, int(every)), "lbm_set_watchdog")


def lbm_use_graphs(h, on):
    return _ck(_lib.lbm_use_graphs(h, int(bool(on))), "lbm_use_graphs")


def lbm_set_timing(h, on):
    return _ck(_lib.lbm_set_timing(h, int(bool(on))), "lbm_set_timing")


def lbm_get_timing(h):
    ms = np.zeros(6)
    la = np.zeros(6, np.int64)
    un = np.zeros(6, np.int64)
    _ck(_lib.lbm_get_timing(h, _dp(ms), la.ctypes.data_as(C.POINTER(C.c_longlong)),
                            un.ctypes.data_as(C.POINTER(C.c_longlong))), "lbm_get_timing")
    return ms, la, un


def lbm_work_per_step(h):
    cu, k = C.c_longlong(), C.c_int()
    _ck(_lib.lbm_work_per_step(h, C.byref(cu), C.byref(k)), "lbm_work_per_step")
    return cu.value, k.value


def lbm_save(h, path):
    return _ck(_lib.lbm_save(h, path.encode()), "lbm_save")


def lbm_load(h, path):
    return _ck(_lib.lbm_load(h, path.encode()), "lbm_load")


def lbm_destroy(h):
    _lib.lbm_destroy(h)


def lbm_status_string(code):
    return _lib.lbm_status_string(code).decode()


# ---------------------------------------------------------------- descriptors

def domain_desc(nx, ny, nz, levels=1, block=16, bc=("inout", "slip", "slip"), u_in=0.05, re_h=0.0,
                nu_finest=0.0, refine_margin=0.25, galilean=True, omega2=1.0, boxes=None, precision=LBM_FP32,
                i_u=0.0, seed=0):
    d = DomainDesc()
    d.nx, d.ny, d.nz, d.levels, d.block = nx, ny, nz, levels, block
    for a in range(3):
        d.bc[a] = BC[bc[a]] if isinstance(bc[a], str) else int(bc[a])
    d.u_in, d.re_h, d.nu_finest, d.i_u, d.seed = u_in, re_h, nu_finest, i_u, seed
    d.refine_margin, d.precision, d.galilean, d.omega2 = refine_margin, precision, int(galilean), omega2
    if boxes:
        for l, b in enumerate(boxes):
            if b is not None:
                for q in range(6):
                    d.boxes[l][q] = int(b[q])
    return d


def tree_desc(n, children=2, s0=100.0, w0=30.0, r=(0.8,), dfac=(0.5 ** 0.5,), alpha_deg=(30.0, -30.0),
              phi_deg=(137.0,), azimuth_mode=0, seed=0, min_len=0.02, trunk_cells=None):
    t = TreeDesc()
    t.n, t.children, t.s0, t.w0, t.min_len = n, children, s0, w0, min_len
    for k in range(children):
        t.r[k] = r[k % len(r)]
        t.dfac[k] = dfac[k % len(dfac)]
        t.alpha_deg[k] = alpha_deg[k % len(alpha_deg)]
        t.phi_deg[k] = phi_deg[k % len(phi_deg)]
    t.azimuth_mode, t.seed = azimuth_mode, seed
    t.trunk_cells = s0 if trunk_cells is None else trunk_cells
    return t


class Domain:
    """Convenience owner of a domain handle and its torch-allocated buffer."""

    def __init__(self, desc, tree=None, segments=None, prims=None, device="cuda", stream=None, bind=True):
        self._torch = None
        self.stream = stream
        sp = 0
        if stream is not None:
            sp = stream.cuda_stream
        self.h = lbm_create_domain(desc, sp)
        self.desc = desc
        if tree is not None:
            lbm_set_geometry(self.h, tree)
        elif segments is not None:
            lbm_set_geometry_segments(self.h, segments)
        else:
            kinds, params = prims if prims is not None else ([], np.zeros((0, 8)))
            lbm_set_geometry_prims(self.h, kinds, params)
        self.nbytes = lbm_memory_requirements(self.h)
        self.buffer = None
        if bind:
            self.bind(device)

    def bind(self, device="cuda"):
        import torch
        self._torch = torch
        self.buffer = torch.empty(max(self.nbytes, 256), dtype=torch.uint8, device=device)
        lbm_bind_memory(self.h, self.buffer.data_ptr(), self.buffer.numel())

    def __getattr__(self, name):
        fn = globals().get("lbm_" + name)
        if fn is None:
            raise AttributeError(name)
        return lambda *a, **k: fn(self.h, *a, **k)

    def close(self):
        if getattr(self, "h", None):
            if self.buffer is not None:
                self._torch.cuda.synchronize(self.buffer.device)
            lbm_destroy(self.h)
            self.h = None
            self.buffer = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- surrogate network

class MlpError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s failed (%d): %s" % (where, code, _lib.lbm_mlp_last_error().decode()))


def _mck(rc, where):
    if rc != LBM_OK:
        raise MlpError(rc, where)


def _fp(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


class Mlp:
    """Owner of an lbm_mlp handle and its torch-allocated buffer.  Device
    arrays are torch tensors; this class only passes their pointers."""

    def __init__(self, n_in=6, width=128, hidden=3, max_batch=4096, stream=None, device="cuda"):
        import torch
        self._torch = torch
        self.stream = stream
        h = C.c_void_p()
        _mck(_lib.lbm_mlp_create(n_in, width, hidden, C.c_void_p(stream.cuda_stream if stream else 0),
                                 C.byref(h)), "lbm_mlp_create")
        self.h = h
        n = C.c_size_t()
        _mck(_lib.lbm_mlp_memory_requirements(h, max_batch, C.byref(n)), "lbm_mlp_memory_requirements")
        self.buffer = torch.empty(n.value, dtype=torch.uint8, device=device)
        _mck(_lib.lbm_mlp_bind_memory(h, self.buffer.data_ptr(), n.value, max_batch), "lbm_mlp_bind_memory")
        p = C.c_longlong()
        _mck(_lib.lbm_mlp_param_count(h, C.byref(p)), "lbm_mlp_param_count")
        self.n_params, self.max_batch, self.n_in = p.value, max_batch, n_in

    # stream ordering: the network's kernels run on its own stream; tensors
    # the caller made on its current stream are ready before they start
    # (_enter), and the caller's stream waits for their results (_leave)
    def _enter(self):
        if self.stream is not None:
            self.stream.wait_stream(self._torch.cuda.current_stream())

    def _leave(self):
        if self.stream is not None:
            self._torch.cuda.current_stream().wait_stream(self.stream)

    def set_params(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        _mck(_lib.lbm_mlp_set_params(self.h, _fp(w), len(w)), "lbm_mlp_set_params")

    def get_params(self):
        w = np.zeros(self.n_params, np.float32)
        _mck(_lib.lbm_mlp_get_params(self.h, _fp(w), len(w)), "lbm_mlp_get_params")
        return w

    def set_normalization(self, mu_x, sd_x, mu_y, sd_y):
        mu = np.ascontiguousarray(mu_x, dtype=np.float32)
        sd = np.ascontiguousarray(sd_x, dtype=np.float32)
        _mck(_lib.lbm_mlp_set_normalization(self.h, _fp(mu), _fp(sd), float(mu_y), float(sd_y)),
             "lbm_mlp_set_normalization")

    def forward(self, x):
        """x: device float32 tensor (batch, n_in) -> device tensor (batch,)."""
        y = self._torch.empty(x.shape[0], dtype=self._torch.float32, device=x.device)
        self._enter()
        _mck(_lib.lbm_mlp_forward(self.h, C.c_void_p(x.data_ptr()), x.shape[0], C.c_void_p(y.data_ptr())),
             "lbm_mlp_forward")
        self._leave()
        return y

    def gradients(self, x, y, idx=None):
        g = np.zeros(self.n_params, np.float32)
        loss = C.c_double()
        n = idx.shape[0] if idx is not None else x.shape[0]
        self._enter()
        _mck(_lib.lbm_mlp_gradients(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                    C.c_void_p(idx.data_ptr() if idx is not None else 0), n, _fp(g),
                                    C.byref(loss)), "lbm_mlp_gradients")
        return g, loss.value

    def train_step(self, x, y, idx=None, lr=1e-3, want_loss=False):
        loss = C.c_double()
        n = idx.shape[0] if idx is not None else x.shape[0]
        self._enter()
        _mck(_lib.lbm_mlp_train_step(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                     C.c_void_p(idx.data_ptr() if idx is not None else 0), n, float(lr),
                                     C.byref(loss) if want_loss else None), "lbm_mlp_train_step")
        self._leave()
        return loss.value if want_loss else None

    def close(self):
        if getattr(self, "h", None):
            self._torch.cuda.synchronize()
            _lib.lbm_mlp_destroy(self.h)
            self.h = None
            self.buffer = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mlp_ensemble_forward(nets, x):
    """Mean prediction of several Mlp objects (device tensor x) -> device tensor."""
    import torch
    y = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
    arr = (C.c_void_p * len(nets))(*[m.h for m in nets])
    nets[0]._enter()
    _mck(_lib.lbm_mlp_ensemble_forward(arr, len(nets), C.c_void_p(x.data_ptr()), x.shape[0], C.c_void_p(y.data_ptr())),
         "lbm_mlp_ensemble_forward")
    nets[0]._leave()
    return y


class Batch:
    """Owner of an lbm_batch over several bound Domain objects (kept alive here)."""

    def __init__(self, domains, stream=None, device="cuda"):
        import torch
        self._torch = torch
        self.domains = list(domains)
        arr = (C.c_void_p * len(self.domains))(*[d.h for d in self.domains])
        h = C.c_void_p()
        _ck(_lib.lbm_batch_create(arr, len(self.domains), C.c_void_p(stream.cuda_stream if stream else 0),
                                  C.byref(h)), "lbm_batch_create")
        self.h = h
        n = C.c_size_t()
        _ck(_lib.lbm_batch_memory_requirements(h, C.byref(n)), "lbm_batch_memory_requirements")
        self.buffer = torch.empty(max(n.value, 256), dtype=torch.uint8, device=device)
        _ck(_lib.lbm_batch_bind_memory(h, self.buffer.data_ptr(), self.buffer.numel()), "lbm_batch_bind_memory")

    def step(self, n=1):
        return _ck(_lib.lbm_batch_step(self.h, int(n)), "lbm_batch_step")

    def set_schedule(self, ctas_per_sm=0, odd_variant=0, z_split_even=0, z_split_odd=0, even_variant=0):
        s = Schedule(ctas_per_sm, odd_variant, even_variant, z_split_even, z_split_odd)
        return _ck(_lib.lbm_batch_set_schedule(self.h, C.byref(s)), "lbm_batch_set_schedule")

    def get_schedule(self):
        s = Schedule()
        _ck(_lib.lbm_batch_get_schedule(self.h, C.byref(s)), "lbm_batch_get_schedule")
        return s

    def use_graphs(self, on):
        return _ck(_lib.lbm_batch_use_graphs(self.h, int(bool(on))), "lbm_batch_use_graphs")

    def autotune(self, steps=2):
        s, ms = Schedule(), C.c_double()
        _ck(_lib.lbm_batch_autotune(self.h, int(steps), C.byref(s), C.byref(ms)), "lbm_batch_autotune")
        return s, ms.value

    def close(self):
        if getattr(self, "h", None):
            self._torch.cuda.synchronize()
            _lib.lbm_batch_destroy(self.h)
            self.h = None
            self.buffer = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
