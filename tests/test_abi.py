"""The C-ABI boundary without a GPU: the library loads and exports every
function include/lbm.h declares, the header is plain C whose struct layouts
and prototypes the Python binding mirrors, and the error paths (null
arguments, calls out of order) return statuses instead of crashing."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_2603_27954_gb300 import lbm as L
    lib = C.CDLL(L.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings():
    from paper_2603_27954_gb300 import lbm as L
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert L.lbm_status_string(code) != "unknown status"


C_CALLER = r"""
#include <stdio.h>
#include "lbm.h"
int main(void) {
  lbm_domain_desc dd = {256, 128, 128, 2, 16, {LBM_BC_INOUT, LBM_BC_INFLOW, LBM_BC_INFLOW},
                        0.05, 2500.0, 0.0, 0.0, 0, 0.25, LBM_FP32, 1, 1.0, {{0}}};
  lbm_tree_desc td = {4, 3, 64.0, 19.2, 0.02, {0.6, 0.6, 0.6}, {0.6, 0.6, 0.6}, {35.0, 35.0, 35.0}, {0.0},
                      1, 1, 64.0};
  lbm_domain* d;
  if (lbm_create_domain(&dd, NULL, &d) || lbm_set_geometry(d, &td)) {
    printf("error %s\n", lbm_last_error());
    return 1;
  }
  size_t bytes;
  double H, A, nu;
  int ns;
  lbm_memory_requirements(d, &bytes);
  lbm_geometry_info(d, &H, &A, &ns, &nu);
  printf("%zu %.17g %.17g %d %.17g\n", bytes, H, A, ns, nu);
  lbm_destroy(d);
  return 0;
}
"""


def test_header_compiles_as_c_and_a_c_caller_matches_the_binding(tmp_path):
    """include/lbm.h is plain C (C11, warnings as errors), and a C caller that
    fills the descriptors by position builds the two-level benchmark tree's
    geometry exactly as the Python binding's ctypes structures do: the
    struct layouts on both sides of the boundary agree."""
    import subprocess
    from paper_2603_27954_gb300 import lbm as L
    from paper_2603_27954_gb300 import workloads as W
    src = tmp_path / "caller.c"
    src.write_text(C_CALLER)
    exe = tmp_path / "caller"
    libdir = os.path.dirname(L.LIB_PATH)
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-L", libdir, "-llbm", "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    c = W.CASES["amr2"]
    h = L.lbm_create_domain(L.domain_desc(*c["n0"], levels=c["levels"], block=c["block"], bc=c["bc"],
                                          u_in=c["u_in"], re_h=c["re_h"]))
    L.lbm_set_geometry(h, L.tree_desc(**c["tree"]))
    g = L.lbm_geometry_info(h)
    assert int(out[0]) == L.lbm_memory_requirements(h)
    assert float(out[1]) == g["H"] and float(out[2]) == g["A_x"] and float(out[4]) == g["nu_finest"]
    assert int(out[3]) == g["n_segments"] == 40
    L.lbm_destroy(h)


LAYOUT_PROBE = r"""
#include <stddef.h>
#include <stdio.h>
#include "lbm.h"
#define F(T, m) printf(#T " " #m " %zu\n", offsetof(T, m))
int main(void) {
  printf("lbm_domain_desc size %zu\n", sizeof(lbm_domain_desc));
  F(lbm_domain_desc, nx); F(lbm_domain_desc, ny); F(lbm_domain_desc, nz); F(lbm_domain_desc, levels);
  F(lbm_domain_desc, block); F(lbm_domain_desc, bc); F(lbm_domain_desc, u_in); F(lbm_domain_desc, re_h);
  F(lbm_domain_desc, nu_finest); F(lbm_domain_desc, i_u); F(lbm_domain_desc, seed);
  F(lbm_domain_desc, refine_margin); F(lbm_domain_desc, precision); F(lbm_domain_desc, galilean);
  F(lbm_domain_desc, omega2); F(lbm_domain_desc, boxes);
  printf("lbm_tree_desc size %zu\n", sizeof(lbm_tree_desc));
  F(lbm_tree_desc, n); F(lbm_tree_desc, children); F(lbm_tree_desc, s0); F(lbm_tree_desc, w0);
  F(lbm_tree_desc, min_len); F(lbm_tree_desc, r); F(lbm_tree_desc, dfac); F(lbm_tree_desc, alpha_deg);
  F(lbm_tree_desc, phi_deg); F(lbm_tree_desc, azimuth_mode); F(lbm_tree_desc, seed);
  F(lbm_tree_desc, trunk_cells);
  printf("lbm_schedule size %zu\n", sizeof(lbm_schedule));
  F(lbm_schedule, ctas_per_sm); F(lbm_schedule, odd_variant); F(lbm_schedule, even_variant);
  F(lbm_schedule, z_split_even); F(lbm_schedule, z_split_odd);
  return 0;
}
"""


def test_descriptor_layouts_match_the_binding(tmp_path):
    """Every field offset and the size of the three descriptor structs, as a
    C compiler lays them out from include/lbm.h, equal those of the Python
    binding's ctypes structures."""
    import subprocess
    from paper_2603_27954_gb300 import lbm as L
    src = tmp_path / "layout.c"
    src.write_text(LAYOUT_PROBE)
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines()
    types = {"lbm_domain_desc": L.DomainDesc, "lbm_tree_desc": L.TreeDesc, "lbm_schedule": L.Schedule}
    seen = 0
    for line in lines:
        name, field, value = line.split()
        py = types[name]
        if field == "size":
            assert C.sizeof(py) == int(value), name
        else:
            assert getattr(py, field).offset == int(value), (name, field)
        seen += 1
    assert seen == 3 + 16 + 12 + 5


def _prototypes():
    """name -> list of parameter declarations, from include/*.h (comments stripped)."""
    out = {}
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(lbm_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src):
            params = [p.strip() for p in m.group(2).split(",")]
            out[m.group(1)] = [] if params == ["void"] or params == [""] else params
    return out


def test_binding_signatures_match_the_header():
    """For every function the Python binding declares, its ctypes argument
    list has the header's arity, and each argument is a pointer exactly where
    the header's parameter is a pointer or an array."""
    from paper_2603_27954_gb300 import lbm as L
    lib = L._lib
    protos = _prototypes()
    pointerish = (C.c_void_p, C.c_char_p)
    checked = 0
    for name, params in protos.items():
        fn = getattr(lib, name, None)
        if fn is None or fn.argtypes is None:
            continue
        assert len(fn.argtypes) == len(params), (name, params, fn.argtypes)
        for p, t in zip(params, fn.argtypes):
            is_ptr = "*" in p or "[" in p
            py_ptr = t in pointerish or issubclass(t, C._Pointer)
            assert is_ptr == py_ptr, (name, p, t)
        checked += 1
    assert checked >= 60


NULL_PROBE = r"""
import ctypes as C
import re
import sys
sys.path.insert(0, %r)
from paper_2603_27954_gb300 import lbm as L
src = re.sub(r"/\*.*?\*/", "", open(%r).read(), flags=re.S)
void_fns = {"lbm_destroy", "lbm_batch_destroy", "lbm_mlp_destroy"}
text_fns = {"lbm_status_string", "lbm_last_error", "lbm_mlp_last_error"}
for name in sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src))):
    if name in text_fns:
        continue
    fn = getattr(L._lib, name)
    args = [None if (t in (C.c_void_p, C.c_char_p) or issubclass(t, C._Pointer)) else
            (0.0 if t in (C.c_double, C.c_float) else 0) for t in fn.argtypes]
    rc = fn(*args)
    print(name, "void" if name in void_fns else rc)
"""


def test_every_entry_point_rejects_null_arguments(tmp_path):
    """The error path of the boundary without a GPU: every declared function
    called with null pointers and zero sizes returns a negative status
    (LBM_EINVAL, or LBM_ESTATE where the call is out of order) and the
    destroy functions accept a null handle; nothing crashes (run in a child
    process, so that a crash is a test failure, not the end of the run)."""
    import subprocess
    import sys
    code = NULL_PROBE % (ROOT, os.path.join(ROOT, "include", "lbm.h"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    seen = dict(line.split() for line in r.stdout.splitlines())
    assert len(seen) >= 75
    for name, rc in seen.items():
        if rc != "void":
            assert int(rc) in (-1, -5), (name, rc)


def test_device_calls_before_binding_are_out_of_order(tmp_path):
    """With the geometry set but no device buffer bound, every call that needs
    the device state returns LBM_ESTATE (no device work is attempted), and the
    host-only queries succeed."""
    import numpy as np
    from paper_2603_27954_gb300 import lbm as L
    from paper_2603_27954_gb300 import workloads as W
    c = W.CASES["amr2_small"]
    h = L.lbm_create_domain(L.domain_desc(*c["n0"], levels=c["levels"], block=c["block"], bc=c["bc"],
                                          u_in=c["u_in"], re_h=c["re_h"]))
    L.lbm_set_geometry(h, L.tree_desc(**c["tree"]))
    nx, ny, nz = (L.lbm_level_info(h, 0)["hi"][a] - L.lbm_level_info(h, 0)["lo"][a] for a in range(3))
    n = nx * ny * nz
    acc = np.zeros(8)
    calls = {
        "lbm_step": lambda: L.lbm_step(h, 1),
        "lbm_drag": lambda: L.lbm_drag(h),
        "lbm_drag_enqueue": lambda: L._ck(L._lib.lbm_drag_enqueue(h, acc.ctypes.data), "lbm_drag_enqueue"),
        "lbm_reset_force": lambda: L.lbm_reset_force(h),
        "lbm_get_populations": lambda: L.lbm_get_populations(h, 0),
        "lbm_get_populations_window": lambda: L.lbm_get_populations_window(h, 0, (0, 0, 0), (2, 2, 2)),
        "lbm_mass": lambda: L.lbm_mass(h),
        "lbm_mass_noalloc": lambda: L.lbm_mass_noalloc(h),
        "lbm_level_mass": lambda: L.lbm_level_mass(h, 0),
        "lbm_interface_ledger": lambda: L.lbm_interface_ledger(h, 0),
        "lbm_init_uniform": lambda: L.lbm_init_uniform(h, 1.0, (0.05, 0.0, 0.0)),
        "lbm_init_field": lambda: L.lbm_init_field(h, 0, np.ones(n), np.zeros((n, 3))),
        "lbm_get_branch_forces": lambda: L.lbm_get_branch_forces(h, 64),
        "lbm_friction": lambda: L.lbm_friction(h),
        "lbm_save": lambda: L.lbm_save(h, str(tmp_path / "state.bin")),
        "lbm_load": lambda: L.lbm_load(h, str(tmp_path / "state.bin")),
        "lbm_autotune": lambda: L.lbm_autotune(h, 1),
    }
    for name, call in calls.items():
        with pytest.raises(L.LbmError) as e:
            call()
        assert e.value.code == L.LBM_ESTATE, (name, str(e.value))
    assert L.lbm_memory_requirements(h) > 0
    assert L.lbm_geometry_info(h)["n_segments"] == 13
    assert L.lbm_work_per_step(h)[0] > 0
    L.lbm_destroy(h)
