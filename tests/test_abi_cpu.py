"""The C-ABI library builds, loads without a GPU and exports every symbol that
include/*.h declares; host-side validation works without touching CUDA."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2005_05436_gb300 import _lib, build
    build.build()
    return _lib.load()


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(to_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_paper_entry_points():
    names = _declared_functions()
    for n in ["to_init_grid", "to_assemble_lower", "to_apply_K", "to_solve", "to_filter",
              "to_project", "to_sensitivity", "to_oc_update", "to_step", "to_destroy",
              "to_last_error"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layouts_match(lib):
    from paper_2005_05436_gb300 import _lib as L
    assert lib.to_sizeof_params() == C.sizeof(L.Params)
    assert lib.to_sizeof_state() == C.sizeof(L.State)
    assert lib.to_sizeof_iter_info() == C.sizeof(L.IterInfo)


def test_params_defaults_follow_the_paper(lib):
    from paper_2005_05436_gb300 import _lib as L
    p = L.default_params(2, 60, 20)
    assert (p.E0, p.Emin, p.nu, p.penal, p.eta, p.beta, p.move) == (1.0, 1e-9, 0.3, 3.0, 0.5, 2.0, 0.2)
    assert chr(p.ftBC) == "N" and p.ft == 3
    assert (p.penal_cnt.istart, p.penal_cnt.maxpar, p.penal_cnt.isteps, p.penal_cnt.delta) == (1, 3.0, 25, 0.25)
    assert (p.newton_tol, p.oc_tol) == (1e-6, 1e-4)
    assert (p.inner_rtol, p.inner_maxit) == (1e-3, 2000)
    # solver options (no counterpart in the paper): l1-Jacobi weight 1.8 on every level, the finest
    # level's sweeps as mg_nu, programmatic dependent launch on, the fusions on
    assert (p.mg_omega, p.mg_omega_coarse, p.mg_nu_fine, p.pdl_off, p.mg_unfused) == (1.8, 0.0, 0, 0, 0)


@pytest.mark.parametrize("field,value", [("dim", 4), ("nelx", 0), ("volfrac", 1.5), ("ft", 7),
                                         ("ftBC", ord("X")), ("rmin", -1.0), ("nelz", 3), ("inner_maxit", 0),
                                         ("oc_method", 7), ("pae_m", 5), ("inner_rtol", 1.0),
                                         ("mg_omega", 2.0), ("mg_omega_coarse", 2.5), ("mg_omega_coarse", -0.5),
                                         ("mg_nu_fine", 17), ("mg_nu_fine", -1)])
def test_invalid_params_rejected_on_host(lib, field, value):
    from paper_2005_05436_gb300 import _lib as L
    p = L.default_params(2, 8, 4)
    setattr(p, field, value)
    h = C.c_void_p()
    st = lib.to_init_grid(C.byref(p), C.c_void_p(1), C.c_void_p(1), None, None, C.byref(h))
    assert st == L.TO_EINVAL
    assert len(lib.to_last_error()) > 0
    assert h.value is None


def test_null_arguments_rejected(lib):
    from paper_2005_05436_gb300 import _lib as L
    p = L.default_params(3, 4, 2, 2)
    h = C.c_void_p()
    assert lib.to_init_grid(C.byref(p), None, None, None, None, C.byref(h)) == L.TO_EINVAL
    assert lib.to_apply_K(None, None, None, None, 1) == L.TO_EINVAL
    assert lib.to_step(None, None, None) == L.TO_EINVAL
    lib.to_destroy(None)
