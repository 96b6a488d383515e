"""C-ABI library: loads and exports every symbol the header declares (no
device calls), and the host-side validation of the Python layer."""
import ctypes
import os

import numpy as np
import pytest

from paper_2207_06043_gb300 import binding


def _built():
    return os.path.exists(binding.LIB_PATH)


@pytest.fixture(scope="module")
def lib():
    if not _built():
        from paper_2207_06043_gb300 import build
        build.build()
    return binding.lib()


def test_header_declares_the_boundary_calls():
    names = binding.header_functions()
    for required in ("ibl_create", "ibl_set_geometry", "ibl_set_inlet_velocity", "ibl_set_outlet_pressure",
                     "ibl_init_equilibrium", "ibl_add_capsule", "ibl_step", "ibl_read_fields",
                     "ibl_read_capsule", "ibl_ensemble_create", "ibl_last_error", "ibl_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in binding.header_functions():
        assert hasattr(lib, name), name


def test_struct_layouts_match_header():
    assert ctypes.sizeof(binding.WallLink) == 16
    assert ctypes.sizeof(binding.LatticeDesc) == 4 * 8 + 8 * 5
    assert ctypes.sizeof(binding.CapsuleParams) == 5 * 8 + 8


def test_create_rejects_bad_arguments_without_a_gpu(lib):
    d = binding.LatticeDesc()
    d.nx, d.ny, d.nz = 8, 8, 8
    d.tau = 0.4   # tau must exceed 1/2
    h = ctypes.c_void_p()
    st = lib.ibl_create(ctypes.byref(d), None, ctypes.byref(h))
    assert st == binding.ERR_ARG
    assert b"tau" in lib.ibl_last_error(None)


def test_product_path_fails_loudly_without_the_library(tmp_path, monkeypatch):
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        binding.lib()


def _header_arities():
    """Parameter count of every function prototype in include/ibl.h (comments
    stripped; `(void)` counts as none)."""
    import re
    txt = open(binding.HEADER).read()
    txt = re.sub(r"/\*.*?\*/", " ", txt, flags=re.S)
    out = {}
    for m in re.finditer(r"(?:ibl_status|int32_t|void|const char\s*\*)\s+(ibl_\w+)\s*\(([^)]*)\)\s*;", txt):
        params = " ".join(m.group(2).split())
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_signatures_match_the_header_arity(lib):
    """Every declared call is bound with as many arguments as its prototype
    has, and the binding binds nothing the header does not declare."""
    ar = _header_arities()
    assert set(ar) == set(binding.header_functions())
    for name, n in ar.items():
        fn = getattr(lib, name)
        assert fn.argtypes is not None, name
        assert len(fn.argtypes) == n, (name, len(fn.argtypes), n)
    bound = {k for k in vars(lib) if k.startswith("ibl_")}     # the functions the binding set up
    assert bound and bound <= set(ar), bound - set(ar)
