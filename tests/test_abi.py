"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"\b(molgw_\w+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2210_17093_gb300 import build, native
    build.build()
    return native.load()


def test_exports_every_declared_symbol(lib):
    from paper_2210_17093_gb300 import native
    decl = declared_symbols()
    assert decl, "no declarations found"
    assert decl == set(native.EXPORTS), decl ^ set(native.EXPORTS)
    for name in decl:
        assert hasattr(lib, name), name


def test_status_strings(lib):
    assert lib.molgw_b200_status_string(0) == b"ok"
    assert lib.molgw_b200_status_string(-5).startswith(b"eigensolver")
    assert lib.molgw_b200_status_string(123) == b"unknown status"


def test_create_rejects_bad_opts_without_touching_the_device(lib):
    import ctypes
    from paper_2210_17093_gb300 import native
    h = ctypes.c_void_p()
    assert lib.molgw_b200_create(None, ctypes.byref(h)) == -1
    o = native.Opts()
    o.struct_size = 3           # wrong struct size
    o.max_mols = 1
    o.eta = 1e-3
    assert lib.molgw_b200_create(ctypes.byref(o), ctypes.byref(h)) == -1
    assert h.value is None
    assert lib.molgw_b200_destroy(None) == 0


def test_context_setters_reject_a_null_context_without_touching_the_device(lib):
    assert lib.molgw_b200_set_panel_matvec(None, 0) == -1
    assert lib.molgw_b200_set_panel_matvec(None, 3) == -1
    assert lib.molgw_b200_set_wait_limits(None, -1, -1) == -1
    assert lib.molgw_b200_inject_fault(None, -6) == -1


def test_no_cpu_fallback(lib):
    """Without a usable CUDA device the product path raises; a missing library raises on load."""
    import torch
    from paper_2210_17093_gb300 import Context, MolgwError, native
    with pytest.raises(RuntimeError, match="not built"):
        saved, native._lib = native._lib, None
        try:
            native.load(os.path.join(ROOT, "no_such_library.so"))
        finally:
            native._lib = saved
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: covered by the gpu tests")
    with pytest.raises(MolgwError) as e:
        Context()
    assert e.value.code == -4          # MOLGW_E_CUDA
