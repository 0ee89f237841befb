"""The C-ABI library builds, loads and exports every symbol its header declares.

CPU-only: no compute call is made (there may be no GPU here).
"""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib_path():
    import __graft_entry__ as ge
    b = ge._build_module()
    if not os.path.exists(b.LIB):
        b.build()
    return b.LIB


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(sp_[a-z0-9_]+)\s*\(", txt))
    return names


def test_header_declares_the_entry_points():
    names = declared_symbols()
    for n in ("sp_step", "sp_jvp", "sp_vjp", "sp_newton_gmres", "sp_set_base", "sp_create"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(_lib_path())
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_export():
    _lib_path()
    import paper_1804_05087_gb300 as sp
    assert set(sp.EXPORTS) == declared_symbols()


def test_create_rejects_bad_sizes_without_a_gpu_call():
    _lib_path()
    import paper_1804_05087_gb300 as sp
    import pytest
    for bad in (sp.Config(10, 33, 16), sp.Config(16, 32, 16), sp.Config(16, 33, 14)):
        with pytest.raises(sp.SpError) as e:
            sp.Context(bad)
        assert e.value.status == 1
