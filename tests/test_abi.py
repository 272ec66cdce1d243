"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every entry point that include/sp.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(sp_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2506_23917_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("sp_init", "sp_step", "sp_moments", "sp_free", "sp_set_particles"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    import paper_2506_23917_gb300 as sp
    assert set(sp.SYMBOLS) <= set(_declared())


def test_status_strings(libpath):
    lib = ctypes.CDLL(libpath)
    lib.sp_status_str.restype = ctypes.c_char_p
    assert lib.sp_status_str(0) == b"ok"
    assert lib.sp_status_str(-3) == b"capacity exceeded"


def test_config_struct_layout_matches_oracle():
    import oracle
    import paper_2506_23917_gb300 as sp
    assert ctypes.sizeof(sp.SpConfig) == ctypes.sizeof(oracle.OrConfig)
    assert [f[0] for f in sp.SpConfig._fields_] == [f[0] for f in oracle.OrConfig._fields_]
