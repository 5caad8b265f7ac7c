"""The C-ABI library loads and exports every symbol include/chhs.h declares.

CPU-only: no compute call is made (there may be no GPU here).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(chhs_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1611_02967_gb300 import build, chhs
    build.build()
    return ctypes.CDLL(chhs.LIB_PATH)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "chhs_create" in names and "chhs_step" in names
    assert "chhs_mass" in names and "chhs_energy" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    from paper_1611_02967_gb300 import chhs
    assert sorted(chhs.EXPORTS) == sorted(n for n in _declared() if n in chhs.EXPORTS)
    assert set(_declared()) >= set(chhs.EXPORTS)


def test_host_only_calls(lib):
    # calls that touch no device: defaults and the workspace size
    from paper_1611_02967_gb300 import chhs
    o = chhs.default_opts()
    assert (o.nu1, o.nu2, o.coarsest, o.tol, o.precision) == (2, 2, 2, 1e-10, 0)
    assert chhs.workspace_bytes((512, 512)) > 0
    assert chhs.workspace_bytes((128, 128, 128)) > chhs.workspace_bytes((512, 512))
    bad = (ctypes.c_int * 3)(0, 16, 1)
    assert chhs.lib().chhs_workspace_bytes(2, bad, None) == 0
    assert chhs.lib().chhs_workspace_bytes(4, (ctypes.c_int * 3)(8, 8, 8), None) == 0
