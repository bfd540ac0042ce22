"""The C-ABI library builds, loads without a GPU and exports every entry point of include/crk.h."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "crk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("defined",)))


@pytest.fixture(scope="module")
def lib():
    from paper_2310_16122_gb300.build import build_library
    from paper_2310_16122_gb300 import native

    build_library()
    return native.lib()


def test_header_declares_entry_points():
    names = header_functions()
    for must in ("crk_build_leaves", "crk_geometry", "crk_corrections", "crk_hydro", "grav_short",
                 "grav_short_adjoint", "crk_geometry_adjoint"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2310_16122_gb300 import native

    for name in header_functions():
        assert hasattr(lib, name), name
        assert name in native.SIGNATURES, f"binding lacks {name}"


def test_version_string(lib):
    assert lib.crk_version().decode().startswith("libcrk")
