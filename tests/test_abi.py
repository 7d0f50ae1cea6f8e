"""C ABI checks that need no GPU: the library builds for sm_103a, loads, and
exports every function declared in include/rve.h; the binding declares them all."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "rve.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


@pytest.fixture(scope="module")
def lib():
    from paper_1610_03484_gb300 import _build
    _build.build()
    import paper_1610_03484_gb300 as pkg
    return pkg.load_library()


def test_header_parses():
    names = header_functions()
    for must in ("rve_mesh_load", "rve_set_materials", "rve_set_bc", "rve_homogenise",
                 "macro_update_gauss_points"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), f"librve.so does not export {name}"


def test_binding_covers_header(lib):
    import paper_1610_03484_gb300 as pkg
    assert sorted(pkg.exported_symbols()) == header_functions()


def test_no_device_is_reported_not_faked(lib):
    # Without a GPU the context must fail loudly, never fall back to the CPU.
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    import paper_1610_03484_gb300 as pkg
    with pytest.raises(pkg.RveError) as e:
        pkg.Context()
    assert e.value.code == -7


def test_strerror(lib):
    assert lib.rve_strerror(-2) == b"bad mesh"
    assert lib.rve_strerror(0) == b"ok"
