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


def test_default_options_agree_with_header_binding_and_bench(lib):
    """rve_default_options (no GPU needed) gives the defaults the header documents,
    the Python binding's keyword defaults repeat them, and the struct layouts agree."""
    import inspect

    import ctypes as C
    import paper_1610_03484_gb300 as pkg
    o = pkg.default_options()
    assert C.sizeof(o) == C.sizeof(pkg.Options)
    documented = {}
    hdr = open(os.path.join(ROOT, "include", "rve.h")).read()
    body = hdr[hdr.index("typedef struct rve_options"):hdr.index("} rve_options;")]
    for name, default in re.findall(r"\b(\w+);\s*/\*(?:(?!\*/).)*?\(default ([0-9.e+-]+)\)", body, flags=re.S):
        documented[name] = float(default)
    for name in ("device", "rtol", "max_iter", "inner_rtol", "max_refine"):
        assert name in documented, name
    for name, v in documented.items():
        assert getattr(o, name) == pytest.approx(v), name
    # warm_start's default is documented as "4 (default)" inside its list of modes
    assert re.search(r"4 \(default\)", body[body.index("warm_start"):])
    assert o.warm_start == 4 and o.precision == pkg.PREC_FP64 and o.deterministic == 0
    sig = inspect.signature(pkg.Context.__init__).parameters
    for name in ("rtol", "max_iter", "inner_rtol", "max_refine", "check_every", "batch", "warm_start"):
        assert sig[name].default == getattr(o, name), name
    import bench
    assert bench.WARM_START == o.warm_start
