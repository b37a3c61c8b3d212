"""The C-ABI library builds, loads and exports every function include/pp.h declares (no GPU)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", fn)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(pp_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    import paper_2512_09811_gb300 as pp
    from paper_2512_09811_gb300 import _build

    if not os.path.exists(pp.LIB_PATH):
        _build.build()
    return pp.LIB_PATH


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("pp_create", "pp_sigma", "pp_solve_window", "pp_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_lists_every_symbol():
    import paper_2512_09811_gb300 as pp

    assert sorted(pp.EXPORTS) == declared_functions()


def test_default_options_without_gpu(lib_path):
    import paper_2512_09811_gb300 as pp

    opt = pp.pp_default_options()
    assert opt.order == 2 and opt.block == 8 and opt.res_tol == 1e-7


def test_invalid_create_is_rejected_on_host(lib_path):
    """Argument validation runs before any device call."""
    import numpy as np

    import paper_2512_09811_gb300 as pp

    eps = np.array([0.5, 1.2, 1.0])  # an occupied level above the virtual one
    B = np.zeros((1, 3, 3))
    with pytest.raises(pp.PPError) as e:
        pp.pp_create(2, 1, 1, eps, B)
    assert e.value.status == pp.PP_EINVAL
    eps = np.array([-1.0, np.nan, 1.0])
    with pytest.raises(pp.PPError):
        pp.pp_create(2, 1, 1, eps, B)
