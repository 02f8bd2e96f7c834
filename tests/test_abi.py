"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/kbl.h declares (no compute calls: this runs without a GPU)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "kbl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kbl_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2407_20966_gb300 import build, kbl
    build.build()
    return kbl.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    from paper_2407_20966_gb300 import kbl
    assert sorted(kbl.exported_symbols()) == _declared()


def test_config_defaults_follow_the_paper(lib):
    from paper_2407_20966_gb300 import kbl
    cfg = kbl.KblConfig()
    assert lib.kbl_config_default(C.byref(cfg), 2, 3) == kbl.OK
    assert (cfg.dim, cfg.p, cfg.nu[0], cfg.nu[1]) == (2, 3, 32, 32)   # Sec. 5: 32^2 in 2D
    assert (cfg.k, cfg.r_fac, cfg.eps) == (4.0, 1e-3, 1e-13)          # Sec. 5, Eq. 40, Eq. 37
    assert (cfg.rho_floor, cfg.p_floor, cfg.gamma) == (1e-12, 1e-12, 1.4)
    assert lib.kbl_config_default(C.byref(cfg), 3, 3) == kbl.EINVAL
    assert lib.kbl_config_default(C.byref(cfg), 2, 0) == kbl.EINVAL


def test_invalid_configs_rejected_before_any_device_call(lib):
    from paper_2407_20966_gb300 import kbl
    cfg = kbl.KblConfig()
    lib.kbl_config_default(C.byref(cfg), 2, 3)
    h = C.c_void_p()
    bad = []
    for field, val in (("nu", (65, 65)), ("nu", (17, 33)), ("gamma", 1.0), ("r_fac", 1.0), ("k", 0.0),
                       ("precision", 7), ("flux", 3), ("quadrature", 2),
                       ("quadrature", 1),    # 31 intervals: no coarser grid for Romberg
                       ("stencil", 1),       # the wider stencil is 1D only
                       ("stencil", 2), ("eps_rule", 2), ("uncoupled", 2)):
        c2 = kbl.KblConfig()
        C.pointer(c2)[0] = cfg
        if field == "nu":
            c2.nu[0], c2.nu[1] = val
        else:
            setattr(c2, field, val)
        bad.append(lib.kbl_create(C.byref(h), C.byref(c2), None))
    assert all(st == kbl.EINVAL for st in bad)
    assert lib.kbl_destroy(None) == kbl.EINVAL
    # the triangle mesh refuses orders outside {1, 2} and 1D configurations before any device call
    t = C.c_void_p()
    tri = kbl.KblConfig()
    lib.kbl_config_default(C.byref(tri), 2, 3)
    assert lib.kbl_tri_create(C.byref(t), C.byref(tri), 0, None, None, None, 0, None, None) == kbl.EINVAL
    lib.kbl_config_default(C.byref(tri), 1, 2)
    assert lib.kbl_tri_create(C.byref(t), C.byref(tri), 0, None, None, None, 0, None, None) == kbl.EINVAL
    rs, w = (C.c_double * 12)(), (C.c_double * 6)()
    assert lib.kbl_tri_points(3, rs, w) == kbl.EINVAL


def test_triangle_points_on_the_host(lib):
    """kbl_tri_points runs on the host: the 3- and 6-point rules, interior, weights summing to the
    area, exact to degree 2p."""
    import numpy as np
    from paper_2407_20966_gb300 import kbl
    for p in (1, 2):
        rs, w = kbl.tri_points(p)
        assert abs(w.sum() - 0.5) < 1e-15 and (w > 0).all()
        assert (1 - rs.sum(axis=1)).min() > 0 and rs.min() > 0
        for i in range(2 * p + 1):
            for j in range(2 * p + 1 - i):
                from math import factorial
                exact = factorial(i) * factorial(j) / factorial(i + j + 2)
                assert abs((w * rs[:, 0] ** i * rs[:, 1] ** j).sum() - exact) < 1e-15


def test_product_path_has_no_cpu_fallback():
    """The package never imports the CPU checker."""
    pkg = os.path.join(ROOT, "paper_2407_20966_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
