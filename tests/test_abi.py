"""The C-ABI library loads and exports every function that include/grmhd.h declares
(no GPU needed: nothing is called except the pure host helpers)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "grmhd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(grmhd_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_2508_18221_gb300 as pkg
    if not os.path.exists(pkg.LIB_PATH):
        from paper_2508_18221_gb300 import _build
        _build.build()
    return pkg.load()


def test_exports(lib):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    import paper_2508_18221_gb300 as pkg
    assert sorted(pkg.SIGNATURES) == names


def test_host_only_calls(lib):
    import paper_2508_18221_gb300 as pkg
    g, p, o = pkg.defaults()
    assert g.n_r == 12 and abs(o.filt_alpha - 36.0) < 1e-15 and o.filter == 47
    assert lib.grmhd_strerror(-1) == b"invalid argument"
    # invalid parameters are rejected before any device work
    h = ctypes.c_void_p()
    g.n_phi = 15
    assert lib.grmhd_create(ctypes.byref(g), ctypes.byref(p), ctypes.byref(o), None,
                            ctypes.byref(h)) == pkg.GRMHD_EINVAL
    g.n_phi = 16
    p.a = 1.5
    assert lib.grmhd_create(ctypes.byref(g), ctypes.byref(p), ctypes.byref(o), None,
                            ctypes.byref(h)) == pkg.GRMHD_EINVAL
    p.a = 0.5
    o.precision = 7
    assert lib.grmhd_create(ctypes.byref(g), ctypes.byref(p), ctypes.byref(o), None,
                            ctypes.byref(h)) == pkg.GRMHD_EUNSUPPORTED
    assert lib.grmhd_destroy(None) == pkg.GRMHD_EINVAL
