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


@pytest.mark.parametrize("which,field,value", [
    ("g", "n_elem", 0), ("g", "n_r", 3), ("g", "n_r", 65), ("g", "n_theta", 3),
    ("g", "n_theta", 129), ("g", "n_phi", 2), ("g", "n_phi", 130), ("g", "n_phi", 17),
    ("g", "r_min", 0.0), ("g", "r_min", -1.0), ("g", "r_max", 1.0), ("g", "theta_min", -0.1),
    ("g", "theta_max", 3.2), ("g", "elem_map", 2), ("g", "theta_basis", 2),
    ("p", "M", 0.0), ("p", "a", 1.0), ("p", "a", -1.0), ("p", "gamma_eos", 1.0),
    ("p", "rho_atm", 0.0), ("p", "eps_atm", -1.0),
    ("o", "integrator", 2), ("o", "gauge", 2), ("o", "cfl", 0.0), ("o", "c2p_maxit", 0),
    ("o", "c2p_tol", 0.0), ("o", "filter", 64), ("o", "filter", -1), ("o", "contraction", 2),
    ("o", "coupling", 2), ("o", "glm", 2), ("o", "dealias23_theta", 2), ("o", "c2p_lambda", -0.1),
    ("o", "c2p_lambda", 1.5), ("o", "c2p_lambda", float("nan")),
])
def test_invalid_parameters_rejected_before_device_work(lib, which, field, value):
    """Each parameter outside its documented range gives GRMHD_EINVAL from grmhd_create and
    from grmhd_batch_create, before any device call (this host has no GPU)."""
    import paper_2508_18221_gb300 as pkg
    g, p, o = pkg.defaults()
    if (which, field) == ("g", "r_max"):
        g.r_min = 2.0
    setattr({"g": g, "p": p, "o": o}[which], field, value)
    h = ctypes.c_void_p()
    assert lib.grmhd_create(ctypes.byref(g), ctypes.byref(p), ctypes.byref(o), None,
                            ctypes.byref(h)) == pkg.GRMHD_EINVAL
    assert not h.value
    assert lib.grmhd_batch_create(1, ctypes.byref(g), ctypes.byref(p), ctypes.byref(o), None,
                                  ctypes.byref(h)) == pkg.GRMHD_EINVAL


def test_fourier_theta_needs_the_whole_sphere(lib):
    import paper_2508_18221_gb300 as pkg
    g, p, o = pkg.defaults()
    g.theta_basis = 1
    g.theta_min, g.theta_max = 0.1, 3.0
    h = ctypes.c_void_p()
    assert lib.grmhd_create(ctypes.byref(g), ctypes.byref(p), ctypes.byref(o), None,
                            ctypes.byref(h)) == pkg.GRMHD_EINVAL


def test_empty_and_oversized_inputs_rejected(lib):
    """Zero instances, zero nodes and a node count above the no-allocation limit are
    argument errors, reported before any device call."""
    import paper_2508_18221_gb300 as pkg
    g, p, o = pkg.defaults()
    h = ctypes.c_void_p()
    assert lib.grmhd_batch_create(0, ctypes.byref(g), ctypes.byref(p), ctypes.byref(o), None,
                                  ctypes.byref(h)) == pkg.GRMHD_EINVAL
    dt = ctypes.c_double()
    buf = (ctypes.c_double * 1)()
    for n in (0, -1, 16_777_217):
        assert lib.grmhd_cfl_dt_noalloc(buf, n, 0.1, 0.3, ctypes.byref(dt), None) == pkg.GRMHD_EINVAL
    assert lib.grmhd_cfl_dt_noalloc(buf, 10, 0.0, 0.3, ctypes.byref(dt), None) == pkg.GRMHD_EINVAL
    assert lib.grmhd_cfl_dt_noalloc(buf, 10, 0.1, -0.3, ctypes.byref(dt), None) == pkg.GRMHD_EINVAL


def test_warning_status_of_the_tf32_mode(lib):
    """Positive statuses are warnings (the call did its work); the TF32 mode's warning
    names the mode and the recommended one, and the binding turns it into a Python
    warning instead of an error."""
    import warnings
    import paper_2508_18221_gb300 as pkg
    msg = lib.grmhd_strerror(pkg.GRMHD_WPRECISION).decode()
    assert pkg.GRMHD_WPRECISION > 0 and "TF32" in msg and "precision 1" in msg
    with warnings.catch_warnings(record=True) as w:
        warnings.simplefilter("always")
        pkg.check(pkg.GRMHD_WPRECISION)
    assert len(w) == 1 and "TF32" in str(w[0].message)
    with pytest.raises(pkg.GrmhdError):
        pkg.check(pkg.GRMHD_EINVAL)


def test_tuning_table_entries(lib):
    """The contraction tuning table (host side): entries in range are kept and read back,
    entries outside the documented ranges are refused, 0 restores the untuned default."""
    import paper_2508_18221_gb300 as pkg
    assert lib.grmhd_tune_set(1, 33, 0, 2) == pkg.GRMHD_OK
    assert lib.grmhd_tune_get(1, 33, 0) == 2
    assert lib.grmhd_tune_get(1, 33, 1) == 0          # the filter class is separate
    assert lib.grmhd_tune_set(1, 33, 0, 0) == pkg.GRMHD_OK
    assert lib.grmhd_tune_get(1, 33, 0) == 0
    for args in ((3, 24, 0, 1), (0, 1, 0, 1), (0, 129, 0, 1), (0, 24, 2, 1), (0, 24, -1, 1), (0, 24, 0, 3),
                 (0, 24, 0, -1)):
        assert lib.grmhd_tune_set(*args) == pkg.GRMHD_EINVAL, args
    assert lib.grmhd_tune_get(0, 24, 2) == pkg.GRMHD_EINVAL
