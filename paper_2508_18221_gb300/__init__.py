"""GB300 (sm_103a) coupled BSSN-Valencia spectral right-hand side.

Thin ctypes binding of the C ABI declared in include/grmhd.h (libgrmhd.so, built in
tree by `paper_2508_18221_gb300._build.build()`).  Argument marshalling only: every
step of the right-hand side runs in the library's CUDA kernels.  PyTorch, when used,
provides device memory and the CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgrmhd.so")

GRMHD_OK, GRMHD_EINVAL, GRMHD_ENOMEM, GRMHD_ECUDA = 0, -1, -2, -3
GRMHD_ENAN, GRMHD_ETIMEOUT, GRMHD_EUNSUPPORTED = -4, -5, -6
GRMHD_WPRECISION = 1          # warning: created, but the TF32 mode misses the mixed bar
NV, NPRIM, NDIAG = 32, 7, 8


class Grid(C.Structure):
    _fields_ = [("n_elem", C.c_int), ("r_min", C.c_double), ("r_max", C.c_double),
                ("elem_map", C.c_int), ("n_r", C.c_int), ("n_theta", C.c_int),
                ("n_phi", C.c_int), ("theta_min", C.c_double), ("theta_max", C.c_double),
                ("theta_basis", C.c_int)]


class Physics(C.Structure):
    _fields_ = [("M", C.c_double), ("a", C.c_double), ("gamma_eos", C.c_double),
                ("rho_atm", C.c_double), ("eps_atm", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("integrator", C.c_int), ("evolve_metric", C.c_int),
                ("gauge", C.c_int), ("eta", C.c_double), ("cfl", C.c_double),
                ("filter", C.c_int), ("filt_alpha", C.c_double), ("filt_p", C.c_double),
                ("dealias23_phi", C.c_int), ("c2p_maxit", C.c_int), ("c2p_tol", C.c_double),
                ("contraction", C.c_int), ("coupling", C.c_int), ("glm", C.c_int),
                ("glm_ch", C.c_double), ("glm_tau", C.c_double), ("dealias23_theta", C.c_int),
                ("c2p_lambda", C.c_double)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
# exported symbol -> (restype, argtypes)
SIGNATURES = {
    "grmhd_defaults": (C.c_int, [C.POINTER(Grid), C.POINTER(Physics), C.POINTER(Opts)]),
    "grmhd_create": (C.c_int, [C.POINTER(Grid), C.POINTER(Physics), C.POINTER(Opts), _P,
                               C.POINTER(_P)]),
    "grmhd_destroy": (C.c_int, [_P]),
    "grmhd_num_points": (C.c_longlong, [_P]),
    "grmhd_num_vars": (C.c_int, [_P]),
    "grmhd_coords": (C.c_int, [_P, _P, _P, _P]),
    "grmhd_init_prims": (C.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "grmhd_set_state": (C.c_int, [_P, _P, C.c_int]),
    "grmhd_get_state": (C.c_int, [_P, _P, C.c_int]),
    "grmhd_rhs": (C.c_int, [_P, _P, C.c_int]),
    "grmhd_con2prim": (C.c_int, [_P, _P, C.c_int, C.POINTER(C.c_longlong)]),
    "grmhd_step": (C.c_int, [_P, C.c_double, C.c_int, _D]),
    "grmhd_cfl_dt": (C.c_int, [_P, _D]),
    "grmhd_diag": (C.c_int, [_P, _D]),
    "grmhd_launch_count": (C.c_longlong, [_P]),
    "grmhd_kernel_times": (C.c_int, [_P, C.c_int, _D, _D, _D, C.c_int]),
    "grmhd_batch_create": (C.c_int, [C.c_int, C.POINTER(Grid), C.POINTER(Physics),
                                     C.POINTER(Opts), _P, C.POINTER(_P)]),
    "grmhd_batch_num_groups": (C.c_int, [_P]),
    "grmhd_batch_num_points": (C.c_longlong, [_P, C.c_int]),
    "grmhd_batch_num_vars": (C.c_int, [_P, C.c_int]),
    "grmhd_batch_coords": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "grmhd_batch_init_prims": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, _P, _P]),
    "grmhd_batch_set_state": (C.c_int, [_P, C.c_int, _P, C.c_int]),
    "grmhd_batch_get_state": (C.c_int, [_P, C.c_int, _P, C.c_int]),
    "grmhd_batch_step": (C.c_int, [_P, _D, C.c_int]),
    "grmhd_batch_cfl_dt": (C.c_int, [_P, _D]),
    "grmhd_batch_launch_count": (C.c_longlong, [_P]),
    "grmhd_batch_destroy": (C.c_int, [_P]),
    "grmhd_batch_last_error": (C.c_char_p, [_P]),
    "grmhd_xcts_init": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, C.c_int, C.c_double, _P, _P, _P]),
    "grmhd_tune_contractions": (C.c_int, [_P, C.c_int, C.c_int, _P, _P]),
    "grmhd_tune_set": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int]),
    "grmhd_tune_get": (C.c_int, [C.c_int, C.c_int, C.c_int]),
    "grmhd_debug_deriv": (C.c_int, [_P, _P, _P, C.c_int, C.c_int]),
    "grmhd_debug_theta": (C.c_int, [_P, _P, _P, C.c_int, C.POINTER(C.c_int), C.c_int]),
    "grmhd_debug_wait_timeout": (C.c_int, [_P]),
    "grmhd_cfl_dt_noalloc": (C.c_int, [_P, C.c_longlong, C.c_double, C.c_double, _P, _P]),
    "grmhd_strerror": (C.c_char_p, [C.c_int]),
    "grmhd_last_error": (C.c_char_p, [_P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libgrmhd.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run paper_2508_18221_gb300._build.build() "
                           "(nvcc, sm_103a); this package has no CPU implementation")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class GrmhdError(RuntimeError):
    pass


def check(status, ctx=None):
    if status > 0:            # a warning: the call did its work
        import warnings
        warnings.warn(load().grmhd_strerror(status).decode(), RuntimeWarning, stacklevel=3)
        return
    if status != GRMHD_OK:
        lib = load()
        msg = lib.grmhd_strerror(status).decode()
        if ctx:
            msg += ": " + lib.grmhd_last_error(ctx).decode()
        raise GrmhdError(f"grmhd status {status}: {msg}")


def defaults():
    g, p, o = Grid(), Physics(), Opts()
    check(load().grmhd_defaults(C.byref(g), C.byref(p), C.byref(o)))
    return g, p, o


def _ptr(x):
    """Raw pointer of a torch tensor / numpy array / int."""
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(type(x))


class Context:
    """One solver instance (owns its device buffers); methods map 1:1 to the C calls."""

    def __init__(self, grid: Grid, phys: Physics, opts: Opts, stream: int = 0):
        self.lib = load()
        h = C.c_void_p()
        check(self.lib.grmhd_create(C.byref(grid), C.byref(phys), C.byref(opts),
                                    C.c_void_p(stream or None), C.byref(h)))
        self.h = h
        self.grid, self.phys, self.opts = grid, phys, opts
        self.n_points = int(self.lib.grmhd_num_points(h))
        self.nv = int(self.lib.grmhd_num_vars(h))

    def close(self):
        if self.h:
            self.lib.grmhd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st):
        check(st, self.h)

    def coords(self):
        import numpy as np
        r, t, p = (np.empty(self.n_points) for _ in range(3))
        self._chk(self.lib.grmhd_coords(self.h, _ptr(r), _ptr(t), _ptr(p)))
        return r, t, p

    def init_prims(self, rho, p, vr, vth, vph, A_phi):
        import numpy as np
        arrs = [np.ascontiguousarray(a, dtype=np.float64).ravel()
                for a in (rho, p, vr, vth, vph, A_phi)]
        self._chk(self.lib.grmhd_init_prims(self.h, *[_ptr(a) for a in arrs]))

    def xcts_init(self, rho, p, vr, vth, vph, A_phi, iters: int = 20, tol: float = 0.0):
        """Approximate XCTS initial data (grmhd_xcts_init); returns (psi, changes, stats)"""
        import numpy as np
        arrs = [np.ascontiguousarray(a, dtype=np.float64).ravel()
                for a in (rho, p, vr, vth, vph, A_phi)]
        psi = np.empty(self.n_points)
        changes = np.zeros(iters)
        stats = np.zeros(3)
        self._chk(self.lib.grmhd_xcts_init(self.h, *[_ptr(a) for a in arrs], int(iters), float(tol),
                                           _ptr(psi), _ptr(changes), _ptr(stats)))
        return psi, changes[:int(stats[2])], stats

    def set_state(self, state, on_device: bool):
        self._chk(self.lib.grmhd_set_state(self.h, _ptr(state), int(on_device)))

    def get_state(self, out, on_device: bool):
        self._chk(self.lib.grmhd_get_state(self.h, _ptr(out), int(on_device)))

    def rhs(self, out, on_device: bool):
        self._chk(self.lib.grmhd_rhs(self.h, _ptr(out), int(on_device)))

    def con2prim(self, out, on_device: bool):
        nf = C.c_longlong(0)
        self._chk(self.lib.grmhd_con2prim(self.h, _ptr(out) if out is not None else None,
                                          int(on_device), C.byref(nf)))
        return int(nf.value)

    def step(self, dt: float, nsteps: int):
        used = C.c_double(0.0)
        self._chk(self.lib.grmhd_step(self.h, float(dt), int(nsteps), C.byref(used)))
        return used.value

    def cfl_dt(self):
        v = C.c_double(0.0)
        self._chk(self.lib.grmhd_cfl_dt(self.h, C.byref(v)))
        return v.value

    def diag(self):
        out = (C.c_double * NDIAG)()
        self._chk(self.lib.grmhd_diag(self.h, out))
        return list(out)

    def launch_count(self):
        return int(self.lib.grmhd_launch_count(self.h))

    KERNEL_CLASSES = ("prep", "d1_r", "d1_theta", "d1_phi", "iface_d1", "d2_r", "d2_theta",
                      "d2_phi", "iface_d2", "rhs", "filter_r", "filter_theta", "filter_phi")

    def kernel_times(self, reps: int = 5):
        """{class: (ms per launch, algorithmic flops per launch, algorithmic bytes)}"""
        n = len(self.KERNEL_CLASSES)
        ms = (C.c_double * n)()
        fl = (C.c_double * n)()
        by = (C.c_double * n)()
        self._chk(self.lib.grmhd_kernel_times(self.h, int(reps), ms, fl, by, n))
        return {k: (ms[i], fl[i], by[i]) for i, k in enumerate(self.KERNEL_CLASSES)}

    def tune_contractions(self, nfields: int = 21, reps: int = 10):
        """Run the contraction autotuner on this context (grmhd_tune_contractions): returns
        {(direction, kind): (ms with one accumulator set, ms with two, chosen sets)}, kind
        "derivative" or "filter"; classes on the FP64 units are left out."""
        ms = (C.c_double * 12)()
        ch = (C.c_int * 6)()
        self._chk(self.lib.grmhd_tune_contractions(self.h, nfields, reps, ms, ch))
        out = {}
        for d in range(3):
            for k, kind in enumerate(("derivative", "filter")):
                if ch[d * 2 + k]:
                    out[(d, kind)] = (ms[(d * 2 + k) * 2], ms[(d * 2 + k) * 2 + 1], int(ch[d * 2 + k]))
        return out

    def debug_deriv(self, src, dst, nfields: int, direction: int):
        self._chk(self.lib.grmhd_debug_deriv(self.h, _ptr(src), _ptr(dst), nfields, direction))

    def debug_wait_timeout(self):
        """status of grmhd_debug_wait_timeout (GRMHD_ETIMEOUT expected)"""
        return int(self.lib.grmhd_debug_wait_timeout(self.h))

    def debug_theta(self, src, dst, parities, filter: bool = False):
        """theta derivative (or theta filter) of len(parities) fields, field f with the
        extension parity parities[f] (Fourier theta basis)"""
        n = len(parities)
        arr = (C.c_int * n)(*[int(x) for x in parities])
        self._chk(self.lib.grmhd_debug_theta(self.h, _ptr(src), _ptr(dst), n, arr, int(filter)))


class Batch:
    """Many independent instances advanced together (grmhd_batch_*)."""

    def __init__(self, structs, stream: int = 0):
        self.lib = load()
        n = len(structs)
        grids = (Grid * n)(*[s[0] for s in structs])
        physs = (Physics * n)(*[s[1] for s in structs])
        opts = (Opts * n)(*[s[2] for s in structs])
        h = C.c_void_p()
        check(self.lib.grmhd_batch_create(n, grids, physs, opts, C.c_void_p(stream or None),
                                          C.byref(h)))
        self.h, self.n = h, n

    def _chk(self, st):
        if st != GRMHD_OK:
            raise GrmhdError(f"grmhd status {st}: {self.lib.grmhd_strerror(st).decode()}: "
                             f"{self.lib.grmhd_batch_last_error(self.h).decode()}")

    def num_groups(self):
        return int(self.lib.grmhd_batch_num_groups(self.h))

    def num_points(self, i):
        return int(self.lib.grmhd_batch_num_points(self.h, i))

    def num_vars(self, i):
        return int(self.lib.grmhd_batch_num_vars(self.h, i))

    def coords(self, i):
        import numpy as np
        n = self.num_points(i)
        r, t, p = (np.empty(n) for _ in range(3))
        self._chk(self.lib.grmhd_batch_coords(self.h, i, _ptr(r), _ptr(t), _ptr(p)))
        return r, t, p

    def init_prims(self, i, rho, p, vr, vth, vph, A_phi):
        import numpy as np
        arrs = [np.ascontiguousarray(a, dtype=np.float64).ravel()
                for a in (rho, p, vr, vth, vph, A_phi)]
        self._chk(self.lib.grmhd_batch_init_prims(self.h, i, *[_ptr(a) for a in arrs]))

    def set_state(self, i, state, on_device: bool):
        self._chk(self.lib.grmhd_batch_set_state(self.h, i, _ptr(state), int(on_device)))

    def get_state(self, i, out, on_device: bool):
        self._chk(self.lib.grmhd_batch_get_state(self.h, i, _ptr(out), int(on_device)))

    def step(self, dts, nsteps: int):
        arr = (C.c_double * self.n)(*[float(x) for x in dts])
        self._chk(self.lib.grmhd_batch_step(self.h, arr, int(nsteps)))

    def cfl_dt(self):
        arr = (C.c_double * self.n)()
        self._chk(self.lib.grmhd_batch_cfl_dt(self.h, arr))
        return list(arr)

    def launch_count(self):
        return int(self.lib.grmhd_batch_launch_count(self.h))

    def close(self):
        if self.h:
            self.lib.grmhd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_structs(cfg, **opt_overrides):
    """grid/physics/options structs for a workload configuration."""
    g, p, o = defaults()
    g.n_elem, g.r_min, g.r_max, g.elem_map = cfg.n_elem, cfg.r_min, cfg.r_max, cfg.elem_map
    g.n_r, g.n_theta, g.n_phi = cfg.n_r, cfg.n_theta, cfg.n_phi
    g.theta_min, g.theta_max = cfg.theta_min, cfg.theta_max
    g.theta_basis = getattr(cfg, "theta_basis", 0)
    p.M, p.a, p.gamma_eos = cfg.M, cfg.a, cfg.gamma_eos
    o.cfl = cfg.cfl
    for k, v in opt_overrides.items():
        setattr(o, k, v)
    return g, p, o
