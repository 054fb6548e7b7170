"""Rounding floor of the oracle, per evolved variable.  TEST INFRASTRUCTURE ONLY (the
parity tests and the smoke check use it to set their bar; no GPU).

A right-hand side of this system is, for several components, a small residue of large
cancelling terms (the metric of a stationary Kerr-Schild slice, the phi derivative of a
flux that is constant in phi up to small noise): no FP64 evaluation can fix such a
component to 1e-11 of its own size.  The floor measures how far rounding alone moves each
component: the oracle is evaluated again with the result of every stage of its
computation -- the state, the metric, the primitive recovery, the fluxes, the
stress-energy tensor and its 3+1 parts, and every spectral derivative -- multiplied by
(1 + eps xi), xi uniform in [-1, 1) and eps = 2^-52 (one more rounding per stage), and the
largest relative change of each component over a few draws, max |R'_v - R_v| / max |R_v|,
is that component's floor.  A spectral derivative is a dot product: its FP64 value
carries an error of the order of the unit roundoff times sum_j |D_ij| |u_j|, the scale of
its terms rather than of its result (Higham, "Accuracy and Stability of Numerical
Algorithms", section 3.1), which matters where the terms cancel; so each derivative's
result also moves by eps xi (max_i sum_j |D_ij|) max_j |u_j| over its line (one rounding
at the scale of its largest terms).  The GPU path computes the same stages in another
order (matrices instead of coefficient transforms, Newton instead of bisection, fused
products), so its rounding is of this kind; parity tests take max(tol, KAPPA floor_v) of
max |R_v| as the bar.  The mixed-precision modes round their FP32 stages at 2^-23: the
same measurement at that unit gives their floor.
"""
from __future__ import annotations

import contextlib

import numpy as np

from oracle import solver as so
from oracle import valencia as va

EPS64 = 2.0 ** -52    # FP64 stages (twice the unit roundoff: a rounding either way)
EPS32 = 2.0 ** -23    # FP32 stages of the mixed modes
KAPPA = 10.0          # bar = max(tol, KAPPA x floor) of max |ref_v|


def _jitter(rng, x, eps):
    if isinstance(x, np.ndarray) and x.dtype.kind == "f":
        return x * (1.0 + eps * rng.uniform(-1.0, 1.0, x.shape))
    return x


def _wrap(rng, fn, eps):
    def inner(*a, **k):
        out = fn(*a, **k)
        if isinstance(out, tuple):
            return tuple(_jitter(rng, o, eps) for o in out)
        return _jitter(rng, out, eps)
    return inner


def _row_abs_sums(grid, name, orig):
    """max_i sum_j |D_ij| of the grid's derivative operator along one direction (per
    element for r), from the operator applied to unit impulses; cached on the grid."""
    cache = grid.__dict__.setdefault("_row_abs_sums", {})
    if name in cache:
        return cache[name]
    E, nr, nt, npf = grid.shape
    if name == "d_r":
        u = np.zeros((nr, E, nr, 1, 1))
        for k in range(nr):
            u[k, :, k] = 1.0
        out = orig(grid, u)                       # out[k, e, i] = D_e[i, k]
        val = np.abs(out[:, :, :, 0, 0]).sum(axis=0).max(axis=1)        # per element
    elif name == "d_t":
        if grid.fourier_theta:
            # the double-Fourier extension couples the lines at phi and phi + pi: impulses
            # on both lines of one pair, either parity
            u = np.zeros((2 * nt, 1, 1, nt, 2))
            for k in range(nt):
                u[k, 0, 0, k, 0] = 1.0
                u[nt + k, 0, 0, k, 1] = 1.0
            val = 0.0
            for par in (1.0, -1.0):
                out = orig(grid, u, par)
                val = max(val, float(np.abs(out[:, 0, 0, :, 0]).sum(axis=0).max()))
        else:
            u = np.zeros((nt, 1, 1, nt, 1))
            for k in range(nt):
                u[k, 0, 0, k, 0] = 1.0
            val = float(np.abs(orig(grid, u)[:, 0, 0, :, 0]).sum(axis=0).max())
    else:
        u = np.zeros((npf, 1, 1, 1, npf))
        for k in range(npf):
            u[k, 0, 0, 0, k] = 1.0
        val = float(np.abs(orig(grid, u)[:, 0, 0, 0, :]).sum(axis=0).max())
    cache[name] = val
    return val


def _term_scale(grid, name, u, orig):
    """(max_i sum_j |D_ij|) max_j |u_j| over every line of u along the direction."""
    rs = _row_abs_sums(grid, name, orig)
    a = np.abs(u)
    if name == "d_r":
        return a.max(axis=-3, keepdims=True) * np.asarray(rs).reshape((-1, 1, 1, 1))
    if name == "d_t":
        m = a.max(axis=-2, keepdims=True)
        if grid.fourier_theta:                    # the partner line at phi + pi
            m = np.maximum(m, np.roll(m, m.shape[-1] // 2, axis=-1))
        return m * rs
    return a.max(axis=-1, keepdims=True) * rs


def _wrap_deriv(rng, name, orig, eps):
    def inner(grid, u, *a, **k):
        out = orig(grid, u, *a, **k)
        sc = _term_scale(grid, name, u, orig)
        return _jitter(rng, out, eps) + eps * rng.uniform(-1.0, 1.0, out.shape) * sc
    return inner


@contextlib.contextmanager
def rounded_stages(rng, eps=EPS64):
    """Every stage of the oracle's right-hand side rounds once more (see module doc)."""
    saved = []

    def patch(obj, name, wrapped):
        saved.append((obj, name, getattr(obj, name)))
        setattr(obj, name, wrapped)

    patch(so, "metric_from_bssn", _wrap(rng, so.metric_from_bssn, eps))
    patch(va, "con2prim", _wrap(rng, va.con2prim, eps))
    patch(va, "fluxes", _wrap(rng, va.fluxes, eps))
    patch(va, "stress_energy", _wrap(rng, va.stress_energy, eps))
    patch(va, "matter_3p1", _wrap(rng, va.matter_3p1, eps))
    for m in ("d_r", "d_t", "d_p"):
        patch(so.Grid, m, _wrap_deriv(rng, m, getattr(so.Grid, m), eps))
    try:
        yield
    finally:
        for obj, name, fn in reversed(saved):
            setattr(obj, name, fn)


def floor(fn, U, trials=3, seed=12345, eps=EPS64, ref=None):
    """(reference result, per-variable floor) of fn(U) -> array [nv, ...]: the reference
    is fn(U) as it stands (or `ref`, when the caller has it); each trial evaluates fn on
    the state rounded once more with every oracle stage rounded once more too (relative
    perturbations eps xi, xi uniform in [-1, 1))."""
    if ref is None:
        ref = fn(U)
    rng = np.random.default_rng(seed)
    nv = ref.shape[0]
    m = np.abs(ref).reshape(nv, -1).max(1)
    fl = np.zeros(nv)
    for _ in range(trials):
        with rounded_stages(rng, eps):
            alt = fn(_jitter(rng, U, eps))
        d = np.abs(alt - ref).reshape(nv, -1).max(1)
        fl = np.maximum(fl, np.where(m > 0, d / np.where(m > 0, m, 1.0), np.where(d > 0, np.inf, 0.0)))
    return ref, fl
