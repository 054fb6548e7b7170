"""The rounding floor that sets the parity bar (oracle/rounding.py), checked on the CPU:
it is at the unit roundoff for a component that is not a residue (the lapse's right-hand
side -2 alpha K + beta^i d_i alpha of the Kerr-Schild slice), far above 1e-11 for a pure
cancellation residue (the metric's right-hand side of the stationary vacuum Kerr-Schild
slice under the frozen gauge, analytically zero), it grows in proportion to the
perturbation's unit, and the oracle's own functions are restored afterwards."""
import numpy as np

from oracle import rounding
from oracle import solver as so
from oracle import valencia as va
from workloads import config


def _small(**kw):
    return so.workload_state(config("c1", n_elem=2, n_r=8, n_theta=8, n_phi=8), **kw)


def test_floor_separates_residues_from_plain_components():
    # 12 x 12 x 16 nodes: the stationary metric's right-hand side is a rounding-level
    # residue there (on coarser grids the truncation residue dominates it)
    g, p, U = so.workload_state(config("c1"), gauge=1)
    U[so.I_D:] = 0.0                                    # vacuum: no matter terms
    U[so.I_D] = 1e-30
    ref, fl = rounding.floor(lambda X: so.rhs(X, g, p), U, trials=2)
    # gammatilde_ij, phi: residues of O(1) terms, the exact value is zero
    assert fl[so.I_GT:so.I_GT + 6].min() > 1e-10 and fl[so.I_PHI] > 1e-9
    g2, p2, U2 = _small()
    ref2, fl2 = rounding.floor(lambda X: so.rhs(X, g2, p2), U2, trials=2)
    assert fl2[so.I_ALPHA] < 1e-14                      # -2 alpha K + beta d alpha


def test_floor_scales_with_the_unit_and_restores_the_oracle():
    g, p, U = _small()
    fn = lambda X: so.rhs(X, g, p)  # noqa: E731
    before = (so.metric_from_bssn, va.con2prim, va.fluxes, so.Grid.d_r)
    _, f64 = rounding.floor(fn, U, trials=2)
    _, f32 = rounding.floor(fn, U, trials=2, eps=rounding.EPS32)
    assert (so.metric_from_bssn, va.con2prim, va.fluxes, so.Grid.d_r) == before
    ok = f64 > 0
    ratio = np.median(f32[ok] / f64[ok])
    assert 2.0 ** 26 < ratio < 2.0 ** 32                # 2^29 nominal
    # the reference result is the oracle's, untouched
    np.testing.assert_array_equal(fn(U), so.rhs(U, g, p))
