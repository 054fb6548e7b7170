"""Pins of the oracle's Kerr-Schild geometry against closed forms.

Paper: "The Kerr-Schild Metric and 3+1 Decomposition" (line element), the Kerr-Schild
ADM table of the appendix (lapse sqrt(Sigma/(Sigma+2r)), g_thth = Sigma,
g_phph = (r^2 + a^2 + 2 a^2 r sin^2/Sigma) sin^2 at M = 1) and the horizon radius
r_h = M + sqrt(M^2 - a^2).  The oracle extracts alpha, beta, gamma from the 4-metric by
the generic 3+1 split; these closed forms are derived independently.
"""
import os

import numpy as np
import pytest

from oracle import kerr_schild as ks


@pytest.fixture(scope="module")
def pts():
    rng = np.random.default_rng(5)
    r = rng.uniform(1.2, 40.0, 200)
    th = rng.uniform(0.05, np.pi - 0.05, 200)
    return r, th


@pytest.mark.parametrize("a", [0.0, 0.5, 0.94])
def test_adm_closed_forms(pts, a):
    M = 1.0
    r, th = pts
    alpha, beta, gam = ks.adm(M, a, r, th)
    sig = r * r + a * a * np.cos(th) ** 2
    H = M * r / sig
    s2 = np.sin(th) ** 2
    np.testing.assert_allclose(gam[:, 0, 0], 1 + 2 * H, rtol=1e-14)
    np.testing.assert_allclose(gam[:, 0, 2], -a * s2 * (1 + 2 * H), rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(gam[:, 1, 1], sig, rtol=1e-14)
    np.testing.assert_allclose(gam[:, 2, 2], s2 * (sig + a * a * s2 * (1 + 2 * H)), rtol=1e-14)
    np.testing.assert_allclose(gam[:, 0, 1], 0.0)
    np.testing.assert_allclose(ks.det3(gam), sig ** 2 * s2 * (1 + 2 * H), rtol=1e-12)
    np.testing.assert_allclose(alpha, (1 + 2 * H) ** -0.5, rtol=1e-13)
    np.testing.assert_allclose(beta[:, 0], 2 * H / (1 + 2 * H), rtol=1e-12)
    np.testing.assert_allclose(beta[:, 1:], 0.0, atol=1e-14)
    gi = ks.inv3(gam)
    np.testing.assert_allclose(gi[:, 0, 2], a / sig, rtol=1e-11, atol=1e-15)
    np.testing.assert_allclose(gi[:, 2, 2], 1 / (sig * s2), rtol=1e-11)
    np.testing.assert_allclose(gi[:, 1, 1], 1 / sig, rtol=1e-12)
    # sqrt(-g) = alpha sqrt(gamma) = Sigma sin(theta)
    np.testing.assert_allclose(alpha * np.sqrt(ks.det3(gam)), sig * np.sin(th), rtol=1e-12)


def _paper_table():
    path = os.path.join(os.path.dirname(__file__), "golden", "ks_adm_table.txt")
    rows = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            k, v = (x.strip() for x in line.split("|"))
            rows[k] = v
    return rows


@pytest.mark.parametrize("a", [0.5, 0.9])
def test_paper_adm_table(pts, a):
    """Appendix table (M = 1), transcribed in tests/golden/ks_adm_table.txt."""
    r, th = pts
    alpha, beta, gam = ks.adm(1.0, a, r, th)
    env = {"sqrt": np.sqrt, "sin": np.sin, "cos": np.cos, "r": r, "theta": th, "a": a,
           "Sigma": r * r + a * a * np.cos(th) ** 2}
    tab = {k: eval(v, {"__builtins__": {}}, env) for k, v in _paper_table().items()}
    np.testing.assert_allclose(alpha, tab["alpha"], rtol=1e-13)
    np.testing.assert_allclose(beta[:, 1], tab["beta_theta"], atol=1e-15)
    np.testing.assert_allclose(gam[:, 1, 1], tab["g_thth"], rtol=1e-14)
    np.testing.assert_allclose(gam[:, 2, 2], tab["g_phph"], rtol=1e-13)


def test_horizon_radius():
    assert ks.horizon_radius(1.0, 0.0) == 2.0
    np.testing.assert_allclose(ks.horizon_radius(1.0, 0.6), 1.8)
    # g^rr = 0 on the horizon: Delta = r^2 - 2 M r + a^2 = 0
    for a in (0.3, 0.9):
        rh = ks.horizon_radius(1.0, a)
        np.testing.assert_allclose(rh * rh - 2 * rh + a * a, 0.0, atol=1e-14)


def test_schwarzschild_trace_K(pts):
    """a = 0: K = 2 M alpha^3 (1 + 3M/r) / r^2 (ingoing Eddington-Finkelstein slice)."""
    r, th = pts
    M = 1.0
    Kij = ks.extrinsic_curvature(M, 0.0, r, th)
    alpha, _, gam = ks.adm(M, 0.0, r, th)
    K = np.einsum("nij,nij->n", ks.inv3(gam), Kij)
    np.testing.assert_allclose(K, 2 * M * alpha ** 3 * (1 + 3 * M / r) / r ** 2, rtol=1e-12)


def test_bssn_data_consistency(pts):
    r, th = pts
    d = ks.bssn_data(1.0, 0.7, r, th)
    np.testing.assert_allclose(ks.det3(d["gt"]), 1.0, rtol=1e-13)
    # Atilde is trace-free with respect to gammatilde
    tr = np.einsum("nij,nij->n", ks.inv3(d["gt"]), d["At"])
    np.testing.assert_allclose(tr, 0.0, atol=1e-13 * np.abs(d["At"]).max())
    # reconstruct K_ij = e^{4 phi}(Atilde + gammatilde K / 3)
    e4 = np.exp(4 * d["phi"])[:, None, None]
    np.testing.assert_allclose(e4 * (d["At"] + d["gt"] * d["K"][:, None, None] / 3), d["Kij"],
                               rtol=1e-12, atol=1e-14)
