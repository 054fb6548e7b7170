"""Pins of the oracle's spectral operators (Methods: "Grid Discretization",
"The Spectral Derivative Operators", "Dealiasing and Spectral Filtering").

Each check compares against something other than the oracle itself: numpy's
chebder (the routine the paper names), exactness on polynomials / trigonometric
polynomials, analytic derivatives, closed-form filter factors and quadrature rules.
"""
import numpy as np
import numpy.polynomial.chebyshev as npc
import pytest

from oracle import spectral as sp


def test_chebder_matches_numpy():
    rng = np.random.default_rng(1)
    for n in (2, 3, 8, 17):
        c = rng.normal(size=n)
        ref = npc.chebder(c)
        got = sp.chebder(c)
        assert got[-1] == 0.0
        np.testing.assert_allclose(got[:-1], ref, rtol=1e-14, atol=1e-13)


def test_nodes():
    x = sp.cgl_nodes(5)
    np.testing.assert_allclose(x, [-1, -np.sqrt(0.5), 0, np.sqrt(0.5), 1], atol=1e-15)
    # paper: r_j = mid + half cos(j pi/(N-1)); ours are the same set, ascending
    np.testing.assert_allclose(np.sort(np.cos(np.arange(7) * np.pi / 6)), sp.cgl_nodes(7),
                               atol=1e-15)
    xg = sp.gauss_nodes(4)
    assert np.all(np.abs(xg) < 1) and np.all(np.diff(xg) > 0)
    # roots of T_4
    np.testing.assert_allclose(npc.chebval(xg, [0, 0, 0, 0, 1]), 0, atol=1e-15)
    np.testing.assert_allclose(sp.fourier_nodes(4), [0, np.pi / 2, np.pi, 3 * np.pi / 2])


@pytest.mark.parametrize("nodes", ["cgl", "gauss"])
def test_cheb_deriv_exact_on_polynomials(nodes):
    n = 9
    x = sp.cgl_nodes(n) if nodes == "cgl" else sp.gauss_nodes(n)
    a, b = 1.8, 7.5
    y = 0.5 * (a + b) + 0.5 * (b - a) * x
    rng = np.random.default_rng(2)
    coef = rng.normal(size=n)           # degree n-1 polynomial in y (power basis)
    P = np.polynomial.Polynomial(coef)
    u = P(y)
    d1 = sp.cheb_deriv(u, x, axis=0, scale=2.0 / (b - a))
    d2 = sp.cheb_deriv(u, x, axis=0, scale=2.0 / (b - a), order=2)
    scale1 = np.abs(P.deriv()(y)).max()
    scale2 = np.abs(P.deriv(2)(y)).max()
    np.testing.assert_allclose(d1, P.deriv()(y), atol=1e-11 * scale1)
    np.testing.assert_allclose(d2, P.deriv(2)(y), atol=1e-10 * scale2)


def test_cheb_deriv_spectral_convergence_r():
    """f = e^{r/5} sin r on [1.8, 20]: error decays exponentially to a roundoff floor."""
    a, b = 1.8, 20.0
    errs = []
    for n in (8, 12, 16, 20, 24, 32):
        x = sp.cgl_nodes(n)
        r = 0.5 * (a + b) + 0.5 * (b - a) * x
        f = np.exp(r / 5) * np.sin(r)
        df = np.exp(r / 5) * (np.sin(r) / 5 + np.cos(r))
        d = sp.cheb_deriv(f, x, 0, scale=2 / (b - a))
        errs.append(np.abs(d - df).max() / np.abs(df).max())
    assert errs[0] > 1e-2
    assert all(e2 < e1 for e1, e2 in zip(errs[:4], errs[1:5]))
    assert errs[-1] < 1e-11


def test_cheb_deriv_spectral_convergence_theta():
    """cos^3(th) e^{sin th} on Gauss nodes of [0, pi]."""
    errs = []
    for n in (8, 16, 24, 32):
        x = sp.gauss_nodes(n)
        th = 0.5 * np.pi * (1 + x)
        f = np.cos(th) ** 3 * np.exp(np.sin(th))
        df = (-3 * np.cos(th) ** 2 * np.sin(th) + np.cos(th) ** 4) * np.exp(np.sin(th))
        d = sp.cheb_deriv(f, x, 0, scale=2 / np.pi)
        errs.append(np.abs(d - df).max())
    assert all(e2 < e1 for e1, e2 in zip(errs[:-1], errs[1:]))
    assert errs[-1] < 5e-11


def test_fourier_deriv():
    n = 32
    ph = sp.fourier_nodes(n)
    f = np.exp(np.sin(ph))
    d1 = sp.fourier_deriv(f, 0, 1)
    d2 = sp.fourier_deriv(f, 0, 2)
    np.testing.assert_allclose(d1, np.cos(ph) * f, atol=1e-12)
    np.testing.assert_allclose(d2, (np.cos(ph) ** 2 - np.sin(ph)) * f, atol=1e-12)
    # exact on trigonometric polynomials |k| < N/2, and agrees with numpy.fft
    rng = np.random.default_rng(3)
    n = 16
    ph = sp.fourier_nodes(n)
    u = np.zeros(n)
    du = np.zeros(n)
    for k in range(1, n // 2):
        a, b = rng.normal(size=2)
        u += a * np.cos(k * ph) + b * np.sin(k * ph)
        du += -a * k * np.sin(k * ph) + b * k * np.cos(k * ph)
    np.testing.assert_allclose(sp.fourier_deriv(u, 0), du, atol=1e-12)
    k = np.fft.fftfreq(n, 1.0 / n)
    k[n // 2] = 0
    ref = np.real(np.fft.ifft(1j * k * np.fft.fft(u)))
    np.testing.assert_allclose(sp.fourier_deriv(u, 0), ref, atol=1e-12)
    # the Nyquist mode has zero first derivative and -(N/2)^2 second derivative
    nyq = np.cos(n // 2 * ph)
    np.testing.assert_allclose(sp.fourier_deriv(nyq, 0, 1), 0, atol=1e-12)
    np.testing.assert_allclose(sp.fourier_deriv(nyq, 0, 2), -(n // 2) ** 2 * nyq, atol=1e-10)


def test_fourier_deriv_rounding_at_large_n():
    """The DFT table's phase is reduced modulo 2 pi exactly (integer k n mod N): at 64 and
    128 nodes the derivative of a single mode keeps the accuracy of the sums (a few
    1e-14 of its amplitude), where the unreduced angle (up to 2 pi N) would cost an order
    of magnitude more at low modes.  Checked against numpy's FFT too."""
    for n in (64, 128):
        ph = sp.fourier_nodes(n)
        for k in (1, 2, n // 4, n // 2 - 1):
            u = np.sin(k * ph + 0.3)
            d = sp.fourier_deriv(u, 0)
            assert np.abs(d - k * np.cos(k * ph + 0.3)).max() <= 1e-13 * k, (n, k)
            kk = np.fft.fftfreq(n, 1.0 / n)
            kk[n // 2] = 0
            ref = np.real(np.fft.ifft(1j * kk * np.fft.fft(u)))
            assert np.abs(d - ref).max() <= 1e-13 * k, (n, k)


def test_filters():
    # sigma(0) = 1 and sigma(k_max) = e^{-36}
    assert sp.filter_sigma(0.0, 5.0) == 1.0
    np.testing.assert_allclose(sp.filter_sigma(5.0, 5.0), np.exp(-36.0))
    # Fourier: a single mode is scaled by sigma(|k|); 2/3 rule removes |k| > N/3
    n = 24
    ph = sp.fourier_nodes(n)
    for k in (1, 5, 8, 9, 11):
        u = np.cos(k * ph)
        s = np.exp(-36 * (k / 12.0) ** 8) if k <= n / 3 else 0.0
        np.testing.assert_allclose(sp.fourier_filter(u, 0), s * u, atol=1e-13)
    # Chebyshev: T_k(x) scaled by sigma(k/(N-1)); constants are untouched
    m = 10
    x = sp.cgl_nodes(m)
    for k in (0, 3, 9):
        u = npc.chebval(x, np.eye(m)[k])
        s = np.exp(-36 * (k / (m - 1)) ** 8)
        np.testing.assert_allclose(sp.cheb_filter(u, x, 0), s * u, atol=1e-13)


def test_quadrature():
    for n in (5, 6, 9, 12):
        w = sp.clenshaw_curtis_weights(n)
        x = sp.cgl_nodes(n)
        # exact for polynomials of degree n-1
        for deg in range(n):
            exact = (1 - (-1) ** (deg + 1)) / (deg + 1)
            np.testing.assert_allclose(np.sum(w * x ** deg), exact, atol=1e-13)
        # closed-form end weight: 1/(m^2-1) for even m = n-1, 1/m^2 for odd m
        m = n - 1
        end = 1.0 / (m * m - 1) if m % 2 == 0 else 1.0 / (m * m)
        np.testing.assert_allclose(w[0], end, rtol=1e-13)
        np.testing.assert_allclose(w[-1], end, rtol=1e-13)
        wf = sp.fejer_weights(n)
        xg = sp.gauss_nodes(n)
        for deg in range(n):
            exact = (1 - (-1) ** (deg + 1)) / (deg + 1)
            np.testing.assert_allclose(np.sum(wf * xg ** deg), exact, atol=1e-13)
