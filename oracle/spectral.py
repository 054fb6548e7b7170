"""Spectral building blocks, written from the paper's Methods section
("Grid Discretization", "The Spectral Derivative Operators", "Dealiasing and
Spectral Filtering").  Test infrastructure only.

Chebyshev derivatives follow the paper's coefficient route: node values ->
Chebyshev coefficients (interpolation, a linear solve against T_k(x_j)) ->
coefficient-space differentiation (the `chebder` recurrence) -> evaluation at
the nodes.  Fourier derivatives follow the DFT definition with (i k)^d, written
as explicit O(N^2) sums.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------- nodes
def cgl_nodes(n: int) -> np.ndarray:
    """Chebyshev-Gauss-Lobatto nodes on [-1, 1] in ascending order.

    The paper's radial grid (Methods, "Radial Chebyshev-Gauss-Lobatto grid") is
    x_j = cos(j pi / (N_r - 1)), j = 0..N_r-1 (descending); we store them ascending,
    x_i = -cos(i pi / (n - 1))."""
    i = np.arange(n)
    return -np.cos(i * np.pi / (n - 1))


def gauss_nodes(n: int) -> np.ndarray:
    """Chebyshev-Gauss (interior) nodes on [-1, 1], ascending: x_k = -cos((2k+1) pi/(2n)).

    Used for theta: a Chebyshev grid in theta without nodes on the poles (the
    paper's uniform theta grid with a Fourier derivative is replaced by this;
    a reading of the paper)."""
    k = np.arange(n)
    return -np.cos((2 * k + 1) * np.pi / (2 * n))


def fourier_nodes(n: int) -> np.ndarray:
    """phi_l = 2 pi l / N_phi (Methods, uniform azimuthal grid)."""
    return 2.0 * np.pi * np.arange(n) / n


# ------------------------------------------------------------------------ chebyshev
def cheb_T(x: np.ndarray, n: int) -> np.ndarray:
    """Matrix T[j, k] = T_k(x_j), k = 0..n-1, by the three-term recurrence."""
    x = np.asarray(x)
    T = np.empty(x.shape + (n,), dtype=np.result_type(x, np.float64))
    T[..., 0] = 1.0
    if n > 1:
        T[..., 1] = x
    for k in range(2, n):
        T[..., k] = 2.0 * x * T[..., k - 1] - T[..., k - 2]
    return T


def chebder(c: np.ndarray, axis: int = 0) -> np.ndarray:
    """Coefficients of the derivative of sum_k c_k T_k(x) (same length, last entry 0).

    Recurrence d_{k-1} = d_{k+1} + 2 k c_k for k = n-1 .. 1, then d_0 /= 2
    (the coefficient-space differentiation the paper performs with numpy's chebder).
    """
    c = np.moveaxis(np.asarray(c), axis, 0)
    n = c.shape[0]
    d = np.zeros_like(c)
    for k in range(n - 1, 0, -1):
        nxt = d[k + 1] if k + 1 < n else 0.0
        d[k - 1] = nxt + 2.0 * k * c[k]
    d[0] = d[0] / 2.0
    return np.moveaxis(d, 0, axis)


def cheb_coeffs(u: np.ndarray, x: np.ndarray, axis: int) -> np.ndarray:
    """Chebyshev coefficients of the degree-(n-1) interpolant of u at nodes x along axis."""
    n = x.shape[0]
    V = cheb_T(x, n)
    um = np.moveaxis(u, axis, 0)
    c = np.linalg.solve(V, um.reshape(n, -1)).reshape(um.shape)
    return np.moveaxis(c, 0, axis)


def cheb_eval(c: np.ndarray, x: np.ndarray, axis: int) -> np.ndarray:
    """Evaluate sum_k c_k T_k at the nodes x along axis."""
    n = x.shape[0]
    V = cheb_T(x, n)
    cm = np.moveaxis(c, axis, 0)
    u = (V @ cm.reshape(n, -1)).reshape(cm.shape)
    return np.moveaxis(u, 0, axis)


def cheb_deriv(u: np.ndarray, x: np.ndarray, axis: int, scale: float = 1.0, order: int = 1):
    """d^order u / dy^order along axis, with y = y0 + x / scale (scale = 2/(b - a)).

    Coefficient route of the paper's "Radial Chebyshev Spectral Derivative":
    interpolate, apply chebder `order` times, evaluate back at the nodes."""
    c = cheb_coeffs(u, x, axis)
    for _ in range(order):
        c = chebder(c, axis=axis) * scale
    return cheb_eval(c, x, axis)


# -------------------------------------------------------------------------- fourier
def fourier_wavenumbers(n: int) -> np.ndarray:
    """k = 0, 1, ..., n/2, -n/2+1, ..., -1 (the paper's ordering)."""
    k = np.arange(n)
    return np.where(k <= n // 2, k, k - n)


def dft(u: np.ndarray, axis: int) -> np.ndarray:
    """hat U_k = sum_n U_n exp(-2 pi i k n / N) as an explicit O(N^2) sum.

    The phase k n / N is reduced modulo 1 in integers (k n mod N) before it is scaled by
    2 pi: the same table entry, but the angle stays below 2 pi, so each entry is accurate
    to the unit roundoff (with the unreduced angle, up to 2 pi N, its rounding grows in
    proportion to N)."""
    n = u.shape[axis]
    jj = np.arange(n)
    F = np.exp(-2j * np.pi * (np.outer(jj, jj) % n) / n)
    um = np.moveaxis(u, axis, 0)
    U = (F @ um.reshape(n, -1)).reshape(um.shape)
    return np.moveaxis(U, 0, axis)


def idft(U: np.ndarray, axis: int) -> np.ndarray:
    """U_n = (1/N) sum_k hat U_k exp(+2 pi i k n / N)."""
    n = U.shape[axis]
    jj = np.arange(n)
    F = np.exp(2j * np.pi * (np.outer(jj, jj) % n) / n) / n          # phase reduced as in dft
    Um = np.moveaxis(U, axis, 0)
    u = (F @ Um.reshape(n, -1)).reshape(Um.shape)
    return np.moveaxis(u, 0, axis)


def fourier_deriv(u: np.ndarray, axis: int, order: int = 1) -> np.ndarray:
    """d^order u / dphi^order on the periodic uniform grid: multiply hat U_k by (i k)^d.

    For even N and odd d the Nyquist mode k = N/2 has no real derivative and is
    zeroed (reading of the paper's wavenumber list; the mode is not
    distinguishable from -N/2 on the grid)."""
    n = u.shape[axis]
    k = fourier_wavenumbers(n).astype(np.float64)
    mult = (1j * k) ** order
    if order % 2 == 1 and n % 2 == 0:
        mult[n // 2] = 0.0
    U = dft(u, axis)
    shape = [1] * u.ndim
    shape[axis] = n
    return np.real(idft(U * mult.reshape(shape), axis))


# -------------------------------------------------------------------------- filters
def filter_sigma(k_abs: np.ndarray, k_max: float, alpha: float = 36.0, p: float = 8.0):
    """Exponential filter sigma(k) = exp(-alpha (|k|/k_max)^p), alpha = 36, p = 8
    (Methods, "Dealiasing and Spectral Filtering")."""
    return np.exp(-alpha * (np.abs(k_abs) / k_max) ** p)


def cheb_filter(u, x, axis, alpha=36.0, p=8.0, dealias23=False):
    """Filter the Chebyshev modal coefficients k = 0..N-1 with k_max = N-1."""
    n = x.shape[0]
    c = cheb_coeffs(u, x, axis)
    k = np.arange(n, dtype=np.float64)
    s = filter_sigma(k, n - 1, alpha, p)
    if dealias23:
        s = np.where(k > (n - 1) / 3.0 * 2.0, 0.0, s)
    shape = [1] * u.ndim
    shape[axis] = n
    return cheb_eval(c * s.reshape(shape), x, axis)


def fourier_filter(u, axis, alpha=36.0, p=8.0, dealias23=True):
    """Filter Fourier modes with k_max = N/2; with dealias23, zero |k| > N/3 (2/3 rule)."""
    n = u.shape[axis]
    k = np.abs(fourier_wavenumbers(n)).astype(np.float64)
    s = filter_sigma(k, n / 2.0, alpha, p)
    if dealias23:
        s = np.where(k > n / 3.0, 0.0, s)
    shape = [1] * u.ndim
    shape[axis] = n
    return np.real(idft(dft(u, axis) * s.reshape(shape), axis))


# ------------------------------------------------------------------------ quadrature
def clenshaw_curtis_weights(n: int) -> np.ndarray:
    """Clenshaw-Curtis weights on [-1, 1] for the n CGL nodes: the integrals of the
    Lagrange interpolants, obtained from the exact integrals of T_k,
    int T_k = 2/(1-k^2) for even k, 0 for odd k."""
    x = cgl_nodes(n)
    V = cheb_T(x, n)
    k = np.arange(n)
    mom = np.where(k % 2 == 0, 2.0 / (1.0 - k.astype(float) ** 2 + (k % 2)), 0.0)
    # w solves V^T w = mom (sum_j w_j T_k(x_j) = int T_k)
    return np.linalg.solve(V.T, mom)


def fejer_weights(n: int) -> np.ndarray:
    """Fejer's first rule on the n Chebyshev-Gauss nodes, by the same moment system."""
    x = gauss_nodes(n)
    V = cheb_T(x, n)
    k = np.arange(n)
    mom = np.where(k % 2 == 0, 2.0 / (1.0 - k.astype(float) ** 2 + (k % 2)), 0.0)
    return np.linalg.solve(V.T, mom)


# ------------------------------------------------------------ Fourier theta (double Fourier)
def uniform_theta_nodes(n: int) -> np.ndarray:
    """theta_k = (k + 1/2) pi / n, k = 0..n-1: the paper's uniform polar grid on [0, pi]
    ("Grid Discretization", "Pseudo-spectral theta derivative") shifted by half a spacing,
    so that no node lies on the axis, where the spherical metric is singular (reading:
    the printed k pi / (N_theta - 1) puts the first and last node on the poles)."""
    return (np.arange(n) + 0.5) * np.pi / n


def parity_extend(u: np.ndarray, axis_t: int, axis_p: int, parity) -> np.ndarray:
    """Periodic line of length 2n over theta in [0, 2 pi) (double Fourier sphere).

    The point (2 pi - theta, phi) of the extended torus is the point (theta, phi + pi)
    of the sphere, reached across a pole; a component with parity s (s = -1 for each
    theta index, and once more for a sqrt(gamma)-weighted density, which behaves like
    sin(theta) on the axis) takes the value s u(theta, phi + pi) there.  The nodes
    2 pi - theta_k are the extended nodes n + (n - 1 - k), so the second half is the
    phi-shifted line in reversed order."""
    n_p = u.shape[axis_p]
    partner = np.roll(u, -(n_p // 2), axis=axis_p)          # value at phi + pi
    mirrored = np.flip(partner, axis=axis_t) * parity
    return np.concatenate([u, mirrored], axis=axis_t)


def fourier_theta_deriv(u, axis_t: int, axis_p: int, parity, order: int = 1):
    """d^order u / dtheta^order: the paper's Fourier derivative ((i k)^d on the DFT) of
    the parity-extended line, read back on the n nodes of (0, pi)."""
    n = u.shape[axis_t]
    g = parity_extend(u, axis_t, axis_p, parity)
    return np.take(fourier_deriv(g, axis=axis_t, order=order), np.arange(n), axis=axis_t)


def fourier_theta_filter(u, axis_t: int, axis_p: int, parity, alpha=36.0, p=8.0, dealias23=True):
    """Exponential filter (k_max = n, the Nyquist number of the 2n extended nodes) and the
    2/3 rule (|k| > 2n/3 zeroed) on the parity-extended line, read back on (0, pi)."""
    n = u.shape[axis_t]
    g = parity_extend(u, axis_t, axis_p, parity)
    return np.take(fourier_filter(g, axis=axis_t, alpha=alpha, p=p, dealias23=dealias23),
                   np.arange(n), axis=axis_t)


def fourier_theta_weights(n: int) -> np.ndarray:
    """Quadrature of int_0^pi f dtheta on the uniform nodes for f = sin(theta) g(cos theta):
    with x = -cos(theta) the nodes are the Chebyshev-Gauss points, and the integral is
    int_{-1}^{1} f / sin(theta) dx, so w_k = (Fejer weight)_k / sin(theta_k)."""
    return fejer_weights(n) / np.sin(uniform_theta_nodes(n))
